// Steps 2-4 of the cell-graph construction around the sort: hash-based
// duplicate removal (§3.2: duplicates of X are removed so that each pair is
// output once, §2.2), the Hamming-1 search (Algorithm 4: flip one bit of a cell,
// look the result up) and the compaction of hits into the edge list.
//
// Vectors of l <= 64 bits are handled as single 64-bit words ("small"): the
// tables hold the vectors themselves. Longer vectors ("wide", W = ceil(l/64)
// words) are referenced by row number; their lookup table is keyed on a
// GF(2)-linear fingerprint, so the fingerprint of a one-bit change is one XOR
// away, and every fingerprint match is verified word by word.
//
// Every kernel after the dedup step reads U from device memory and returns
// early if the dedup step overflowed its capacity.
#include "../../include/cellgraph.h"
#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

int grid_for(size_t items, int per_block, int blocks_per_sm = 8) {
  const size_t want = (items + per_block - 1) / per_block;
  const size_t cap = size_t(sm_count()) * blocks_per_sm;
  size_t g = want < cap ? want : cap;
  return int(g < 1 ? 1 : g);
}

// 64-bit word j of row r of a caller-layout array of ceil(l/word_bits) words.
__device__ __forceinline__ uint64_t load_word(const void* base, int64_t r, int j, int word_bits,
                                              int w_caller) {
  if (word_bits == 64) return static_cast<const uint64_t*>(base)[r * w_caller + j];
  const uint32_t* p = static_cast<const uint32_t*>(base) + r * w_caller;
  const uint64_t lo = p[2 * j];
  const uint64_t hi = (2 * j + 1 < w_caller) ? p[2 * j + 1] : 0u;
  return lo | (hi << 32);
}

// ------------------------------- utilities -------------------------------

__global__ void fill_u64(uint64_t* p, uint64_t v, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

__global__ void zero_counters(DevCounters* c) {
  if (threadIdx.x < sizeof(DevCounters) / 4) reinterpret_cast<uint32_t*>(c)[threadIdx.x] = 0;
}

// Bits >= l of a caller's row are ignored (cleared on load).
__device__ __forceinline__ uint64_t valid_bits(int j, int w64, int ell) {
  return (j == w64 - 1 && (ell & 63)) ? ((1ull << (ell & 63)) - 1) : ~0ull;
}

__global__ void keys_to_u64(const void* keys, int64_t n, int word_bits, int w_caller, int w64,
                            int ell, uint64_t* out) {
  const int64_t total = n * w64;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / w64;
    const int j = int(t - r * w64);
    out[t] = load_word(keys, r, j, word_bits, w_caller) & valid_bits(j, w64, ell);
  }
}

// A caller's cells must have every bit at or above l clear: a set one is
// reported (kErrHighBits) rather than cleared, so the same bad row is refused
// whatever the word width and whether or not the rows are read in place.
__global__ void load_cells(const void* cells, int64_t n, int word_bits, int w_caller, int w64,
                           int ell, uint64_t* out, DevCounters* ctr) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_unique = unsigned(n);
  const int64_t total = n * w64;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / w64;
    const int j = int(t - r * w64);
    const uint64_t raw = load_word(cells, r, j, word_bits, w_caller);
    const uint64_t kept = raw & valid_bits(j, w64, ell);
    if (kept != raw) atomicOr(&ctr->error, kErrHighBits);
    out[t] = kept;
  }
}

__global__ void write_cells(const uint64_t* cells, int w64, int word_bits, int w_caller,
                            void* out, int64_t cap, const DevCounters* ctr,
                            const unsigned int* skip) {
  if (ctr->overflow || (skip && *skip)) return;
  const int64_t u = ctr->n_unique;
  if (u > cap) return;  // capacity error: the host reports it, nothing is written
  const int64_t total = u * w_caller;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / w_caller;
    const int j = int(t - r * w_caller);
    if (word_bits == 64) {
      static_cast<uint64_t*>(out)[t] = cells[r * w64 + j];
    } else {
      static_cast<uint32_t*>(out)[t] = uint32_t(cells[r * w64 + j / 2] >> (32 * (j & 1)));
    }
  }
}

// ------------------------------- small path ------------------------------

struct SmallHash {
  const uint64_t* keys;
  const uint32_t* vals;
  uint32_t mask;
  int shift;
  const DevCounters* ctr;
  __device__ __forceinline__ int64_t find(uint64_t y) const {
    if (y == kEmpty) return ctr->ones_present ? int64_t(ctr->ones_rank) : -1;
    uint32_t slot = home_slot(y, shift);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const uint64_t cur = keys[slot];
      if (cur == y) return vals[slot];
      if (cur == kEmpty) return -1;
      slot = (slot + 1) & mask;
    }
    return -1;
  }
};

struct SmallSorted {
  const uint64_t* cells;
  const DevCounters* ctr;
  __device__ __forceinline__ int64_t find(uint64_t y) const {
    uint32_t lo = 0, hi = ctr->n_unique;
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      const uint64_t v = cells[mid];
      if (v < y) lo = mid + 1;
      else hi = mid;
    }
    return (lo < ctr->n_unique && cells[lo] == y) ? int64_t(lo) : -1;
  }
};

__global__ void insert_small(const void* keys, int64_t n, int word_bits, int w_caller,
                             SmallTable t) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n;
       p += int64_t(gridDim.x) * blockDim.x)
    small_insert(t, load_word(keys, p, 0, word_bits, w_caller));
}


__global__ void rank_small(const uint64_t* cells, SmallTable t) {
  if (t.ctr->overflow) return;
  const uint32_t u = t.ctr->n_unique;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint64_t key = cells[i];
    if (key == kEmpty) {
      t.ctr->ones_rank = i;
      continue;
    }
    const int64_t slot = small_find_slot(t.keys, t.mask, t.shift, key);
    if (slot < 0) {
      atomicOr(&t.ctr->error, 1u);
      continue;
    }
    t.vals[slot] = i;
  }
}

__global__ void index_small(const uint64_t* cells, SmallTable t) {
  const uint32_t u = t.ctr->n_unique;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint64_t key = cells[i];
    if (key == kEmpty) {
      t.ctr->ones_present = 1u;
      t.ctr->ones_rank = i;
      continue;
    }
    uint32_t slot = home_slot(key, t.shift);
    bool placed = false;
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
      const unsigned long long old =
          atomicCAS(reinterpret_cast<unsigned long long*>(t.keys + slot),
                    static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(key));
      if (old == kEmpty) {
        t.vals[slot] = i;
        placed = true;
        break;
      }
      if (old == key) break;  // repeated cell: input is not unique
      slot = (slot + 1) & t.mask;
    }
    if (!placed) atomicOr(&t.ctr->error, 2u);
  }
}

__global__ void point_cell_small(const void* keys, int64_t n, int word_bits, int w_caller,
                                 SmallTable t, uint32_t* point_cell) {
  if (t.ctr->overflow) return;
  const SmallHash h{t.keys, t.vals, t.mask, t.shift, t.ctr};
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = h.find(load_word(keys, p, 0, word_bits, w_caller));
    if (j < 0) atomicOr(&t.ctr->error, 4u);
    point_cell[p] = uint32_t(j);
  }
}

// One warp per cell; lane l of chunk h tests bit k = 32h + l (Algorithm 4,
// one thread per bit). Only zero bits are flipped, so each edge is found once,
// from its smaller endpoint.
template <class L>
__global__ void __launch_bounds__(kThreads)
    neighbors_small(const uint64_t* __restrict__ cells, L look, const DevCounters* ctr, int ell,
                    uint32_t* __restrict__ masks, uint32_t* __restrict__ counts) {
  if (ctr->overflow) return;
  const uint32_t u = ctr->n_unique;
  const int nh = (ell + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    const uint64_t x = cells[i];
    uint32_t total = 0;
    for (int h = 0; h < nh; ++h) {
      const int k = h * 32 + lane;
      bool hit = false;
      if (k < ell && !((x >> k) & 1ull)) hit = look.find(x | (1ull << k)) >= 0;
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) masks[uint64_t(i) * nh + h] = m;
      total += __popc(m);
    }
    if (lane == 0) counts[i] = total;
  }
}

template <class L>
__global__ void __launch_bounds__(kThreads)
    emit_small(const uint64_t* __restrict__ cells, L look, DevCounters* ctr, int ell,
               const uint32_t* __restrict__ masks, const unsigned long long* __restrict__ offsets,
               uint32_t* __restrict__ edges, int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = ctr->n_unique;
  const int nh = (ell + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    const uint64_t x = cells[i];
    unsigned long long off = offsets[i];
    for (int h = 0; h < nh; ++h) {
      const uint32_t m = masks[uint64_t(i) * nh + h];
      if ((m >> lane) & 1u) {
        const int k = h * 32 + lane;
        const int64_t j = look.find(x | (1ull << k));
        if (j < 0) atomicOr(&ctr->error, 8u);
        const unsigned long long r = off + __popc(m & lanemask_lt());
        if (r < (unsigned long long)cap) {
          edges[2 * r] = i;
          edges[2 * r + 1] = uint32_t(j);
        }
      }
      off += __popc(m);
    }
  }
}

__global__ void clear_build(uint64_t* table, size_t cap, uint64_t* table2, size_t cap2,
                            unsigned long long* status, size_t n_status, DevCounters* ctr,
                            uint32_t* zero32, size_t n_zero32) {
  griddep_wait();  // the previous build's kernels may still read this table
  griddep_release();
  if (blockIdx.x == 0 && threadIdx.x < sizeof(DevCounters) / 4)
    reinterpret_cast<uint32_t*>(ctr)[threadIdx.x] = 0;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < cap; i += stride)
    table[i] = kEmpty;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < cap2; i += stride)
    table2[i] = kEmpty;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n_status; i += stride)
    status[i] = 0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n_zero32; i += stride)
    zero32[i] = 0;
}

// Steps 3-4 in one pass (l <= 64). Work is handed out in chunks of 32 cells
// by an atomic ticket, so every chunk's predecessors are already running.
// For a chunk: the warps find the hits of their cells (one lane per bit, hits
// kept in shared memory), warp 0 scans the 32 counts, publishes the chunk's
// total, and looks back over the predecessors' published totals (decoupled
// look-back, Merrill & Garland 2016) for the chunk's first edge position;
// then the block writes its edges. The look-back wait is bounded.
constexpr int kNEThreads = 256;
constexpr int kNECells = 32;
// Blocks of the one-word kernels: one warp per cell of a chunk, so a chunk's
// table probes are all in flight at once (with 256 threads each warp walked 4
// cells one after another: 16 dependent L2 round trips per chunk).
constexpr int kNESmallThreads = 32 * kNECells;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
// Polls of the look-back before it gives up (a wait that can never end).
constexpr unsigned kSpinLimit = 1u << 22;

struct EmitShared {
  uint32_t hits[kNECells][64];
  uint32_t cnt[kNECells];
  uint32_t off[kNECells];
  uint32_t chunk;
  unsigned long long base;
};

// Chunk c (< nchunks) of the U = u sorted cells: every warp finds the hits of
// its cells (one lane per bit, kept in shared memory), warp 0 scans the 32
// counts, publishes the chunk's total and looks back over the predecessors'
// totals (decoupled look-back, Merrill & Garland 2016; at most `polls` polls)
// for the chunk's first edge position, then the block writes its edges.
// Called by the whole block.
template <class L, int T = kNESmallThreads>
__device__ __forceinline__ void emit_small_chunk(EmitShared& sm,
                                                 const uint64_t* __restrict__ cells, const L& look,
                                                 DevCounters* ctr, int ell,
                                                 unsigned long long* status,
                                                 uint32_t* __restrict__ edges, int64_t cap,
                                                 uint32_t u, uint32_t nchunks, uint32_t c,
                                                 uint32_t polls) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nh = (ell + 31) >> 5;
  for (int cl = warp; cl < kNECells; cl += T / 32) {
    const uint32_t i = c * kNECells + cl;
    uint32_t total = 0;
    if (i < u) {
      const uint64_t x = cells[i];
      for (int h = 0; h < nh; ++h) {
        const int k = h * 32 + lane;
        int64_t j = -1;
        if (k < ell && !((x >> k) & 1ull)) j = look.find(x | (1ull << k));
        const uint32_t m = __ballot_sync(0xffffffffu, j >= 0);
        if (j >= 0) sm.hits[cl][total + __popc(m & lanemask_lt())] = uint32_t(j);
        total += __popc(m);
      }
    }
    if (lane == 0) sm.cnt[cl] = total;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = sm.cnt[lane];
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    sm.off[lane] = inc - v;
    const unsigned long long T = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) {
      unsigned long long base = 0;
      if (c == 0) {
        atomicExch(&status[0], kFlagPre | T);
      } else {
        atomicExch(&status[c], kFlagAgg | T);
        int64_t p = int64_t(c) - 1;
        uint32_t looked = 0;
        while (p >= 0) {
          if (looked++ >= polls) {  // every look counts; 0 polls gives up at once
            atomicOr(&ctr->error, kErrTimeout);
            break;
          }
          const unsigned long long sv =
              *reinterpret_cast<volatile unsigned long long*>(&status[p]);
          const unsigned long long f = sv & ~kValMask;
          if (f == 0) {
            __nanosleep(64);
            continue;
          }
          base += sv & kValMask;
          if (f == kFlagPre) break;
          --p;
        }
        atomicExch(&status[c], kFlagPre | (base + T));
      }
      sm.base = base;
      if (c == nchunks - 1) ctr->n_edges = base + T;
    }
  }
  __syncthreads();
  const unsigned long long base = sm.base;
  for (int cl = warp; cl < kNECells; cl += T / 32) {
    const uint32_t i = c * kNECells + cl;
    const uint32_t m = sm.cnt[cl];
    const unsigned long long o = base + sm.off[cl];
    for (uint32_t r = lane; r < m; r += 32) {
      const unsigned long long e = o + r;
      if (e < (unsigned long long)cap) {
        edges[2 * e] = i;
        edges[2 * e + 1] = sm.hits[cl][r];
      }
    }
  }
  __syncthreads();
}

template <class L>
__global__ void __launch_bounds__(kNESmallThreads)
    neighbors_emit_small(const uint64_t* __restrict__ cells, L look, DevCounters* ctr, int ell,
                         unsigned long long* status, uint32_t* __restrict__ edges, int64_t cap,
                         uint32_t max_n, uint32_t polls) {
  __shared__ EmitShared sm;
  griddep_wait();
  griddep_release();
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint32_t nchunks = (u + kNECells - 1) / kNECells;
  for (;;) {
    if (threadIdx.x == 0) sm.chunk = atomicAdd(&ctr->ticket, 1u);
    __syncthreads();
    const uint32_t c = sm.chunk;
    if (c >= nchunks) break;
    emit_small_chunk(sm, cells, look, ctr, ell, status, edges, cap, u, nchunks, c, polls);
  }
}

// ------------------------- many scenes per launch -------------------------
//
// Batches: the single-pass edge kernel over the chunks of every scene of
// l <= 64 at once. A global ticket hands out (scene, chunk) items in scene
// order, so every chunk's predecessors in its own scene were handed out
// earlier and are running; the look-back stays within the scene's own status
// words, and each scene's last chunk writes its edge count.
__global__ void __launch_bounds__(1024)
    seg_emit_offsets(const SegSearchScene* __restrict__ sc, int n_scenes, unsigned int* off) {
  __shared__ unsigned long long wsum[32];
  unsigned long long carry = 0;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (int base = 0; base < n_scenes; base += 1024) {
    const int i = base + int(threadIdx.x);
    unsigned long long c = 0;
    if (i < n_scenes && !sc[i].t.ctr->overflow)
      c = (min(sc[i].t.ctr->n_unique, sc[i].ucap) + kNECells - 1) / kNECells;
    unsigned long long inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      unsigned long long v = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      wsum[lane] = v;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? wsum[warp - 1] : 0ull;
    if (i < n_scenes) off[i] = unsigned(carry + before + inc - c);
    carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[n_scenes] = unsigned(carry);  // chunks in all
    off[n_scenes + 1] = 0u;           // ticket
  }
}

template <bool kSorted>
__global__ void __launch_bounds__(kNESmallThreads)
    neighbors_seg_small(const SegSearchScene* __restrict__ sc, int n_scenes, unsigned int* off,
                        uint32_t polls) {
  __shared__ EmitShared sm;
  const uint32_t total = off[n_scenes];
  for (;;) {
    if (threadIdx.x == 0) sm.chunk = atomicAdd(&off[n_scenes + 1], 1u);
    __syncthreads();
    const uint32_t g = sm.chunk;
    if (g >= total) break;
    int lo = 0, hi = n_scenes - 1;  // the last scene whose first chunk is <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const SegSearchScene& z = sc[lo];
    const uint32_t u = min(z.t.ctr->n_unique, z.ucap);
    const uint32_t nchunks = (u + kNECells - 1) / kNECells;
    if (kSorted)
      emit_small_chunk(sm, z.cells, SmallSorted{z.cells, z.t.ctr}, z.t.ctr, z.ell, z.status,
                       z.edges, z.edges_cap, u, nchunks, g - off[lo], polls);
    else
      emit_small_chunk(sm, z.cells, SmallHash{z.t.keys, z.t.vals, z.t.mask, z.t.shift, z.t.ctr},
                       z.t.ctr, z.ell, z.status, z.edges, z.edges_cap, u, nchunks, g - off[lo],
                       polls);
  }
}

// One block per scene: its table (kEmpty), table values and look-back words
// (zero) and counters.
__global__ void __launch_bounds__(1024) clear_seg(const SegClear* __restrict__ sc) {
  const SegClear& z = sc[blockIdx.x];
  if (threadIdx.x < sizeof(DevCounters) / 4) reinterpret_cast<uint32_t*>(z.ctr)[threadIdx.x] = 0;
  for (size_t i = threadIdx.x; i < z.cap; i += blockDim.x) {
    z.keys[i] = kEmpty;
    if (z.vals) z.vals[i] = 0u;
  }
  for (size_t i = threadIdx.x; i < z.cap2; i += blockDim.x) z.keys2[i] = kEmpty;
  for (size_t i = threadIdx.x; i < z.n_status; i += blockDim.x) z.status[i] = 0ull;
}

// ------------------------------- wide path -------------------------------

// Row hash: every word mixed on its own (salted by its position) and the
// results folded, so that the multiplies of different words overlap instead
// of forming one dependent chain through the row.
__device__ __forceinline__ uint64_t hash_row(const uint64_t* r, int w) {
  uint64_t h = 0x9e3779b97f4a7c15ull * uint64_t(w);
#pragma unroll 4
  for (int j = 0; j < w; ++j) h ^= mix64(r[j] + 0xd1b54a32d192ed03ull * uint64_t(j + 1));
  return mix64(h);
}

__device__ __forceinline__ bool rows_equal(const uint64_t* x, const uint64_t* y, int w) {
  for (int j = 0; j < w; ++j)
    if (x[j] != y[j]) return false;
  return true;
}

// Insertion of row p (kp: its words, in global or shared memory) into the
// table of distinct rows; a row found equal to a stored one is dropped.
__device__ __forceinline__ void insert_row(const uint64_t* __restrict__ keys, int w,
                                           const WideTable& t, int64_t p, const uint64_t* kp) {
  const uint64_t h = hash_row(kp, w);
  const uint32_t tag = uint32_t(h >> 32);
  const uint64_t entry = (uint64_t(tag) << 32) | uint64_t(p);
  uint32_t slot = uint32_t(h) & t.mask;
  for (uint32_t probe = 0; probe <= t.mask; ++probe) {
    uint64_t cur = t.slots[slot];
    if (cur == kEmpty) {
      cur = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + slot),
                      static_cast<unsigned long long>(kEmpty),
                      static_cast<unsigned long long>(entry));
      if (cur == kEmpty) {
        const unsigned int idx = atomicAdd(&t.ctr->n_unique, 1u);
        if (idx < t.ucap) {
          t.ulist[idx] = uint32_t(p);
          if (t.ukeys) {
            const ulonglong2 k = top128(kp, t.ell);
            t.ukeys[idx] = k;
            atomicAdd(&t.bucket_count[t.bucket_bits ? uint32_t(k.x >> (64 - t.bucket_bits)) : 0u],
                      1u);
          }
        } else {
          atomicOr(&t.ctr->overflow, 1u);
        }
        return;
      }
    }
    if (uint32_t(cur >> 32) == tag && rows_equal(keys + uint64_t(uint32_t(cur)) * w, kp, w))
      return;
    slot = (slot + 1) & t.mask;
  }
  atomicOr(&t.ctr->overflow, 1u);
}

__global__ void insert_wide(const uint64_t* __restrict__ keys, int64_t n, int w, WideTable t) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n;
       p += int64_t(gridDim.x) * blockDim.x)
    insert_row(keys, w, t, p, keys + p * w);
}

// The inserts of many scenes: point g of the batch numbering belongs to the
// last scene whose p0 is <= g (binary search over the scene table).
__global__ void insert_wide_seg(const SegInsertWide* __restrict__ sc, int n_scenes,
                                uint64_t total) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < total;
       g += uint64_t(gridDim.x) * blockDim.x) {
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sc[mid].p0 <= g) lo = mid;
      else hi = mid - 1;
    }
    const SegInsertWide& z = sc[lo];
    const int64_t p = int64_t(g - z.p0);
    if (p < z.n) insert_row(z.keys64, z.w, z.t, p, z.keys64 + p * z.w);
  }
}

// Rows idx[0 .. U) of keys, in that order, to out (nothing when out_cap >= 0
// and U > out_cap: the caller reports the capacity error).
__global__ void gather_rows(const uint64_t* __restrict__ keys, int w,
                            const uint32_t* __restrict__ idx, const unsigned int* n_dev,
                            uint32_t max_n, uint64_t* __restrict__ out,
                            const unsigned int* skip, int64_t out_cap) {
  if (skip && *skip) return;
  const uint32_t u = min(*n_dev, max_n);
  if (out_cap >= 0 && int64_t(u) > out_cap) return;
  const uint64_t total = uint64_t(u) * w;
  if (total < (1ull << 32)) {  // 32-bit index arithmetic
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < uint32_t(total);
         t += gridDim.x * blockDim.x) {
      const uint32_t r = t / uint32_t(w);
      out[t] = keys[uint64_t(idx[r]) * w + (t - r * uint32_t(w))];
    }
    return;
  }
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < total;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = t / w;
    out[t] = keys[uint64_t(idx[r]) * w + (t - r * w)];
  }
}

__global__ void rank_by_row(const uint32_t* __restrict__ idx, const unsigned int* n_dev,
                            uint32_t max_n, uint32_t* __restrict__ rank) {
  const uint32_t n = min(*n_dev, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rank[idx[i]] = i;
}

__global__ void point_cell_wide(const uint64_t* __restrict__ keys, int64_t n, int w, WideTable t,
                                const uint32_t* __restrict__ rank, uint32_t* point_cell) {
  if (t.ctr->overflow) return;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n;
       p += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t* kp = keys + p * w;
    const uint64_t h = hash_row(kp, w);
    const uint32_t tag = uint32_t(h >> 32);
    uint32_t slot = uint32_t(h) & t.mask;
    int64_t found = -1;
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
      const uint64_t cur = t.slots[slot];
      if (cur == kEmpty) break;
      if (uint32_t(cur >> 32) == tag && rows_equal(keys + uint64_t(uint32_t(cur)) * w, kp, w)) {
        found = uint32_t(cur);
        break;
      }
      slot = (slot + 1) & t.mask;
    }
    if (found < 0) atomicOr(&t.ctr->error, 16u);
    point_cell[p] = found < 0 ? 0xffffffffu : rank[found];
  }
}

// Per-block table of fp_bit(k) for k < l in shared memory.
__device__ __forceinline__ void load_fp_bits(uint64_t* hbits, int ell) {
  for (int k = threadIdx.x; k < ell; k += blockDim.x) hbits[k] = fp_bit(k);
  __syncthreads();
}

// Fingerprint of every cell (warp per cell, lanes over words) and insertion
// of (fingerprint tag, cell number) into the table.
__global__ void __launch_bounds__(kThreads)
    index_wide(const uint64_t* __restrict__ cells, int w, int ell, WideTable t,
               uint64_t* __restrict__ fp) {
  extern __shared__ uint64_t hbits[];
  load_fp_bits(hbits, ell);
  if (t.ctr->overflow) return;
  const uint32_t u = t.ctr->n_unique;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    uint64_t f = 0;
    for (int j = lane; j < w; j += 32) {
      uint64_t x = cells[uint64_t(i) * w + j] & valid_bits(j, w, ell);
      while (x) {
        const int b = __ffsll(static_cast<long long>(x)) - 1;
        f ^= hbits[64 * j + b];
        x &= x - 1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f ^= __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) {
      fp[i] = f;
      const uint64_t entry = (f & 0xffffffff00000000ull) | uint64_t(i);
      uint32_t slot = uint32_t(f) & t.mask;
      bool placed = false;
      for (uint32_t probe = 0; probe <= t.mask; ++probe) {
        const unsigned long long old = atomicCAS(
            reinterpret_cast<unsigned long long*>(t.slots + slot),
            static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(entry));
        if (old == kEmpty) {
          placed = true;
          break;
        }
        slot = (slot + 1) & t.mask;
      }
      if (!placed) atomicOr(&t.ctr->overflow, 1u);
    }
  }
}

// Does cells[j] equal cells[i] with bit k flipped?
__device__ __forceinline__ bool is_flip(const uint64_t* cells, int w, uint32_t i, uint32_t j,
                                        int k) {
  const uint64_t* xi = cells + uint64_t(i) * w;
  const uint64_t* xj = cells + uint64_t(j) * w;
  for (int q = 0; q < w; ++q) {
    const uint64_t want = xi[q] ^ (q == (k >> 6) ? (1ull << (k & 63)) : 0ull);
    if (xj[q] != want) return false;
  }
  return true;
}

struct WideHash {
  const uint64_t* cells;
  const uint64_t* fp;
  const uint64_t* slots;
  uint32_t mask;
  int w;
  __device__ __forceinline__ int64_t find(uint32_t i, int k, const uint64_t* hbits) const {
    const uint64_t f = fp[i] ^ hbits[k];
    const uint32_t tag = uint32_t(f >> 32);
    uint32_t slot = uint32_t(f) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const uint64_t cur = slots[slot];
      if (cur == kEmpty) return -1;
      if (uint32_t(cur >> 32) == tag && is_flip(cells, w, i, uint32_t(cur), k))
        return uint32_t(cur);
      slot = (slot + 1) & mask;
    }
    return -1;
  }
};

struct WideSorted {
  const uint64_t* cells;
  const DevCounters* ctr;
  int w;
  // Three-way compare of cells[m] with (cells[i] xor e_k), most significant word first.
  __device__ __forceinline__ int cmp(uint32_t m, uint32_t i, int k) const {
    const uint64_t* xm = cells + uint64_t(m) * w;
    const uint64_t* xi = cells + uint64_t(i) * w;
    for (int q = w - 1; q >= 0; --q) {
      const uint64_t t = xi[q] ^ (q == (k >> 6) ? (1ull << (k & 63)) : 0ull);
      if (xm[q] != t) return xm[q] < t ? -1 : 1;
    }
    return 0;
  }
  __device__ __forceinline__ int64_t find(uint32_t i, int k, const uint64_t*) const {
    uint32_t lo = 0, hi = ctr->n_unique;
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (cmp(mid, i, k) < 0) lo = mid + 1;
      else hi = mid;
    }
    return (lo < ctr->n_unique && cmp(lo, i, k) == 0) ? int64_t(lo) : -1;
  }
};

// TREE lookups (Algorithm 4's walk): from the root, follow the child for the
// query's digit on each node's branching level; a missing child ends the
// search; a leaf is compared with the whole query.
struct TreeSmall {
  const uint64_t* cells;
  const TreeNode* nodes;
  int ell;
  __device__ __forceinline__ int64_t find(uint64_t y) const {
    uint32_t c = 0;
    for (int guard = 0; guard <= tree_levels(ell) + 1; ++guard) {
      const TreeNode& nd = nodes[c];
      if (nd.cnt <= 1) return (nd.cnt == 1 && cells[nd.lo] == y) ? int64_t(nd.lo) : -1;
      int lo, hi;
      tree_digit_bits(ell, int(nd.lv), &lo, &hi);
      const uint32_t v = uint32_t((y >> lo) & ((1ull << (hi - lo)) - 1ull));
      const int64_t ch = tree_child(nd, v);
      if (ch < 0) return -1;
      c = uint32_t(ch);
    }
    return -1;
  }
};

struct TreeWide {
  const uint64_t* cells;
  const TreeNode* nodes;
  int w;
  int ell;
  // Digit on level lv of cells[i] with bit k flipped.
  __device__ __forceinline__ uint32_t digit(uint32_t i, int k, int lv) const {
    int lo, hi;
    tree_digit_bits(ell, lv, &lo, &hi);
    const uint64_t* row = cells + uint64_t(i) * w;
    const int q = lo >> 6, sh = lo & 63;
    uint64_t a = row[q], b = (sh + (hi - lo) > 64) ? row[q + 1] : 0ull;
    if ((k >> 6) == q) a ^= 1ull << (k & 63);
    if ((k >> 6) == q + 1) b ^= 1ull << (k & 63);
    uint64_t v = a >> sh;
    if (sh + (hi - lo) > 64) v |= b << (64 - sh);
    return uint32_t(v & ((1ull << (hi - lo)) - 1ull));
  }
  __device__ __forceinline__ int64_t find(uint32_t i, int k, const uint64_t*) const {
    uint32_t c = 0;
    for (int guard = 0; guard <= tree_levels(ell) + 1; ++guard) {
      const TreeNode& nd = nodes[c];
      if (nd.cnt <= 1)
        return (nd.cnt == 1 && is_flip(cells, w, i, nd.lo, k)) ? int64_t(nd.lo) : -1;
      const int64_t ch = tree_child(nd, digit(i, k, int(nd.lv)));
      if (ch < 0) return -1;
      c = uint32_t(ch);
    }
    return -1;
  }
};

template <class L>
__global__ void __launch_bounds__(kThreads)
    neighbors_wide(const uint64_t* __restrict__ cells, int w, int ell, L look,
                   const DevCounters* ctr, uint32_t* __restrict__ masks,
                   uint32_t* __restrict__ counts) {
  extern __shared__ uint64_t hbits[];
  load_fp_bits(hbits, ell);
  if (ctr->overflow) return;
  const uint32_t u = ctr->n_unique;
  const int nh = (ell + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    uint32_t total = 0;
    for (int h = 0; h < nh; ++h) {
      const int k = h * 32 + lane;
      const uint64_t xw = cells[uint64_t(i) * w + (h >> 1)];
      bool hit = false;
      if (k < ell && !((xw >> (k & 63)) & 1ull)) hit = look.find(i, k, hbits) >= 0;
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) masks[uint64_t(i) * nh + h] = m;
      total += __popc(m);
    }
    if (lane == 0) counts[i] = total;
  }
}

template <class L>
__global__ void __launch_bounds__(kThreads)
    emit_wide(const uint64_t* __restrict__ cells, int w, int ell, L look, DevCounters* ctr,
              const uint32_t* __restrict__ masks, const unsigned long long* __restrict__ offsets,
              uint32_t* __restrict__ edges, int64_t cap) {
  extern __shared__ uint64_t hbits[];
  load_fp_bits(hbits, ell);
  if (ctr->overflow) return;
  const uint32_t u = ctr->n_unique;
  const int nh = (ell + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    unsigned long long off = offsets[i];
    for (int h = 0; h < nh; ++h) {
      const uint32_t m = masks[uint64_t(i) * nh + h];
      if ((m >> lane) & 1u) {
        const int k = h * 32 + lane;
        const int64_t j = look.find(i, k, hbits);
        if (j < 0) atomicOr(&ctr->error, 32u);
        const unsigned long long r = off + __popc(m & lanemask_lt());
        if (r < (unsigned long long)cap) {
          edges[2 * r] = i;
          edges[2 * r + 1] = uint32_t(j);
        }
      }
      off += __popc(m);
    }
  }
}

// Steps 3-4 in one pass for vectors of W words (single-pass counterpart of
// neighbors_wide + scan + emit_wide): same chunking, ticket and bounded
// decoupled look-back as neighbors_emit_small; hits are kept in shared memory
// (up to l per cell).
template <class L>
__global__ void __launch_bounds__(kNEThreads)
    neighbors_emit_wide(const uint64_t* __restrict__ cells, int w, int ell, L look,
                        DevCounters* ctr, unsigned long long* status,
                        uint32_t* __restrict__ edges, int64_t cap, uint32_t max_n,
                        uint32_t polls) {
  extern __shared__ uint64_t dsm[];
  uint64_t* hbits = dsm;
  uint32_t* hits = reinterpret_cast<uint32_t*>(dsm + ell);  // [kNECells][ell]
  __shared__ uint32_t cnt[kNECells];
  __shared__ uint32_t off[kNECells];
  __shared__ uint32_t s_chunk;
  __shared__ unsigned long long s_base;
  load_fp_bits(hbits, ell);
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint32_t nchunks = (u + kNECells - 1) / kNECells;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nh = (ell + 31) >> 5;
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(&ctr->ticket, 1u);
    __syncthreads();
    const uint32_t c = s_chunk;
    if (c >= nchunks) break;
    for (int cl = warp; cl < kNECells; cl += kNEThreads / 32) {
      const uint32_t i = c * kNECells + cl;
      uint32_t total = 0;
      if (i < u) {
        for (int h = 0; h < nh; ++h) {
          const int k = h * 32 + lane;
          const uint64_t xw = cells[uint64_t(i) * w + (h >> 1)];
          int64_t j = -1;
          if (k < ell && !((xw >> (k & 63)) & 1ull)) j = look.find(i, k, hbits);
          const uint32_t m = __ballot_sync(0xffffffffu, j >= 0);
          if (j >= 0) hits[cl * ell + total + __popc(m & lanemask_lt())] = uint32_t(j);
          total += __popc(m);
        }
      }
      if (lane == 0) cnt[cl] = total;
    }
    __syncthreads();
    if (warp == 0) {
      const uint32_t v = cnt[lane];
      uint32_t inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      off[lane] = inc - v;
      const unsigned long long T = __shfl_sync(0xffffffffu, inc, 31);
      if (lane == 0) {
        unsigned long long base = 0;
        if (c == 0) {
          atomicExch(&status[0], kFlagPre | T);
        } else {
          atomicExch(&status[c], kFlagAgg | T);
          int64_t p = int64_t(c) - 1;
          uint32_t looked = 0;
          while (p >= 0) {
            if (looked++ >= polls) {  // every look counts; 0 polls gives up at once
              atomicOr(&ctr->error, kErrTimeout);
              break;
            }
            const unsigned long long sv =
                *reinterpret_cast<volatile unsigned long long*>(&status[p]);
            const unsigned long long f = sv & ~kValMask;
            if (f == 0) {
              __nanosleep(64);
              continue;
            }
            base += sv & kValMask;
            if (f == kFlagPre) break;
            --p;
          }
          atomicExch(&status[c], kFlagPre | (base + T));
        }
        s_base = base;
        if (c == nchunks - 1) ctr->n_edges = base + T;
      }
    }
    __syncthreads();
    const unsigned long long base = s_base;
    for (int cl = warp; cl < kNECells; cl += kNEThreads / 32) {
      const uint32_t i = c * kNECells + cl;
      const uint32_t m = cnt[cl];
      const unsigned long long o = base + off[cl];
      for (uint32_t r = lane; r < m; r += 32) {
        const unsigned long long e = o + r;
        if (e < (unsigned long long)cap) {
          edges[2 * e] = i;
          edges[2 * e + 1] = hits[cl * ell + r];
        }
      }
    }
    __syncthreads();
  }
}


// ------------------------------- batch gather ------------------------------

// Prefix sums of the scenes' word and edge counts (one block), plus a flag
// telling whether every scene fitted its internal regions and the totals fit
// the outputs.
__global__ void __launch_bounds__(1024)
    batch_offsets(const BatchEntry* __restrict__ tab, int n, long long* cells_off,
                  long long* edges_off, int64_t cells_cap, int64_t edges_cap, int* ok) {
  __shared__ long long wsum[2][32];
  long long carry_c = 0, carry_e = 0;
  int good = 1;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    long long c = 0, e = 0;
    if (i < n) {
      const DevCounters* ctr = tab[i].ctr;
      const unsigned u = ctr->n_unique;
      const unsigned long long en = ctr->n_edges;
      if (ctr->overflow || ctr->error || u > tab[i].ucap || en > tab[i].ecap) good = 0;
      c = (long long)min(u, tab[i].ucap) * tab[i].w;
      e = (long long)(en < tab[i].ecap ? en : tab[i].ecap);
    }
    long long ic = c, ie = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long tc = __shfl_up_sync(0xffffffffu, ic, o);
      const long long te = __shfl_up_sync(0xffffffffu, ie, o);
      if (lane >= o) {
        ic += tc;
        ie += te;
      }
    }
    if (lane == 31) {
      wsum[0][warp] = ic;
      wsum[1][warp] = ie;
    }
    __syncthreads();
    long long bc = 0, be = 0, tc = 0, te = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      if (w < warp) {
        bc += wsum[0][w];
        be += wsum[1][w];
      }
      tc += wsum[0][w];
      te += wsum[1][w];
    }
    if (i < n) {
      cells_off[i] = carry_c + bc + ic - c;
      edges_off[i] = carry_e + be + ie - e;
    }
    carry_c += tc;
    carry_e += te;
    __syncthreads();
  }
  good = __syncthreads_and(good);
  if (threadIdx.x == 0) {
    cells_off[n] = carry_c;
    edges_off[n] = carry_e;
    *ok = good && carry_c <= cells_cap && carry_e <= edges_cap;
  }
}

// Copies every scene's cells and edges to its place in the outputs. The
// output elements (cell words, then edge pairs) are split into equal
// warp-sized chunks over the whole grid, so one scene with a million edges
// does not keep a single block busy while the others idle: a warp takes
// 32 * kCopyPer consecutive elements (lane l every 32nd, coalesced), each
// lane finds the scene of its first element by binary search over the
// offsets and advances it as its position passes scene boundaries.
constexpr int kCopyPer = 16;

template <class Emit>
__device__ __forceinline__ void copy_segments(const long long* __restrict__ off, int n,
                                              long long total, Emit emit) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long chunk = 32LL * kCopyPer;
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * chunk;
       base < total; base += warps * chunk) {
    long long g = base + lane;
    if (g >= total) continue;
    int lo = 0, hi = n - 1;  // the last scene s with off[s] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    int sc = lo;
    for (int j = 0; j < kCopyPer && g < total; ++j, g += 32) {
      while (g >= off[sc + 1]) ++sc;
      emit(sc, g, g - off[sc]);
    }
  }
}

template <bool kPairs64>
__global__ void batch_copy(const BatchEntry* __restrict__ tab, int n, const long long* cells_off,
                           const long long* edges_off, const int* ok, uint64_t* out_cells,
                           uint32_t* out_edges) {
  if (!*ok) return;
  copy_segments(cells_off, n, cells_off[n], [&](int sc, long long g, long long t) {
    out_cells[g] = tab[sc].cells[t];
  });
  copy_segments(edges_off, n, edges_off[n], [&](int sc, long long g, long long t) {
    if (kPairs64) {
      reinterpret_cast<uint64_t*>(out_edges)[g] =
          reinterpret_cast<const uint64_t*>(tab[sc].edges)[t];
    } else {
      out_edges[2 * g] = tab[sc].edges[2 * t];
      out_edges[2 * g + 1] = tab[sc].edges[2 * t + 1];
    }
  });
}

template <class F>
cudaError_t finish(F) {
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// ------------------------------- launchers -------------------------------

cudaError_t launch_fill_u64(uint64_t* p, uint64_t v, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  fill_u64<<<grid_for(n, kThreads * 4, 16), kThreads, 0, s>>>(p, v, n);
  return finish(0);
}

cudaError_t launch_zero_counters(DevCounters* c, cudaStream_t s) {
  zero_counters<<<1, 32, 0, s>>>(c);
  return finish(0);
}

cudaError_t launch_clear_build(uint64_t* table, size_t cap, unsigned long long* status,
                               size_t n_status, DevCounters* ctr, cudaStream_t s,
                               uint64_t* table2, size_t cap2, uint32_t* zero32,
                               size_t n_zero32) {
  const size_t most = std::max(std::max(std::max(cap, cap2), n_status), n_zero32);
  const cudaError_t e = launch_dep(clear_build, dim3(grid_for(most + 1, kThreads * 4, 16)),
                                   dim3(kThreads), 0, s, table, cap, table2, cap2, status,
                                   n_status, ctr, zero32, n_zero32);
  count_launch();
  return e;
}

size_t ne_status_words(size_t max_n) { return (max_n + kNECells - 1) / kNECells + 1; }

cudaError_t launch_neighbors_emit_small(const uint64_t* cells, const SmallTable& t, int ell,
                                        int strategy, unsigned long long* status,
                                        uint32_t* edges, int64_t edges_cap, size_t max_n,
                                        cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  if (ell > 64) return cudaErrorInvalidValue;
  const int g = grid_for(max_n, kNECells, 2048 / kNESmallThreads);
  cudaError_t e;
  if (strategy == 2) {
    e = launch_dep(neighbors_emit_small<SmallSorted>, dim3(g), dim3(kNESmallThreads), 0, s, cells,
                   SmallSorted{cells, t.ctr}, t.ctr, ell, status, edges, edges_cap,
                   uint32_t(max_n), wait_limit(kSpinLimit));
  } else {
    e = launch_dep(neighbors_emit_small<SmallHash>, dim3(g), dim3(kNESmallThreads), 0, s, cells,
                   SmallHash{t.keys, t.vals, t.mask, t.shift, t.ctr}, t.ctr, ell, status, edges,
                   edges_cap, uint32_t(max_n), wait_limit(kSpinLimit));
  }
  count_launch();
  return e;
}

cudaError_t launch_neighbors_seg_small(const SegSearchScene* scenes, int n_scenes,
                                       size_t total_chunks, bool sorted_lookup,
                                       unsigned int* scratch, cudaStream_t s) {
  if (n_scenes <= 0) return cudaSuccess;
  seg_emit_offsets<<<1, 1024, 0, s>>>(scenes, n_scenes, scratch);
  const int g = int(std::max<size_t>(
      1, std::min<size_t>(total_chunks, size_t(sm_count()) * (2048 / kNESmallThreads))));
  if (sorted_lookup)
    neighbors_seg_small<true><<<g, kNESmallThreads, 0, s>>>(scenes, n_scenes, scratch,
                                                            wait_limit(kSpinLimit));
  else
    neighbors_seg_small<false><<<g, kNESmallThreads, 0, s>>>(scenes, n_scenes, scratch,
                                                             wait_limit(kSpinLimit));
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_insert_wide_seg(const SegInsertWide* scenes, int n_scenes,
                                   uint64_t total_points, cudaStream_t s) {
  if (n_scenes <= 0 || total_points == 0) return cudaSuccess;
  insert_wide_seg<<<grid_for(size_t(total_points), kThreads), kThreads, 0, s>>>(
      scenes, n_scenes, total_points);
  return finish(0);
}

cudaError_t launch_clear_seg(const SegClear* scenes, int n_scenes, cudaStream_t s) {
  if (n_scenes <= 0) return cudaSuccess;
  clear_seg<<<unsigned(n_scenes), 1024, 0, s>>>(scenes);
  return finish(0);
}

cudaError_t launch_keys_to_u64(const void* keys, int64_t n, int word_bits, int ell, uint64_t* out,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int w64 = (ell + 63) / 64;
  const int wc = (ell + word_bits - 1) / word_bits;
  keys_to_u64<<<grid_for(size_t(n) * w64, kThreads), kThreads, 0, s>>>(keys, n, word_bits, wc,
                                                                          w64, ell, out);
  return finish(0);
}

cudaError_t launch_load_cells(const void* cells, int64_t n, int word_bits, int ell, uint64_t* out,
                              DevCounters* ctr, cudaStream_t s) {
  const int w64 = (ell + 63) / 64;
  const int wc = (ell + word_bits - 1) / word_bits;
  load_cells<<<grid_for(size_t(n) * w64 + 1, kThreads), kThreads, 0, s>>>(
      cells, n, word_bits, wc, w64, ell, out, ctr);
  return finish(0);
}

cudaError_t launch_write_cells(const uint64_t* cells, int ell, int word_bits, void* out,
                               int64_t cap, const DevCounters* ctr, size_t max_n, cudaStream_t s,
                               const unsigned int* skip) {
  if (max_n == 0 || cap == 0) return cudaSuccess;
  const int w64 = (ell + 63) / 64;
  const int wc = (ell + word_bits - 1) / word_bits;
  write_cells<<<grid_for(max_n * wc, kThreads), kThreads, 0, s>>>(cells, w64, word_bits, wc, out,
                                                                   cap, ctr, skip);
  return finish(0);
}

cudaError_t launch_insert_small(const void* keys, int64_t n, int word_bits, int ell,
                                const SmallTable& t, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int wc = (ell + word_bits - 1) / word_bits;
  insert_small<<<grid_for(size_t(n), kThreads), kThreads, 0, s>>>(keys, n, word_bits, wc, t);
  return finish(0);
}

cudaError_t launch_rank_small(const uint64_t* cells, const SmallTable& t, size_t max_n,
                              cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  rank_small<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(cells, t);
  return finish(0);
}

cudaError_t launch_index_small(const uint64_t* cells, const SmallTable& t, size_t max_n,
                               cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  index_small<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(cells, t);
  return finish(0);
}

cudaError_t launch_point_cell_small(const void* keys, int64_t n, int word_bits, int ell,
                                    const SmallTable& t, uint32_t* point_cell, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int wc = (ell + word_bits - 1) / word_bits;
  point_cell_small<<<grid_for(size_t(n), kThreads), kThreads, 0, s>>>(keys, n, word_bits, wc, t,
                                                                      point_cell);
  return finish(0);
}

cudaError_t launch_neighbors_small(const uint64_t* cells, const SmallTable& t, int ell,
                                   int strategy, uint32_t* masks, uint32_t* counts, size_t max_n,
                                   cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const int g = grid_for(max_n, kThreads / 32);
  if (strategy == 2) {
    neighbors_small<<<g, kThreads, 0, s>>>(cells, SmallSorted{cells, t.ctr}, t.ctr, ell, masks,
                                           counts);
  } else {
    neighbors_small<<<g, kThreads, 0, s>>>(cells, SmallHash{t.keys, t.vals, t.mask, t.shift, t.ctr}, t.ctr,
                                           ell, masks, counts);
  }
  return finish(0);
}

cudaError_t launch_emit_small(const uint64_t* cells, const SmallTable& t, int ell, int strategy,
                              const uint32_t* masks, const unsigned long long* offsets,
                              uint32_t* edges, int64_t edges_cap, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const int g = grid_for(max_n, kThreads / 32);
  if (strategy == 2) {
    emit_small<<<g, kThreads, 0, s>>>(cells, SmallSorted{cells, t.ctr}, t.ctr, ell, masks,
                                      offsets, edges, edges_cap);
  } else {
    emit_small<<<g, kThreads, 0, s>>>(cells, SmallHash{t.keys, t.vals, t.mask, t.shift, t.ctr}, t.ctr, ell,
                                      masks, offsets, edges, edges_cap);
  }
  return finish(0);
}

cudaError_t launch_insert_wide(const uint64_t* keys, int64_t n, int w64, const WideTable& t,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  insert_wide<<<grid_for(size_t(n), kThreads), kThreads, 0, s>>>(keys, n, w64, t);
  return finish(0);
}

cudaError_t sort_wide(const uint64_t* keys, int w64, int ell, uint32_t* idx0, uint32_t* idx1,
                      uint64_t* kw0, uint64_t* kw1, const unsigned int* n_dev, size_t max_n,
                      void* scratch, cudaStream_t s, uint32_t** sorted_idx,
                      const unsigned int* skip, unsigned int* flag, const void* ukeys) {
  return merge_sort_rows(keys, w64, ell, idx0, kw0, kw1, idx0, idx1, n_dev, max_n, s,
                         sorted_idx, skip, flag, scratch, radix_scratch_bytes(max_n),
                         static_cast<const ulonglong2*>(ukeys));
}

cudaError_t launch_gather_rows(const uint64_t* keys, int w64, const uint32_t* idx,
                               const unsigned int* n_dev, size_t max_n, uint64_t* out,
                               cudaStream_t s, const unsigned int* skip, int64_t out_cap) {
  if (max_n == 0) return cudaSuccess;
  gather_rows<<<grid_for(max_n * w64, kThreads), kThreads, 0, s>>>(
      keys, w64, idx, n_dev, uint32_t(max_n), out, skip, out_cap);
  return finish(0);
}

cudaError_t launch_rank_by_row(const uint32_t* idx, const unsigned int* n_dev, size_t max_n,
                               uint32_t* rank, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  rank_by_row<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(idx, n_dev, uint32_t(max_n), rank);
  return finish(0);
}

cudaError_t launch_point_cell_wide(const uint64_t* keys, int64_t n, int w64, const WideTable& t,
                                   const uint32_t* rank, uint32_t* point_cell, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  point_cell_wide<<<grid_for(size_t(n), kThreads), kThreads, 0, s>>>(keys, n, w64, t, rank,
                                                                     point_cell);
  return finish(0);
}

static size_t hbits_bytes(int ell) { return size_t(ell) * sizeof(uint64_t); }

static cudaError_t allow_smem(const void* kern, size_t bytes) {
  return ensure_smem_limit(kern, bytes);
}

cudaError_t launch_index_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                              uint64_t* fp, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = hbits_bytes(ell);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(index_wide), smem);
  if (e != cudaSuccess) return e;
  index_wide<<<grid_for(max_n, kThreads / 32), kThreads, smem, s>>>(cells, w64, ell, t, fp);
  return finish(0);
}

cudaError_t launch_neighbors_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                                  const uint64_t* fp, int strategy, uint32_t* masks,
                                  uint32_t* counts, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = hbits_bytes(ell);
  const int g = grid_for(max_n, kThreads / 32);
  cudaError_t e;
  if (strategy == 2) {
    auto k = neighbors_wide<WideSorted>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kThreads, smem, s>>>(cells, w64, ell, WideSorted{cells, t.ctr, w64}, t.ctr, masks,
                                counts);
  } else {
    auto k = neighbors_wide<WideHash>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kThreads, smem, s>>>(cells, w64, ell, WideHash{cells, fp, t.slots, t.mask, w64}, t.ctr,
                                masks, counts);
  }
  return finish(0);
}

cudaError_t launch_emit_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                             const uint64_t* fp, int strategy, const uint32_t* masks,
                             const unsigned long long* offsets, uint32_t* edges,
                             int64_t edges_cap, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = hbits_bytes(ell);
  const int g = grid_for(max_n, kThreads / 32);
  cudaError_t e;
  if (strategy == 2) {
    auto k = emit_wide<WideSorted>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kThreads, smem, s>>>(cells, w64, ell, WideSorted{cells, t.ctr, w64}, t.ctr, masks,
                                offsets, edges, edges_cap);
  } else {
    auto k = emit_wide<WideHash>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kThreads, smem, s>>>(cells, w64, ell, WideHash{cells, fp, t.slots, t.mask, w64}, t.ctr,
                                masks, offsets, edges, edges_cap);
  }
  return finish(0);
}

cudaError_t launch_neighbors_emit_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                                       const uint64_t* fp, int strategy,
                                       unsigned long long* status, uint32_t* edges,
                                       int64_t edges_cap, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = size_t(ell) * sizeof(uint64_t) + size_t(kNECells) * ell * sizeof(uint32_t);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int g = grid_for(max_n, kNECells, 4);
  cudaError_t e;
  if (strategy == 2) {
    auto k = neighbors_emit_wide<WideSorted>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kNEThreads, smem, s>>>(cells, w64, ell, WideSorted{cells, t.ctr, w64}, t.ctr, status,
                                  edges, edges_cap, uint32_t(max_n),
                                  wait_limit(kSpinLimit));
  } else {
    auto k = neighbors_emit_wide<WideHash>;
    if ((e = allow_smem(reinterpret_cast<const void*>(k), smem)) != cudaSuccess) return e;
    k<<<g, kNEThreads, smem, s>>>(cells, w64, ell, WideHash{cells, fp, t.slots, t.mask, w64},
                                  t.ctr, status, edges, edges_cap, uint32_t(max_n),
                                  wait_limit(kSpinLimit));
  }
  return finish(0);
}

cudaError_t launch_batch_gather(const BatchEntry* tab, int n, long long* cells_off,
                                long long* edges_off, int* ok, uint64_t* out_cells,
                                int64_t cells_cap, uint32_t* out_edges, int64_t edges_cap,
                                cudaStream_t s) {
  batch_offsets<<<1, 1024, 0, s>>>(tab, n, cells_off, edges_off, cells_cap, edges_cap, ok);
  const unsigned g = unsigned(sm_count()) * 8;
  if (reinterpret_cast<uintptr_t>(out_edges) % 8 == 0)
    batch_copy<true><<<g, 256, 0, s>>>(tab, n, cells_off, edges_off, ok, out_cells, out_edges);
  else
    batch_copy<false><<<g, 256, 0, s>>>(tab, n, cells_off, edges_off, ok, out_cells, out_edges);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_neighbors_emit_tree(const uint64_t* cells, int w64, int ell,
                                       const TreeNode* nodes, DevCounters* ctr,
                                       unsigned long long* status, uint32_t* edges,
                                       int64_t edges_cap, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  if (w64 == 1 && ell <= 64) {
    const int g = grid_for(max_n, kNECells, 2048 / kNESmallThreads);
    neighbors_emit_small<<<g, kNESmallThreads, 0, s>>>(cells, TreeSmall{cells, nodes, ell}, ctr,
                                                       ell, status, edges, edges_cap,
                                                       uint32_t(max_n), wait_limit(kSpinLimit));
    return finish(0);
  }
  const size_t smem = size_t(ell) * sizeof(uint64_t) + size_t(kNECells) * ell * sizeof(uint32_t);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto k = neighbors_emit_wide<TreeWide>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  const int g = grid_for(max_n, kNECells, 4);
  k<<<g, kNEThreads, smem, s>>>(cells, w64, ell, TreeWide{cells, nodes, w64, ell}, ctr, status,
                                edges, edges_cap, uint32_t(max_n),
                                wait_limit(kSpinLimit));
  return finish(0);
}

bool neighbors_emit_tree_fits(int w64, int ell) {
  return (w64 == 1 && ell <= 64) ||
         size_t(ell) * sizeof(uint64_t) + size_t(kNECells) * ell * sizeof(uint32_t) <= 200 * 1024;
}

cudaError_t launch_neighbors_tree_masks(const uint64_t* cells, int w64, int ell,
                                        const TreeNode* nodes, DevCounters* ctr, uint32_t* masks,
                                        uint32_t* counts, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = hbits_bytes(ell);
  auto k = neighbors_wide<TreeWide>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(max_n, kThreads / 32), kThreads, smem, s>>>(
      cells, w64, ell, TreeWide{cells, nodes, w64, ell}, ctr, masks, counts);
  return finish(0);
}

cudaError_t launch_emit_tree(const uint64_t* cells, int w64, int ell, const TreeNode* nodes,
                             DevCounters* ctr, const uint32_t* masks,
                             const unsigned long long* offsets, uint32_t* edges,
                             int64_t edges_cap, size_t max_n, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const size_t smem = hbits_bytes(ell);
  auto k = emit_wide<TreeWide>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<grid_for(max_n, kThreads / 32), kThreads, smem, s>>>(
      cells, w64, ell, TreeWide{cells, nodes, w64, ell}, ctr, masks, offsets, edges, edges_cap);
  return finish(0);
}

namespace {

__global__ void check_sorted(const uint64_t* __restrict__ cells, int w, DevCounters* ctr,
                             uint32_t max_n) {
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x + 1; i < u;
       i += gridDim.x * blockDim.x) {
    const uint64_t* x = cells + uint64_t(i - 1) * w;
    const uint64_t* y = cells + uint64_t(i) * w;
    int q = w - 1;
    while (q > 0 && x[q] == y[q]) --q;
    if (!(x[q] < y[q])) atomicOr(&ctr->error, kErrUnsorted);
  }
}

__global__ void adopt_cells(const uint64_t* __restrict__ cells, int w, int ell, uint32_t n,
                            DevCounters* ctr) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_unique = n;
  const uint64_t high = (ell & 63) ? ~((1ull << (ell & 63)) - 1) : 0ull;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t* y = cells + uint64_t(i) * w;
    if (y[w - 1] & high) atomicOr(&ctr->error, kErrHighBits);
    if (i == 0) continue;
    const uint64_t* x = y - w;
    int q = w - 1;
    while (q > 0 && x[q] == y[q]) --q;
    if (!(x[q] < y[q])) atomicOr(&ctr->error, kErrUnsorted);
  }
}

// Rows of 2 .. 32 words checked with lanes over words: a warp step covers
// R = 32 / w consecutive rows (lane l: row r0 + l / w, word l % w), reading
// each row coalesced and the row before it (cached, the previous lanes' row).
// Row i is after row i - 1 when they differ and the highest differing word
// is larger in row i; bits at or above l in the top word are an error too
// (high = the mask of those bits, or 0 to skip that check).
__device__ __forceinline__ void check_rows_warp(const uint64_t* __restrict__ cells, int w,
                                                uint32_t n, uint64_t high, DevCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const int R = 32 / w;
  const int a = lane / w, q = lane - a * w;
  const uint32_t seg_mask = w == 32 ? 0xffffffffu : ((1u << w) - 1u);
  const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const uint64_t wg = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  for (uint64_t r0 = wg * R; r0 < n; r0 += warps * R) {
    const uint64_t i = r0 + a;
    const bool live = a < R && i < n;
    uint64_t y = 0, x = 0;
    if (live) {
      y = cells[i * w + q];
      if (i > 0) x = cells[(i - 1) * w + q];
    }
    const uint32_t diff = __ballot_sync(0xffffffffu, live && i > 0 && x != y);
    const uint32_t lt = __ballot_sync(0xffffffffu, x < y);
    if (live && i > 0 && q == 0) {
      const uint32_t seg = (diff >> (a * w)) & seg_mask;
      if (seg == 0 || !((lt >> (a * w + 31 - __clz(seg))) & 1u))
        atomicOr(&ctr->error, kErrUnsorted);
    }
    if (live && q == w - 1 && (y & high)) atomicOr(&ctr->error, kErrHighBits);
  }
}

__global__ void adopt_cells_warp(const uint64_t* __restrict__ cells, int w, int ell, uint32_t n,
                                 DevCounters* ctr) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_unique = n;
  check_rows_warp(cells, w, n, (ell & 63) ? ~((1ull << (ell & 63)) - 1) : 0ull, ctr);
}

__global__ void check_sorted_warp(const uint64_t* __restrict__ cells, int w, DevCounters* ctr,
                                  uint32_t max_n) {
  check_rows_warp(cells, w, min(ctr->n_unique, max_n), 0ull, ctr);
}

__global__ void publish_done(const DevCounters* __restrict__ ctr, DevCounters* host_ctr,
                             unsigned int* host_flag, unsigned int seq) {
  static_assert(sizeof(DevCounters) % sizeof(unsigned int) == 0, "DevCounters words");
  constexpr int kWords = int(sizeof(DevCounters) / sizeof(unsigned int));
  const unsigned int* src = reinterpret_cast<const unsigned int*>(ctr);
  unsigned int* dst = reinterpret_cast<unsigned int*>(host_ctr);
  if (threadIdx.x < kWords) dst[threadIdx.x] = src[threadIdx.x];
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile unsigned int*>(host_flag) = seq;
  }
}

// publish_done for several requests at once: block i publishes entry i.
__global__ void publish_group(const PublishEntry* __restrict__ e, int n) {
  constexpr int kWords = int(sizeof(DevCounters) / sizeof(unsigned int));
  if (int(blockIdx.x) >= n) return;
  const PublishEntry p = e[blockIdx.x];
  const unsigned int* src = reinterpret_cast<const unsigned int*>(p.ctr);
  unsigned int* dst = reinterpret_cast<unsigned int*>(p.host_ctr);
  if (threadIdx.x < kWords) dst[threadIdx.x] = src[threadIdx.x];
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile unsigned int*>(p.host_flag) = p.seq;
  }
}

__global__ void publish_counts(const DevCounters* ctr, int64_t* out, int64_t cells_cap,
                               int64_t edges_cap) {
  griddep_wait();
  int64_t status = CG_OK;
  if (ctr->error & kErrTimeout) status = CG_ERR_TIMEOUT;
  else if (ctr->error || ctr->overflow) status = CG_ERR_INTERNAL;
  else if (int64_t(ctr->n_unique) > cells_cap || int64_t(ctr->n_edges) > edges_cap)
    status = CG_ERR_CAPACITY;
  out[0] = int64_t(ctr->n_unique);
  out[1] = int64_t(ctr->n_edges);
  out[2] = status;
}

}  // namespace

cudaError_t launch_check_sorted(const uint64_t* cells, int w64, DevCounters* ctr, size_t max_n,
                                cudaStream_t s) {
  if (max_n < 2) return cudaSuccess;
  if (w64 >= 2 && w64 <= 32) {
    const size_t steps = (max_n + (32 / w64) - 1) / (32 / w64);
    check_sorted_warp<<<grid_for(steps, kThreads / 32), kThreads, 0, s>>>(cells, w64, ctr,
                                                                         uint32_t(max_n));
    return finish(0);
  }
  check_sorted<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(cells, w64, ctr, uint32_t(max_n));
  return finish(0);
}

cudaError_t launch_adopt_cells(const uint64_t* cells, int64_t n, int ell, DevCounters* ctr,
                               cudaStream_t s) {
  const int w64 = (ell + 63) / 64;
  if (w64 >= 2 && w64 <= 32) {
    const size_t steps = (size_t(n) + (32 / w64) - 1) / (32 / w64) + 1;
    adopt_cells_warp<<<grid_for(steps, kThreads / 32), kThreads, 0, s>>>(cells, w64, ell,
                                                                        uint32_t(n), ctr);
    return finish(0);
  }
  adopt_cells<<<grid_for(size_t(n) + 1, kThreads), kThreads, 0, s>>>(cells, w64, ell,
                                                                      uint32_t(n), ctr);
  return finish(0);
}

cudaError_t launch_publish_done(const DevCounters* ctr, DevCounters* host_ctr,
                                unsigned int* host_flag, unsigned int seq, cudaStream_t s) {
  publish_done<<<1, 32, 0, s>>>(ctr, host_ctr, host_flag, seq);
  return finish(0);
}

cudaError_t launch_publish_group(const PublishEntry* e, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  publish_group<<<n, 32, 0, s>>>(e, n);
  return finish(0);
}

cudaError_t launch_publish_counts(const DevCounters* ctr, int64_t* out, int64_t cells_cap,
                                  int64_t edges_cap, cudaStream_t s) {
  const cudaError_t e = launch_dep(publish_counts, dim3(1), dim3(1), 0, s, ctr, out, cells_cap,
                                   edges_cap);
  count_launch();
  return e;
}

}  // namespace cg
