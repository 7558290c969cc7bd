// PIVOT lookup strategy of the Hamming-1 search: distance-to-pivot bucketing
// by inequality (⋆) of §3.1, then XOR/popcount comparison of the candidates.
//
// For any pivot vectors p_0..p_{h-1}, two vectors at Hamming distance 1 have
// |dist(x, p_d) - dist(y, p_d)| = 1 for every d: the triangle inequality
// bounds the difference by 1, and a one-bit change flips the parity of every
// distance. The paper's heuristic (Algorithms 1-2) uses this to skip pairs
// while still visiting all n^2/2 of them. Here the cells are grouped instead:
// the key of a cell is its distance vector (dist(x, p_0), ..., dist(x,
// p_{h-1})) packed into one word, the cells are sorted by key, and a cell's
// neighbours can only be in the 2^h buckets whose keys differ from its own by
// +-1 in every coordinate. Each candidate in those buckets is compared word
// by word; a pair with exactly one differing bit k is an edge, reported from
// the endpoint whose bit k is 0 (the smaller one, as for the other
// strategies). The search counts each cell's edges and keeps the first few
// partners in a small per-cell buffer; an exclusive scan of the counts gives
// every cell's first output position; cells whose partners all fit in the
// buffer are written from it (in partner order), and only the rare cells with
// more edges are searched again to write theirs, then ordered.
//
// Pivots: h cells spread over the sorted order (cells floor((2d+1) U / 2h)),
// so that they are far apart in value; the choice does not change the output.
//
// This file also holds the HALVES strategy (two-part multi-index hashing,
// described below), which shares the hit buffer, scan and ordered output.
#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxW = 64;  // l <= 4096

int grid_for(size_t items, int per_block, int blocks_per_sm = 8) {
  const size_t want = (items + per_block - 1) / per_block;
  const size_t cap = size_t(sm_count()) * blocks_per_sm;
  size_t g = want < cap ? want : cap;
  return int(g < 1 ? 1 : g);
}

__device__ __forceinline__ uint32_t pivot_row(int d, int h, uint32_t u) {
  return uint32_t((uint64_t(2 * d + 1) * u) / uint64_t(2 * h));
}

// Key of every cell: h distances of `bits` bits each. A group of gs lanes
// (gs = W rounded up to a power of two, at most 32) works on one cell, lanes
// over words, so that rows are read with coalesced loads.
__global__ void __launch_bounds__(kThreads)
    pivot_keys(const uint64_t* __restrict__ cells, int w, int gs, int h, int bits,
               const DevCounters* ctr, uint32_t max_n, uint64_t* __restrict__ key_by_cell,
               uint64_t* __restrict__ skeys, uint32_t* __restrict__ sidx) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  if (u == 0) return;
  const int lane = threadIdx.x & 31;
  const int sub = lane % gs;
  const uint32_t per_warp = 32 / gs;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t groups = (u + per_warp - 1) / per_warp;
  for (uint32_t gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < groups;
       gi += warps) {
    const uint32_t i = gi * per_warp + lane / gs;
    const bool live = i < u;
    const uint64_t* xi = cells + uint64_t(live ? i : 0) * w;
    uint64_t key = 0;
    for (int d = 0; d < h; ++d) {
      const uint64_t* pd = cells + uint64_t(pivot_row(d, h, u)) * w;
      uint32_t dist = 0;
      if (live)
        for (int q = sub; q < w; q += gs) dist += __popcll(xi[q] ^ pd[q]);
      for (int o = gs >> 1; o > 0; o >>= 1) dist += __shfl_xor_sync(0xffffffffu, dist, o);
      key |= uint64_t(dist) << (bits * d);
    }
    if (live && sub == 0) {
      key_by_cell[i] = key;
      skeys[i] = key;
      sidx[i] = i;
    }
  }
}

// Bucket table: for every distinct key of the sorted key array, one
// 16-byte entry (key, start | count << 32) in an open-addressing table, so
// that a lookup reads one sector.
__global__ void __launch_bounds__(kThreads)
    pivot_index(const uint64_t* __restrict__ skeys, const DevCounters* ctr, uint32_t max_n,
                ulonglong2* __restrict__ table, uint32_t tmask, int tshift, DevCounters* wctr) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < u; t += gridDim.x * blockDim.x) {
    const uint64_t key = skeys[t];
    if (t > 0 && skeys[t - 1] == key) continue;
    uint32_t cnt = 1;
    while (t + cnt < u && skeys[t + cnt] == key) ++cnt;
    uint32_t slot = home_slot(key, tshift);
    bool placed = false;
    for (uint32_t probe = 0; probe <= tmask; ++probe) {
      const unsigned long long old =
          atomicCAS(reinterpret_cast<unsigned long long*>(&table[slot].x),
                    static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(key));
      if (old == kEmpty) {
        table[slot].y = uint64_t(t) | (uint64_t(cnt) << 32);
        placed = true;
        break;
      }
      slot = (slot + 1) & tmask;
    }
    if (!placed) atomicOr(&wctr->overflow, 1u);
  }
}

// (start, count) of a bucket, count 0 when the key is absent.
__device__ __forceinline__ uint64_t bucket_find(const ulonglong2* table, uint32_t tmask,
                                                int tshift, uint64_t key) {
  uint32_t slot = home_slot(key, tshift);
  for (uint32_t probe = 0; probe <= tmask; ++probe) {
    const ulonglong2 e = table[slot];
    if (e.x == key) return e.y;
    if (e.x == kEmpty) return 0;
    slot = (slot + 1) & tmask;
  }
  return 0;
}

// The search. Lanes work on (cell, bucket pattern) pairs in parallel: with
// P = 2^h patterns, a warp takes 32 / P consecutive cells (P <= 32) or one
// cell with the patterns strided over the lanes (P > 32). Each lane looks its
// bucket up and compares every candidate j > i of it with cell i, word by
// word (XOR + popcount, stopping at the second difference). (A 64-bit fold
// filter in bucket order, as HALVES uses, was measured slower here: the
// search is bound by its chain of dependent loads, not by their bytes.)
//   kCount: counts[i] = number of hits of cell i; the first kHitBuf partners
//           are kept in hbuf[i][.].
//   kWrite: cells with more than kHitBuf hits only: hit (i, j) goes to
//           edges[offsets[i] + fill[i]++] (positions below cap only).
constexpr int kHitBuf = 4;
enum { kCount = 0, kWrite = 1 };

// Records the hit (i, j), i < j, of a search pass (see above).
template <int kMode>
__device__ __forceinline__ void record_hit(uint32_t i, uint32_t j, uint32_t* __restrict__ counts,
                                           uint32_t* __restrict__ hbuf,
                                           const unsigned long long* __restrict__ offsets,
                                           uint32_t* __restrict__ fill,
                                           uint32_t* __restrict__ edges, int64_t cap) {
  if (kMode == kCount) {
    const uint32_t r = atomicAdd(&counts[i], 1u);
    if (r < uint32_t(kHitBuf)) hbuf[uint64_t(i) * kHitBuf + r] = j;
  } else {
    const unsigned long long pos = offsets[i] + atomicAdd(&fill[i], 1u);
    if (pos < (unsigned long long)cap) {
      edges[2 * pos] = i;
      edges[2 * pos + 1] = j;
    }
  }
}

template <int kMode>
__global__ void __launch_bounds__(kThreads)
    pivot_search(const uint64_t* __restrict__ cells, int w, int ell, int h, int bits,
                 const DevCounters* ctr, uint32_t max_n, const uint64_t* __restrict__ key_by_cell,
                 const uint32_t* __restrict__ sidx, const ulonglong2* __restrict__ table,
                 uint32_t tmask, int tshift, uint32_t* __restrict__ counts,
                 uint32_t* __restrict__ hbuf, const unsigned long long* __restrict__ offsets,
                 uint32_t* __restrict__ fill, uint32_t* __restrict__ edges, int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const int lane = threadIdx.x & 31;
  const int P = 1 << h;
  const int G = P <= 32 ? 32 / P : 1;
  const uint64_t fmask = (1ull << bits) - 1;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t groups = (u + G - 1) / G;
  for (uint32_t gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < groups;
       gi += warps) {
    const int g = P <= 32 ? lane / P : 0;
    const uint32_t i = gi * G + g;
    if (i >= u) continue;
    if (kMode == kWrite && counts[i] <= uint32_t(kHitBuf)) continue;
    const uint64_t key = key_by_cell[i];
    const uint64_t* xi = cells + uint64_t(i) * w;
    for (int pat = P <= 32 ? lane % P : lane; pat < P; pat += 32) {
      uint64_t target = key;
      bool ok = true;
      for (int d = 0; d < h; ++d) {
        const uint64_t c = (key >> (bits * d)) & fmask;
        const bool up = (pat >> d) & 1;
        if (up ? (c + 1 > uint64_t(ell)) : (c == 0)) ok = false;
        target = up ? target + (1ull << (bits * d)) : target - (1ull << (bits * d));
      }
      if (!ok) continue;
      const uint64_t sc = bucket_find(table, tmask, tshift, target);
      const uint32_t t0 = uint32_t(sc), tn = uint32_t(sc >> 32);
      for (uint32_t t = t0; t < t0 + tn; ++t) {
        const uint32_t j = sidx[t];
        if (j <= i) continue;
        const uint64_t* xj = cells + uint64_t(j) * w;
        int c = 0;
        for (int q = 0; q < w && c < 2; ++q) c += __popcll(xj[q] ^ xi[q]);
        if (c != 1) continue;
        record_hit<kMode>(i, j, counts, hbuf, offsets, fill, edges, cap);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// ALLPAIRS: the heuristic of §3.1 in the paper's own all-pairs form
// (Algorithm 2), for small U. A warp takes cell i and its lanes the cells
// j > i, 32 at a time; a pair is compared only when its pivot distances pass
// inequality (⋆) -- every field of the packed keys differs by exactly 1 (the
// bound of (⋆) plus the parity of a one-bit change) -- and then word by word
// like PIVOT's candidates. U (U - 1) / 2 key tests: quadratic, so the library
// offers it for small U only.
// ---------------------------------------------------------------------------
template <int kMode>
__global__ void __launch_bounds__(kThreads)
    allpairs_search(const uint64_t* __restrict__ cells, int w, int h, int bits,
                    const DevCounters* ctr, uint32_t max_n,
                    const uint64_t* __restrict__ key_by_cell, uint32_t* __restrict__ counts,
                    uint32_t* __restrict__ hbuf, const unsigned long long* __restrict__ offsets,
                    uint32_t* __restrict__ fill, uint32_t* __restrict__ edges, int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  const uint64_t fmask = (1ull << bits) - 1;
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < u; i += warps) {
    if (kMode == kWrite && counts[i] <= uint32_t(kHitBuf)) continue;
    const uint64_t ki = key_by_cell[i];
    const uint64_t* xi = cells + uint64_t(i) * w;
    for (uint32_t j = i + 1 + uint32_t(lane); j < u; j += 32) {
      const uint64_t kj = key_by_cell[j];
      bool ok = true;
      for (int d = 0; d < h && ok; ++d) {
        const uint64_t a = (ki >> (bits * d)) & fmask, b = (kj >> (bits * d)) & fmask;
        ok = a == b + 1 || b == a + 1;
      }
      if (!ok) continue;
      const uint64_t* xj = cells + uint64_t(j) * w;
      int c = 0;
      for (int q = 0; q < w && c < 2; ++q) c += __popcll(xj[q] ^ xi[q]);
      if (c == 1) record_hit<kMode>(i, j, counts, hbuf, offsets, fill, edges, cap);
    }
  }
}

// ---------------------------------------------------------------------------
// HALVES lookup strategy: the pigeonhole split of multi-index hashing
// (Norouzi, Punjani, Fleet, "Fast search in Hamming space with multi-index
// hashing", CVPR 2012) with two parts. Split the l bits at s = floor(l / 2)
// into L = bits [0, s) and H = bits [s, l). Two vectors at distance 1 agree
// exactly on one part:
//   * pairs that differ in L have equal H. In value order the cells are
//     sorted by H first, so these partners are in the same run of equal H,
//     contiguous in the cell array: cell i scans i + 1, i + 2, ... while the
//     H keys match;
//   * pairs that differ in H have equal L. (key of L, cell number) pairs are
//     sorted stably by an LSD radix sort, so equal L values form runs in
//     which cell numbers increase; a cell scans the rest of its run.
// Each group checks its own case exactly (H equal and one differing bit in L,
// resp. L equal and one differing bit in H), so every edge is found once,
// from its smaller endpoint, whatever the keys collide on. For one-word cells
// the keys are the parts themselves and the tests need no row; for wider
// cells the keys are hashes, and the fold of the other part (XOR of its
// masked words) rejects nearly every non-partner before the rows are read.
// Work is the sum of squared run lengths: O(U) when runs are short (random
// and clustered vectors), up to U^1.5 for the hypercube.
// ---------------------------------------------------------------------------

// Mask of the bits of word q that lie in L = [0, s).
__device__ __forceinline__ uint64_t low_mask(int q, int s) {
  const int lo = 64 * q;
  if (s >= lo + 64) return ~0ull;
  if (s <= lo) return 0ull;
  return (1ull << (s - lo)) - 1;
}

// Rows x and y agree on one part and differ in exactly one bit of the other
// (L when in_low, else H).
__device__ __forceinline__ bool one_bit_in_part(const uint64_t* __restrict__ x,
                                                const uint64_t* __restrict__ y, int w, int s,
                                                bool in_low) {
  int c = 0;
  for (int q = 0; q < w; ++q) {
    const uint64_t d = x[q] ^ y[q];
    const uint64_t m = low_mask(q, s);
    if (d & (in_low ? ~m : m)) return false;
    c += __popcll(d);
    if (c > 1) return false;
  }
  return c == 1;
}

// Per cell: hkey (H itself for one word, else a 64-bit hash of H), the folds
// fL and fH of the two parts, the sort key of L (L itself for one word, else
// a 32-bit hash) and the identity permutation.
__global__ void __launch_bounds__(kThreads)
    halves_keys(const uint64_t* __restrict__ cells, int w, int s, const DevCounters* ctr,
                uint32_t max_n, uint64_t* __restrict__ hkey, uint64_t* __restrict__ fl,
                uint64_t* __restrict__ fh, uint64_t* __restrict__ lkey,
                uint32_t* __restrict__ idx) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint64_t* x = cells + uint64_t(i) * w;
    if (w == 1) {
      const uint64_t m = low_mask(0, s);
      hkey[i] = x[0] & ~m;
      fh[i] = x[0] & ~m;
      fl[i] = x[0] & m;
      lkey[i] = x[0] & m;
    } else {
      uint64_t hh = 0, hl = 0, a = 0, b = 0;
      for (int q = 0; q < w; ++q) {
        const uint64_t m = low_mask(q, s);
        const uint64_t lo = x[q] & m, hi = x[q] & ~m;
        const uint64_t salt = 0x9e3779b97f4a7c15ull * uint64_t(q + 1);
        a ^= lo;
        b ^= hi;
        hl ^= mix64(lo + salt);
        hh ^= mix64(hi + salt);
      }
      hkey[i] = hh;
      fl[i] = a;
      fh[i] = b;
      lkey[i] = hl & 0xffffffffull;
    }
    idx[i] = i;
  }
}

// The same for cells of 2 .. kKeysStageW words: a warp reads 32 consecutive
// cells coalesced (lane l takes words l, l + 32, ... of the 32 rows) into
// shared memory, stride w + 1 words, and lane l then computes cell l's keys
// from there (a thread reading its own row puts w * 8 bytes between the
// addresses of consecutive lanes).
constexpr int kKeysStageW = 16;

// adopt_n >= 0: the cells are a caller's rows used in place (U = adopt_n);
// the kernel also sets ctr->n_unique and checks what adopt_cells checks (rows
// strictly ascending, no bit at or above l), from the rows it has staged.
__global__ void __launch_bounds__(kThreads)
    halves_keys_staged(const uint64_t* __restrict__ cells, int w, int s, DevCounters* ctr,
                       uint32_t max_n, uint64_t* __restrict__ hkey, uint64_t* __restrict__ fl,
                       uint64_t* __restrict__ fh, uint64_t* __restrict__ lkey,
                       uint32_t* __restrict__ idx, int64_t adopt_n, int ell) {
  extern __shared__ uint64_t keys_stage[];
  if (ctr->overflow) return;
  const uint32_t u = adopt_n >= 0 ? uint32_t(min(uint64_t(adopt_n), uint64_t(max_n)))
                                  : min(ctr->n_unique, max_n);
  if (adopt_n >= 0 && blockIdx.x == 0 && threadIdx.x == 0) ctr->n_unique = uint32_t(adopt_n);
  const uint64_t high = (ell & 63) ? ~((1ull << (ell & 63)) - 1) : 0ull;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int stride = w + 1;
  uint64_t* sr = keys_stage + size_t(warp) * 32 * stride;
  const int da = 32 / w, dq = 32 % w;
  for (uint64_t r0 = (uint64_t(blockIdx.x) * (kThreads / 32) + warp) * 32; r0 < u;
       r0 += uint64_t(gridDim.x) * kThreads) {
    const uint32_t rows = uint32_t(min(uint64_t(32), u - r0));
    const uint32_t elems = rows * uint32_t(w);
    const uint64_t* src = cells + r0 * w;
    int a = lane / w, q = lane - a * w;
    for (uint32_t e = lane; e < elems; e += 32) {
      sr[a * stride + q] = __ldg(src + e);
      a += da;
      q += dq;
      if (q >= w) {
        q -= w;
        ++a;
      }
    }
    __syncwarp();
    if (uint32_t(lane) < rows) {
      const uint64_t* x = sr + lane * stride;
      if (adopt_n >= 0) {
        const uint64_t i = r0 + uint64_t(lane);
        if (x[w - 1] & high) atomicOr(&ctr->error, kErrHighBits);
        if (i > 0) {
          const uint64_t* y = lane > 0 ? sr + (lane - 1) * stride : cells + (i - 1) * w;
          int q = w - 1;
          while (q > 0 && y[q] == x[q]) --q;
          if (!(y[q] < x[q])) atomicOr(&ctr->error, kErrUnsorted);
        }
      }
      uint64_t hh = 0, hl = 0, fa = 0, fb = 0;
      for (int k = 0; k < w; ++k) {
        const uint64_t m = low_mask(k, s);
        const uint64_t lo = x[k] & m, hi = x[k] & ~m;
        const uint64_t salt = 0x9e3779b97f4a7c15ull * uint64_t(k + 1);
        fa ^= lo;
        fb ^= hi;
        hl ^= mix64(lo + salt);
        hh ^= mix64(hi + salt);
      }
      const uint64_t i = r0 + uint64_t(lane);
      hkey[i] = hh;
      fl[i] = fa;
      fh[i] = fb;
      lkey[i] = hl & 0xffffffffull;
      idx[i] = uint32_t(i);
    }
    __syncwarp();
  }
}

// sfh[t] = fh[sidx[t]]: the H fold of the cell at sorted position t.
__global__ void __launch_bounds__(kThreads)
    halves_gather(const DevCounters* ctr, uint32_t max_n, const uint32_t* __restrict__ sidx,
                  const uint64_t* __restrict__ fh, uint64_t* __restrict__ sfh) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < u; t += gridDim.x * blockDim.x)
    sfh[t] = fh[sidx[t]];
}

// Items g < U: cell g's partners in its run of equal H; items U + t: the
// partners of the cell at sorted position t in its run of equal L.
template <int kMode>
__global__ void __launch_bounds__(kThreads)
    halves_search(const uint64_t* __restrict__ cells, int w, int s, const DevCounters* ctr,
                  uint32_t max_n, const uint64_t* __restrict__ hkey,
                  const uint64_t* __restrict__ fl, const uint64_t* __restrict__ skey,
                  const uint32_t* __restrict__ sidx, const uint64_t* __restrict__ sfh,
                  uint32_t* __restrict__ counts, uint32_t* __restrict__ hbuf,
                  const unsigned long long* __restrict__ offsets, uint32_t* __restrict__ fill,
                  uint32_t* __restrict__ edges, int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint64_t items = 2ull * u;
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < items;
       g += uint64_t(gridDim.x) * blockDim.x) {
    if (g < u) {
      const uint32_t i = uint32_t(g);
      if (kMode == kWrite && counts[i] <= uint32_t(kHitBuf)) continue;
      const uint64_t hk = hkey[i], f = fl[i];
      for (uint32_t j = i + 1; j < u && hkey[j] == hk; ++j) {
        if (__popcll(fl[j] ^ f) != 1) continue;
        if (w > 1 &&
            !one_bit_in_part(cells + uint64_t(i) * w, cells + uint64_t(j) * w, w, s, true))
          continue;
        record_hit<kMode>(i, j, counts, hbuf, offsets, fill, edges, cap);
      }
    } else {
      const uint32_t t = uint32_t(g - u);
      const uint32_t i = sidx[t];
      if (kMode == kWrite && counts[i] <= uint32_t(kHitBuf)) continue;
      const uint64_t k = skey[t], f = sfh[t];
      for (uint32_t t2 = t + 1; t2 < u && skey[t2] == k; ++t2) {
        if (__popcll(sfh[t2] ^ f) != 1) continue;
        const uint32_t j = sidx[t2];
        if (w > 1 &&
            !one_bit_in_part(cells + uint64_t(i) * w, cells + uint64_t(j) * w, w, s, false))
          continue;
        record_hit<kMode>(i, j, counts, hbuf, offsets, fill, edges, cap);
      }
    }
  }
}

// Puts the edges of every cell with more than kHitBuf of them in increasing
// order of j (insertion sort of the segment, whose length is at most the
// cell's degree). Segments that do not lie wholly below cap are left alone
// (the call then reports capacity).
__global__ void __launch_bounds__(kThreads)
    pivot_order(const DevCounters* ctr, uint32_t max_n, const uint32_t* __restrict__ counts,
                const unsigned long long* __restrict__ offsets, uint32_t* __restrict__ edges,
                int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t m = counts[i];
    if (m <= uint32_t(kHitBuf)) continue;
    const unsigned long long o = offsets[i];
    if (o + m > (unsigned long long)cap) continue;
    uint32_t* e = edges + 2 * o;
    for (uint32_t a = 1; a < m; ++a) {
      const uint32_t v = e[2 * a + 1];
      uint32_t b = a;
      while (b > 0 && e[2 * (b - 1) + 1] > v) {
        e[2 * b + 1] = e[2 * (b - 1) + 1];
        --b;
      }
      e[2 * b + 1] = v;
    }
  }
}

int key_bits(int ell) {
  int b = 1;
  while ((1 << b) <= ell) ++b;
  return b;
}

}  // namespace

int pivot_max_h(int ell) {
  const int by_bits = 64 / key_bits(ell);
  return by_bits < 8 ? by_bits : 8;
}

int pivot_sort_bits(int ell, int h) { return key_bits(ell) * h; }

cudaError_t launch_pivot_keys(const uint64_t* cells, int w64, int ell, int h,
                              const DevCounters* ctr, size_t max_n, uint64_t* key_by_cell,
                              uint64_t* skeys, uint32_t* sidx, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  int gs = 1;
  while (gs < w64 && gs < 32) gs <<= 1;
  const size_t groups = (max_n + size_t(32 / gs) - 1) / size_t(32 / gs);
  pivot_keys<<<grid_for(groups, kThreads / 32), kThreads, 0, s>>>(
      cells, w64, gs, h, key_bits(ell), ctr, uint32_t(max_n), key_by_cell, skeys, sidx);
  count_launch();
  return cudaGetLastError();
}

size_t pivot_table_slots(size_t max_n) {
  size_t c = 1024;
  while (c < 2 * max_n) c <<= 1;
  return c;
}

cudaError_t launch_pivot_index(const uint64_t* skeys, const DevCounters* ctr, size_t max_n,
                               void* table, size_t tcap, DevCounters* wctr, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  pivot_index<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(
      skeys, ctr, uint32_t(max_n), static_cast<ulonglong2*>(table), uint32_t(tcap - 1),
      table_shift(tcap), wctr);
  count_launch();
  return cudaGetLastError();
}

namespace {

// Edge offsets of every cell and the edges of the cells whose hits fit the hit
// buffer, in one pass: chunks of kHEChunk cells handed out in order by a
// ticket (status[0]), a block scan of the chunk's counts, and a decoupled
// look-back (Merrill & Garland 2016) over the earlier chunks' published
// totals (status[1 + c]) for the chunk's first edge. The look-back wait is
// bounded: after `polls` looks it sets the timeout bit and gives up.
constexpr int kHEThreads = 512;
constexpr int kHEPer = 8;
constexpr uint32_t kHEChunk = kHEThreads * kHEPer;  // 4096 cells
constexpr unsigned long long kHEAgg = 1ull << 62;
constexpr unsigned long long kHEPre = 2ull << 62;
constexpr unsigned long long kHEVal = (1ull << 62) - 1;
constexpr unsigned kHESpinLimit = 1u << 22;

__global__ void __launch_bounds__(kHEThreads)
    hits_emit(DevCounters* ctr, uint32_t max_n, const uint32_t* __restrict__ counts,
              const uint32_t* __restrict__ hbuf, unsigned long long* __restrict__ offsets,
              unsigned long long* status, uint32_t* __restrict__ edges, int64_t cap,
              uint32_t polls) {
  __shared__ unsigned long long wsum[kHEThreads / 32];
  __shared__ uint32_t chunk_s;
  __shared__ unsigned long long base_s;
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint32_t nchunks = (u + kHEChunk - 1) / kHEChunk;
  if (u == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_edges = 0;
    return;
  }
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) chunk_s = atomicAdd(reinterpret_cast<unsigned int*>(status), 1u);
    __syncthreads();
    const uint32_t c = chunk_s;
    if (c >= nchunks) break;
    const uint32_t i0 = c * kHEChunk + threadIdx.x * kHEPer;
    uint32_t m[kHEPer];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kHEPer; ++q) {
      m[q] = i0 + q < u ? counts[i0 + q] : 0u;
      sum += m[q];
    }
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      unsigned long long v = lane < kHEThreads / 32 ? wsum[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (lane < kHEThreads / 32) wsum[lane] = v;
    }
    __syncthreads();
    const unsigned long long before = (warp > 0 ? wsum[warp - 1] : 0ull) + inc - sum;
    const unsigned long long T = wsum[kHEThreads / 32 - 1];
    if (threadIdx.x == 0) {
      unsigned long long base = 0;
      unsigned long long* st = status + 1;
      if (c == 0) {
        atomicExch(&st[0], kHEPre | T);
      } else {
        atomicExch(&st[c], kHEAgg | T);
        int64_t p = int64_t(c) - 1;
        uint32_t looked = 0;
        while (p >= 0) {
          if (looked++ >= polls) {  // every look counts; 0 polls gives up at once
            atomicOr(&ctr->error, kErrTimeout);
            break;
          }
          const unsigned long long sv = *reinterpret_cast<volatile unsigned long long*>(&st[p]);
          const unsigned long long f = sv & ~kHEVal;
          if (f == 0) {
            __nanosleep(64);
            continue;
          }
          base += sv & kHEVal;
          if (f == kHEPre) break;
          --p;
        }
        atomicExch(&st[c], kHEPre | (base + T));
      }
      base_s = base;
      if (c == nchunks - 1) ctr->n_edges = base + T;
    }
    __syncthreads();
    unsigned long long o = base_s + before;
#pragma unroll
    for (int q = 0; q < kHEPer; ++q) {
      const uint32_t i = i0 + q;
      if (i >= u) break;
      offsets[i] = o;
      const uint32_t mq = m[q];
      if (mq > 0 && mq <= uint32_t(kHitBuf)) {
        uint32_t v[kHitBuf];
#pragma unroll
        for (int r = 0; r < kHitBuf; ++r) v[r] = r < int(mq) ? hbuf[uint64_t(i) * kHitBuf + r] : ~0u;
#pragma unroll
        for (int a = 1; a < kHitBuf; ++a)
#pragma unroll
          for (int b = a; b > 0; --b)
            if (v[b - 1] > v[b]) {
              const uint32_t t = v[b];
              v[b] = v[b - 1];
              v[b - 1] = t;
            }
        for (uint32_t r = 0; r < mq; ++r)
          if (o + r < (unsigned long long)cap) {
            edges[2 * (o + r)] = i;
            edges[2 * (o + r) + 1] = v[r];
          }
      }
      o += mq;
    }
    __syncthreads();  // chunk_s and wsum are reused by the next chunk
  }
}

// Zeroes the hit counters, the write cursors and the one-pass emit's ticket
// and status words in one launch.
__global__ void __launch_bounds__(kThreads)
    zero_hit_state(uint32_t* __restrict__ counts, uint32_t* __restrict__ fill, uint32_t n,
                   unsigned long long* __restrict__ status, uint32_t n_status) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    counts[i] = 0u;
    fill[i] = 0u;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_status; i += stride)
    status[i] = 0ull;
}

// Count pass, the one-pass offsets and edges of the cells whose hits fit the
// hit buffer, write pass for the others, their ordering: shared by PIVOT,
// HALVES and ALLPAIRS. search(mode) launches the strategy's search pass;
// `scan` holds the emit's ticket and status words (one word per chunk + 1).
template <class Search>
cudaError_t hits_to_edges(DevCounters* ctr, size_t max_n, uint32_t* counts, uint32_t* hbuf,
                          unsigned long long* offsets, uint32_t* fill, void* scan,
                          uint32_t* edges, int64_t edges_cap, cudaStream_t s, Search search) {
  unsigned long long* status = static_cast<unsigned long long*>(scan);
  const uint32_t n_status = uint32_t((max_n + kHEChunk - 1) / kHEChunk + 1);
  zero_hit_state<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(counts, fill, uint32_t(max_n),
                                                                 status, n_status);
  count_launch();
  cudaError_t e;
  search(kCount);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ge = int(std::max<size_t>(
      1, std::min<size_t>(n_status - 1, size_t(sm_count()) * (2048 / kHEThreads))));
  hits_emit<<<ge, kHEThreads, 0, s>>>(ctr, uint32_t(max_n), counts, hbuf, offsets, status, edges,
                                     edges_cap, wait_limit(kHESpinLimit));
  count_launch();
  search(kWrite);
  count_launch();
  pivot_order<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(ctr, uint32_t(max_n), counts,
                                                             offsets, edges, edges_cap);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pivot_edges(const uint64_t* cells, int w64, int ell, int h, DevCounters* ctr,
                               size_t max_n, const uint64_t* key_by_cell, const uint32_t* sidx,
                               const void* table, size_t tcap,
                               uint32_t* counts, uint32_t* hbuf, unsigned long long* offsets,
                               uint32_t* fill, void* scan, uint32_t* edges, int64_t edges_cap,
                               cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  if (w64 > kMaxW) return cudaErrorInvalidValue;
  const int P = 1 << h;
  const size_t groups = P <= 32 ? (max_n + size_t(32 / P) - 1) / size_t(32 / P) : max_n;
  const int g = grid_for(groups, kThreads / 32);
  const ulonglong2* tb = static_cast<const ulonglong2*>(table);
  const uint32_t tmask = uint32_t(tcap - 1);
  const int tshift = table_shift(tcap);
  const int bits = key_bits(ell);
  return hits_to_edges(ctr, max_n, counts, hbuf, offsets, fill, scan, edges, edges_cap, s,
                       [&](int mode) {
                         if (mode == kCount)
                           pivot_search<kCount><<<g, kThreads, 0, s>>>(
                               cells, w64, ell, h, bits, ctr, uint32_t(max_n), key_by_cell, sidx,
                               tb, tmask, tshift, counts, hbuf, nullptr, nullptr, nullptr,
                               0);
                         else
                           pivot_search<kWrite><<<g, kThreads, 0, s>>>(
                               cells, w64, ell, h, bits, ctr, uint32_t(max_n), key_by_cell, sidx,
                               tb, tmask, tshift, counts, hbuf, offsets, fill, edges,
                               edges_cap);
                       });
}

cudaError_t launch_allpairs_edges(const uint64_t* cells, int w64, int ell, int h,
                                  DevCounters* ctr, size_t max_n, const uint64_t* key_by_cell,
                                  uint32_t* counts, uint32_t* hbuf, unsigned long long* offsets,
                                  uint32_t* fill, void* scan, uint32_t* edges, int64_t edges_cap,
                                  cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const int g = grid_for(max_n, kThreads / 32);
  const int bits = key_bits(ell);
  return hits_to_edges(ctr, max_n, counts, hbuf, offsets, fill, scan, edges, edges_cap, s,
                       [&](int mode) {
                         if (mode == kCount)
                           allpairs_search<kCount><<<g, kThreads, 0, s>>>(
                               cells, w64, h, bits, ctr, uint32_t(max_n), key_by_cell, counts,
                               hbuf, nullptr, nullptr, nullptr, 0);
                         else
                           allpairs_search<kWrite><<<g, kThreads, 0, s>>>(
                               cells, w64, h, bits, ctr, uint32_t(max_n), key_by_cell, counts,
                               hbuf, offsets, fill, edges, edges_cap);
                       });
}

int halves_split(int ell) { return ell / 2; }

int halves_sort_bits(int ell) { return ell <= 64 ? halves_split(ell) : 32; }

cudaError_t launch_halves_keys(const uint64_t* cells, int w64, int ell, DevCounters* ctr,
                               size_t max_n, uint64_t* hkey, uint64_t* fl, uint64_t* fh,
                               uint64_t* lkey, uint32_t* idx, cudaStream_t s, int64_t adopt_n) {
  if (max_n == 0) return cudaSuccess;
  if (adopt_n >= 0 && !(w64 >= 2 && w64 <= kKeysStageW)) return cudaErrorInvalidValue;
  if (w64 >= 2 && w64 <= kKeysStageW) {
    const size_t smem = size_t(kThreads) * (w64 + 1) * sizeof(uint64_t);
    halves_keys_staged<<<grid_for((max_n + 31) / 32, kThreads / 32), kThreads, smem, s>>>(
        cells, w64, halves_split(ell), ctr, uint32_t(max_n), hkey, fl, fh, lkey, idx, adopt_n,
        ell);
  } else {
    halves_keys<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(
        cells, w64, halves_split(ell), ctr, uint32_t(max_n), hkey, fl, fh, lkey, idx);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_halves_edges(const uint64_t* cells, int w64, int ell, DevCounters* ctr,
                                size_t max_n, const uint64_t* hkey, const uint64_t* fl,
                                const uint64_t* fh, const uint64_t* skey, const uint32_t* sidx,
                                uint64_t* sfh, uint32_t* counts, uint32_t* hbuf,
                                unsigned long long* offsets, uint32_t* fill, void* scan,
                                uint32_t* edges, int64_t edges_cap, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  const int sp = halves_split(ell);
  halves_gather<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(ctr, uint32_t(max_n), sidx, fh,
                                                               sfh);
  count_launch();
  const int g = grid_for(2 * max_n, kThreads);
  return hits_to_edges(ctr, max_n, counts, hbuf, offsets, fill, scan, edges, edges_cap, s,
                       [&](int mode) {
                         if (mode == kCount)
                           halves_search<kCount><<<g, kThreads, 0, s>>>(
                               cells, w64, sp, ctr, uint32_t(max_n), hkey, fl, skey, sidx, sfh,
                               counts, hbuf, nullptr, nullptr, nullptr, 0);
                         else
                           halves_search<kWrite><<<g, kThreads, 0, s>>>(
                               cells, w64, sp, ctr, uint32_t(max_n), hkey, fl, skey, sidx, sfh,
                               counts, hbuf, offsets, fill, edges, edges_cap);
                       });
}

size_t pivot_hit_words(size_t max_n) { return max_n * kHitBuf; }

}  // namespace cg
