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
// strategies). The search runs twice: once to count each cell's edges (an
// exclusive scan of the counts gives every cell's first output position), and
// once, over the cells that have edges, to write them; a last pass orders
// each cell's few edges by partner.
//
// Pivots: h cells spread over the sorted order (cells floor((2d+1) U / 2h)),
// so that they are far apart in value; the choice does not change the output.
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

// key of every cell (thread per cell): h distances of `bits` bits each.
__global__ void __launch_bounds__(kThreads)
    pivot_keys(const uint64_t* __restrict__ cells, int w, int h, int bits,
               const DevCounters* ctr, uint32_t max_n, uint64_t* __restrict__ key_by_cell,
               uint64_t* __restrict__ skeys, uint32_t* __restrict__ sidx) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  if (u == 0) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint64_t* xi = cells + uint64_t(i) * w;
    uint64_t key = 0;
    for (int d = 0; d < h; ++d) {
      const uint64_t* pd = cells + uint64_t(pivot_row(d, h, u)) * w;
      uint32_t dist = 0;
      for (int q = 0; q < w; ++q) dist += __popcll(xi[q] ^ pd[q]);
      key |= uint64_t(dist) << (bits * d);
    }
    key_by_cell[i] = key;
    skeys[i] = key;
    sidx[i] = i;
  }
}

// First position of every distinct key in the sorted key array, in an
// open-addressing table (key -> position).
__global__ void __launch_bounds__(kThreads)
    pivot_index(const uint64_t* __restrict__ skeys, const DevCounters* ctr, uint32_t max_n,
                uint64_t* __restrict__ tkeys, uint32_t* __restrict__ tvals, uint32_t tmask,
                int tshift, DevCounters* wctr) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < u; t += gridDim.x * blockDim.x) {
    const uint64_t key = skeys[t];
    if (t > 0 && skeys[t - 1] == key) continue;
    uint32_t slot = home_slot(key, tshift);
    bool placed = false;
    for (uint32_t probe = 0; probe <= tmask; ++probe) {
      const unsigned long long old =
          atomicCAS(reinterpret_cast<unsigned long long*>(tkeys + slot),
                    static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(key));
      if (old == kEmpty) {
        tvals[slot] = t;
        placed = true;
        break;
      }
      slot = (slot + 1) & tmask;
    }
    if (!placed) atomicOr(&wctr->overflow, 1u);
  }
}

__device__ __forceinline__ int64_t bucket_start(const uint64_t* tkeys, const uint32_t* tvals,
                                                uint32_t tmask, int tshift, uint64_t key) {
  uint32_t slot = home_slot(key, tshift);
  for (uint32_t probe = 0; probe <= tmask; ++probe) {
    const uint64_t cur = tkeys[slot];
    if (cur == key) return tvals[slot];
    if (cur == kEmpty) return -1;
    slot = (slot + 1) & tmask;
  }
  return -1;
}

// The search, in two modes. Lanes work on (cell, bucket pattern) pairs in
// parallel: with P = 2^h patterns, a warp takes 32 / P consecutive cells
// (P <= 32) or one cell with the patterns strided over the lanes (P > 32).
// Each lane looks its bucket up and compares every candidate j > i of it
// with cell i, word by word (XOR + popcount, stopping at the second
// difference).
//   kCount: counts[i] = number of hits of cell i.
//   kWrite: hit (i, j) goes to edges[offsets[i] + fill[i]++] (positions below
//           cap only); the order inside a cell's segment is fixed afterwards.
// Cells without hits are skipped in kWrite.
enum { kCount = 0, kWrite = 1 };

template <int kMode>
__global__ void __launch_bounds__(kThreads)
    pivot_search(const uint64_t* __restrict__ cells, int w, int ell, int h, int bits,
                 const DevCounters* ctr, uint32_t max_n, const uint64_t* __restrict__ key_by_cell,
                 const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ sidx,
                 const uint64_t* __restrict__ tkeys, const uint32_t* __restrict__ tvals,
                 uint32_t tmask, int tshift, uint32_t* __restrict__ counts,
                 const unsigned long long* __restrict__ offsets, uint32_t* __restrict__ fill,
                 uint32_t* __restrict__ edges, int64_t cap) {
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
    if (kMode == kWrite && counts[i] == 0) continue;
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
      const int64_t t0 = bucket_start(tkeys, tvals, tmask, tshift, target);
      if (t0 < 0) continue;
      for (uint32_t t = uint32_t(t0); t < u && skeys[t] == target; ++t) {
        const uint32_t j = sidx[t];
        if (j <= i) continue;
        const uint64_t* xj = cells + uint64_t(j) * w;
        int c = 0;
        for (int q = 0; q < w && c < 2; ++q) c += __popcll(xj[q] ^ xi[q]);
        if (c != 1) continue;
        if (kMode == kCount) {
          atomicAdd(&counts[i], 1u);
        } else {
          const unsigned long long pos = offsets[i] + atomicAdd(&fill[i], 1u);
          if (pos < (unsigned long long)cap) {
            edges[2 * pos] = i;
            edges[2 * pos + 1] = j;
          }
        }
      }
    }
  }
}

// Puts every cell's edges in increasing order of j (insertion sort of the
// segment; segments are short: at most the cell's degree). Segments that do
// not lie wholly below cap are left alone (the call then reports capacity).
__global__ void __launch_bounds__(kThreads)
    pivot_order(const DevCounters* ctr, uint32_t max_n, const uint32_t* __restrict__ counts,
                const unsigned long long* __restrict__ offsets, uint32_t* __restrict__ edges,
                int64_t cap) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t m = counts[i];
    if (m < 2) continue;
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
  pivot_keys<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(
      cells, w64, h, key_bits(ell), ctr, uint32_t(max_n), key_by_cell, skeys, sidx);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pivot_index(const uint64_t* skeys, const DevCounters* ctr, size_t max_n,
                               uint64_t* tkeys, uint32_t* tvals, size_t tcap, DevCounters* wctr,
                               cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  pivot_index<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(
      skeys, ctr, uint32_t(max_n), tkeys, tvals, uint32_t(tcap - 1), table_shift(tcap), wctr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pivot_search(const uint64_t* cells, int w64, int ell, int h,
                                const DevCounters* ctr, size_t max_n,
                                const uint64_t* key_by_cell, const uint64_t* skeys,
                                const uint32_t* sidx, const uint64_t* tkeys, const uint32_t* tvals,
                                size_t tcap, uint32_t* counts, const unsigned long long* offsets,
                                uint32_t* fill, uint32_t* edges, int64_t edges_cap, bool write,
                                cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  if (w64 > kMaxW) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(write ? fill : counts, 0, max_n * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const int P = 1 << h;
  const size_t groups = P <= 32 ? (max_n + size_t(32 / P) - 1) / size_t(32 / P) : max_n;
  auto kern = write ? pivot_search<kWrite> : pivot_search<kCount>;
  kern<<<grid_for(groups, kThreads / 32), kThreads, 0, s>>>(
      cells, w64, ell, h, key_bits(ell), ctr, uint32_t(max_n), key_by_cell, skeys, sidx, tkeys,
      tvals, uint32_t(tcap - 1), table_shift(tcap), counts, offsets, fill, edges, edges_cap);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pivot_order(const DevCounters* ctr, size_t max_n, const uint32_t* counts,
                               const unsigned long long* offsets, uint32_t* edges,
                               int64_t edges_cap, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  pivot_order<<<grid_for(max_n, kThreads), kThreads, 0, s>>>(ctr, uint32_t(max_n), counts,
                                                             offsets, edges, edges_cap);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cg
