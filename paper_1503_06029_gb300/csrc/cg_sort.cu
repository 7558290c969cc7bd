// Sorting and scanning for step 2 (cells, §3.2: "sorting ... using the radix
// sort algorithm") and step 4 (edge offsets).
//
// Stable LSD radix sort, 8-bit digits, one histogram kernel and one scatter
// kernel per pass (plus a device-wide scan of the per-tile histograms when
// there are more than kInlineTiles tiles). Item counts are read from device
// memory, so a whole build can be enqueued without reading anything back.
#include <cooperative_groups.h>

#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kRThreads = 256;
constexpr int kRItems = 8;
constexpr int kRTile = kRThreads * kRItems;  // 2048 items per tile
constexpr int kInlineTiles = 64;             // scatter sums histograms itself below this
constexpr int kSThreads = 256;
constexpr int kSItems = 16;
constexpr int kSTile = kSThreads * kSItems;  // 4096 items per scan block

// Item count read from device memory: mul * ceil(min(*n, cap) / div).
struct Count {
  const unsigned int* n;
  unsigned int mul;
  unsigned int div;
  uint64_t cap;  // the count never exceeds the buffers sized for it
  __device__ __forceinline__ uint64_t get() const {
    const uint64_t v = uint64_t(*n) < cap ? uint64_t(*n) : cap;
    return uint64_t(mul) * ((v + div - 1) / div);
  }
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Inclusive warp scan of 64-bit values.
__device__ __forceinline__ unsigned long long warp_incl(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan over the block (blockDim.x <= 1024); returns the exclusive
// prefix of `v` and the block total through *total.
__device__ unsigned long long block_excl(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long wsum[32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const unsigned long long inc = warp_incl(v);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long s = lane < nw ? wsum[lane] : 0ull;
    s = warp_incl(s);
    if (lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  const unsigned long long before = warp > 0 ? wsum[warp - 1] : 0ull;
  if (total) *total = wsum[nw - 1];
  __syncthreads();
  return before + inc - v;
}

// --------------------------------- scan ---------------------------------

__global__ void __launch_bounds__(kSThreads)
    scan_reduce(const uint32_t* __restrict__ in, Count cnt, unsigned long long* partial) {
  const uint64_t n = cnt.get();
  const uint64_t base = uint64_t(blockIdx.x) * kSTile;
  if (base >= n) return;
  unsigned long long s = 0;
  for (int j = 0; j < kSItems; ++j) {
    const uint64_t i = base + uint64_t(j) * kSThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  unsigned long long tot;
  block_excl(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
    scan_partials(unsigned long long* partial, Count cnt, unsigned long long* total) {
  const uint64_t n = cnt.get();
  const uint64_t nb = (n + kSTile - 1) / kSTile;
  unsigned long long carry = 0;
  for (uint64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const uint64_t i = b0 + threadIdx.x;
    const unsigned long long v = i < nb ? partial[i] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl(v, &tot);
    if (i < nb) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kSThreads)
    scan_down(const uint32_t* __restrict__ in, Count cnt, const unsigned long long* partial,
              unsigned long long* out) {
  const uint64_t n = cnt.get();
  const uint64_t base = uint64_t(blockIdx.x) * kSTile;
  if (base >= n) return;
  // Thread t owns items base + t*kSItems .. +kSItems-1 (consecutive).
  uint32_t v[kSItems];
  unsigned long long s = 0;
  const uint64_t first = base + uint64_t(threadIdx.x) * kSItems;
#pragma unroll
  for (int j = 0; j < kSItems; ++j) {
    v[j] = (first + j < n) ? in[first + j] : 0u;
    s += v[j];
  }
  unsigned long long run = partial[blockIdx.x] + block_excl(s, nullptr);
#pragma unroll
  for (int j = 0; j < kSItems; ++j) {
    if (first + j < n) out[first + j] = run;
    run += v[j];
  }
}

cudaError_t scan_impl(const uint32_t* in, unsigned long long* out, Count cnt, size_t max_n,
                      unsigned long long* total, void* scratch, cudaStream_t s) {
  const size_t nb = (max_n + kSTile - 1) / kSTile;
  if (nb == 0) {
    // Nothing can be scanned; still define the total.
    scan_partials<<<1, 1024, 0, s>>>(static_cast<unsigned long long*>(scratch), cnt, total);
    count_launch();
    return cudaGetLastError();
  }
  auto* partial = static_cast<unsigned long long*>(scratch);
  scan_reduce<<<unsigned(nb), kSThreads, 0, s>>>(in, cnt, partial);
  scan_partials<<<1, 1024, 0, s>>>(partial, cnt, total);
  scan_down<<<unsigned(nb), kSThreads, 0, s>>>(in, cnt, partial, out);
  count_launch(3);
  return cudaGetLastError();
}

// --------------------------------- radix ---------------------------------

__global__ void __launch_bounds__(kRThreads)
    radix_hist(const uint64_t* __restrict__ kin, const unsigned int* n_dev, uint32_t max_n,
               int shift, uint32_t* hist) {
  __shared__ uint32_t h[256];
  const uint32_t n = min(*n_dev, max_n);
  const uint32_t tiles = (n + kRTile - 1) / kRTile;
  const uint32_t t = blockIdx.x;
  if (t >= tiles) return;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = uint64_t(t) * kRTile;
#pragma unroll
  for (int j = 0; j < kRItems; ++j) {
    const uint64_t i = base + uint64_t(j) * kRThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(kin[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[uint64_t(threadIdx.x) * tiles + t] = h[threadIdx.x];
}

// Scatter of one pass. Items of a tile are read "warp-striped" (warp w owns a
// contiguous run of 256 items, lane l the items w*256 + j*32 + l), and ranked
// in that order, which is the input order: the sort is stable.
template <bool kVals>
__global__ void __launch_bounds__(kRThreads)
    radix_scatter(const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout,
                  const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout,
                  const unsigned int* n_dev, uint32_t max_n, int shift,
                  const uint32_t* __restrict__ hist,
                  const unsigned long long* __restrict__ scanned) {
  __shared__ uint32_t wcnt[kRThreads / 32][256];
  __shared__ uint32_t toff[256];
  const uint32_t n = min(*n_dev, max_n);
  const uint32_t tiles = (n + kRTile - 1) / kRTile;
  const uint32_t t = blockIdx.x;
  if (t >= tiles) return;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int d = threadIdx.x;

  // Global offset of digit d for this tile.
  if (scanned) {
    toff[d] = uint32_t(scanned[uint64_t(d) * tiles + t]);
  } else {
    unsigned long long tot = 0, before = 0;
    for (uint32_t u = 0; u < tiles; ++u) {
      const uint32_t c = hist[uint64_t(d) * tiles + u];
      if (u < t) before += c;
      tot += c;
    }
    const unsigned long long dbase = block_excl(tot, nullptr);
    toff[d] = uint32_t(dbase + before);
  }
#pragma unroll
  for (int w = 0; w < kRThreads / 32; ++w) wcnt[w][d] = 0;
  __syncthreads();

  const uint64_t base = uint64_t(t) * kRTile + uint64_t(warp) * (kRItems * 32);
  uint64_t key[kRItems];
  uint32_t val[kRItems];
  uint32_t loc[kRItems];
  uint32_t dig[kRItems];
#pragma unroll
  for (int j = 0; j < kRItems; ++j) {
    const uint64_t i = base + uint64_t(j) * 32 + lane;
    const bool ok = i < n;
    key[j] = ok ? kin[i] : 0ull;
    if (kVals) val[j] = ok ? vin[i] : 0u;
    const uint32_t dj = ok ? uint32_t((key[j] >> shift) & 255u) : 256u;
    dig[j] = dj;
    const uint32_t peers = __match_any_sync(0xffffffffu, dj);
    const uint32_t rank = __popc(peers & lanemask_lt());
    const int leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (ok) b = wcnt[warp][dj];
    __syncwarp();
    if (ok && lane == leader) wcnt[warp][dj] = b + __popc(peers);
    __syncwarp();
    loc[j] = b + rank;
  }
  __syncthreads();
  {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRThreads / 32; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRItems; ++j) {
    if (dig[j] < 256u) {
      const uint32_t pos = toff[dig[j]] + wcnt[warp][dig[j]] + loc[j];
      kout[pos] = key[j];
      if (kVals) vout[pos] = val[j];
    }
  }
}

// ------------------------- one-cluster radix sort -------------------------
//
// For up to a few hundred thousand distinct vectors the multi-launch radix sort
// is launch-bound. Here one thread-block cluster (8 or 16 CTAs, one per SM)
// holds all keys in its distributed shared memory: CTA r owns positions
// [r*per, (r+1)*per). Each 8-bit pass: local histograms -> cluster barrier ->
// every CTA reads all histograms over DSMEM and derives its digit offsets ->
// stable warp-level ranking -> each key is stored straight into the shared
// memory of the CTA that owns its new position -> cluster barrier. A pass
// whose digit is the same for every key is skipped.

constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;

// Keys of W 64-bit words (word W-1 most significant); LSD over the words, 8
// bits per pass; the top word has `top_bits` significant bits. Input row i is
// in[rows[i]] (or in[i] without `rows`).
template <int W>
__global__ void __launch_bounds__(kCThreads)
    cluster_sort_kernel(const uint64_t* __restrict__ in, const uint32_t* __restrict__ rows,
                        const unsigned int* n_dev, uint32_t max_n, int top_bits,
                        ClusterSortOut o, uint32_t per_cap) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cluster = cgx::this_cluster();
  extern __shared__ __align__(16) uint64_t cbuf[];
  __shared__ uint32_t hist[256];
  __shared__ uint32_t wcnt[kCWarps][256];
  __shared__ uint32_t toff[256];
  __shared__ uint32_t wtot[8];
  __shared__ int skip;
  griddep_wait();
  griddep_release();
  // Same values for every CTA of the cluster: a table overflow, or the rank
  // sort (few distinct vectors) already did this work.
  if (o.ctr->overflow || o.ctr->sorted) return;
  const uint32_t C = cluster.num_blocks();
  const uint32_t r = cluster.block_rank();
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  if (*n_dev > max_n) {  // more vectors than this cluster holds: the fallback sorts them
    if (r == 0 && tid == 0) o.ctr->sorted = 0u;
    return;
  }
  const uint32_t n = *n_dev;
  const uint32_t per = (n + C - 1) / C;
  const uint32_t lo = min(r * per, n);
  const uint32_t cnt = min(lo + per, n) - lo;
  uint64_t* cur = cbuf;
  uint64_t* nxt = cbuf + size_t(per_cap) * W;
  for (uint32_t i = tid; i < cnt; i += kCThreads) {
    const uint64_t src = rows ? uint64_t(rows[lo + i]) : uint64_t(lo + i);
#pragma unroll
    for (int w = 0; w < W; ++w) cur[size_t(i) * W + w] = in[src * W + w];
  }
  const uint32_t sw = (cnt + kCWarps - 1) / kCWarps;  // items per warp (contiguous)
  const uint32_t wlo = min(warp * sw, cnt);
  const uint32_t whi = min(wlo + sw, cnt);

  for (int wd = 0; wd < W; ++wd) {
    const int bits = wd == W - 1 ? top_bits : 64;
    for (int shift = 0; shift < bits; shift += 8) {
      if (tid < 256) hist[tid] = 0;
      if (tid == 0) skip = 0;
      __syncthreads();
      for (uint32_t i = tid; i < cnt; i += kCThreads)
        atomicAdd(&hist[(cur[size_t(i) * W + wd] >> shift) & 255u], 1u);
      cluster.sync();
      uint32_t tot = 0, before = 0;
      if (tid < 256) {
        for (uint32_t q = 0; q < C; ++q) {
          const uint32_t v = cluster.map_shared_rank(hist, q)[tid];
          tot += v;
          if (q < r) before += v;
        }
        if (n > 0 && tot == n) skip = 1;
      }
      uint32_t inc = tot;
#pragma unroll
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o2);
        if (lane >= o2) inc += t;
      }
      if (tid < 256 && lane == 31) wtot[warp] = inc;
      for (int w = 0; w < kCWarps; ++w)
        if (tid < 256) wcnt[w][tid] = 0;
      __syncthreads();
      if (tid < 256) {
        uint32_t bw = 0;
        for (int w = 0; w < warp; ++w) bw += wtot[w];
        toff[tid] = bw + inc - tot + before;
      }
      __syncthreads();
      if (!skip) {
        // Count per warp and digit, in item order.
        for (uint32_t b = wlo; b < whi; b += 32) {
          const uint32_t i = b + lane;
          const bool ok = i < whi;
          const uint32_t d = ok ? uint32_t((cur[size_t(i) * W + wd] >> shift) & 255u) : 256u;
          const uint32_t peers = __match_any_sync(0xffffffffu, d);
          if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
          __syncwarp();
        }
        __syncthreads();
        if (tid < 256) {
          uint32_t run = toff[tid];
          for (int w = 0; w < kCWarps; ++w) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
          }
        }
        __syncthreads();
        // Rank and store into the owner CTA's buffer.
        for (uint32_t b = wlo; b < whi; b += 32) {
          const uint32_t i = b + lane;
          const bool ok = i < whi;
          const uint32_t d = ok ? uint32_t((cur[size_t(i) * W + wd] >> shift) & 255u) : 256u;
          const uint32_t peers = __match_any_sync(0xffffffffu, d);
          uint32_t pos = 0;
          if (ok) pos = wcnt[warp][d] + __popc(peers & lanemask_lt());
          __syncwarp();
          if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
          __syncwarp();
          if (ok) {
            const uint32_t dst = pos / per;
            uint64_t* remote = cluster.map_shared_rank(nxt, dst) + size_t(pos - dst * per) * W;
#pragma unroll
            for (int w = 0; w < W; ++w) remote[w] = cur[size_t(i) * W + w];
          }
        }
      }
      cluster.sync();
      if (!skip) {
        uint64_t* t = cur;
        cur = nxt;
        nxt = t;
      }
    }
  }

  // Outputs: internal cells, the caller's copy, and (l <= 64) the numbers.
  const bool user = o.user_cells && int64_t(n) <= o.user_cap;
  const int wc = (o.ell + o.word_bits - 1) / o.word_bits;
  for (uint32_t i = tid; i < cnt; i += kCThreads) {
    const uint32_t g = lo + i;
#pragma unroll
    for (int w = 0; w < W; ++w) o.cells[size_t(g) * W + w] = cur[size_t(i) * W + w];
    if (user) {
      if (o.word_bits == 64) {
#pragma unroll
        for (int w = 0; w < W; ++w)
          static_cast<uint64_t*>(o.user_cells)[size_t(g) * W + w] = cur[size_t(i) * W + w];
      } else {
        uint32_t* u32 = static_cast<uint32_t*>(o.user_cells) + uint64_t(g) * wc;
        for (int c = 0; c < wc; ++c) u32[c] = uint32_t(cur[size_t(i) * W + c / 2] >> (32 * (c & 1)));
      }
    }
    if (W == 1 && o.t.keys) {
      const uint64_t key = cur[i];
      if (key == kEmpty) {
        o.ctr->ones_rank = g;
      } else {
        const int64_t slot = small_find_slot(o.t.keys, o.t.mask, o.t.shift, key);
        if (slot >= 0) o.t.vals[slot] = g;
        else atomicOr(&o.ctr->error, 1u);
      }
    }
  }
  if (r == 0 && tid == 0) o.ctr->sorted = 1u;
}

template <int W>
cudaError_t cluster_sort_w(const uint64_t* in, const uint32_t* rows, const unsigned int* n_dev,
                           size_t max_n, int top_bits, const ClusterSortOut& o, cudaStream_t s,
                           bool* done, bool* tried) {
  constexpr size_t kStaticSmem = 20 * 1024;
  constexpr size_t kMaxDyn = 227 * 1024 - kStaticSmem;
  constexpr size_t kMaxPer = kMaxDyn / (2 * W * sizeof(uint64_t));
  static int cluster16 = -1;  // 1 if a 16-CTA cluster of this kernel can run
  auto kern = cluster_sort_kernel<W>;
  const bool certain = max_n <= 8 * kMaxPer || (cluster16 != 0 && max_n <= 16 * kMaxPer);
  if (!certain && !tried) return cudaSuccess;
  for (int C : {16, 8}) {
    // At full capacity when max_n may not fit: the kernel checks the count.
    const size_t per = certain ? (max_n + C - 1) / C : kMaxPer;
    const size_t dyn = 2 * std::max<size_t>(per, 1) * W * sizeof(uint64_t);
    if (dyn > kMaxDyn) continue;
    const size_t cap_n = certain ? max_n : per * C;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(kern), dyn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kCThreads, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    if (C == 16 && cluster16 == 0) continue;
    if (C == 16 && cluster16 < 0) {
      // First use: allow 16-CTA clusters and check that one fits on an SM set.
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cluster16 = 0;
        continue;
      }
      int nclusters = 0;
      e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
      if (e != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        cluster16 = 0;
        continue;
      }
      cluster16 = 1;
    }
    e = cudaLaunchKernelEx(&cfg, kern, in, rows, n_dev, uint32_t(cap_n), top_bits, o,
                           uint32_t(per));
    if (e != cudaSuccess && C == 16) {
      // A 16-CTA cluster with this much shared memory does not fit: the launch
      // is refused before it starts; use 8-CTA clusters instead.
      cudaGetLastError();
      continue;
    }
    if (e != cudaSuccess) return e;
    count_launch();
    if (certain) *done = true;
    else *tried = true;
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ------------------------- rank sort of few vectors -------------------------
//
// For up to kRankMax distinct vectors of one word the cluster sort's eight
// barrier-separated passes cost more than counting: the rank of key k_i among
// distinct keys is #{j : k_j < k_i}. rank_count splits the n^2 comparisons
// over (256 keys) x (one of kRankSplits slices of all keys) blocks: a block
// stages its slice in shared memory (every thread reads the same entry, a
// broadcast) and adds each key's partial count to the key's value slot in
// the dedup table (zeroed by the build's clear; the all-ones vector, which
// has no slot, counts in ctr->ones_rank). rank_place then writes every key at
// its rank, with the same outputs as the cluster sort (internal cells, the
// caller's copy, the cell number already in the table).
constexpr uint32_t kRankMax = 12288;
constexpr int kRankSplits = 16;
constexpr uint32_t kRankSlice = (kRankMax + kRankSplits - 1) / kRankSplits;  // 768
constexpr int kRankThreads = 256;

__device__ __forceinline__ bool rank_applies(const ClusterSortOut& o, uint32_t n, uint32_t max_n) {
  return !o.ctr->overflow && n <= kRankMax && n <= max_n && o.t.keys != nullptr;
}

__global__ void __launch_bounds__(kRankThreads)
    rank_count(const uint64_t* __restrict__ in, const unsigned int* n_dev, uint32_t max_n,
               ClusterSortOut o) {
  __shared__ ulonglong2 sk[kRankSlice / 2 + 1];
  griddep_wait();
  griddep_release();
  const uint32_t n = *n_dev;
  if (!rank_applies(o, n, max_n)) return;  // the cluster sort takes it
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) o.ctr->sorted = 1u;
  const uint32_t i0 = blockIdx.x * kRankThreads;
  if (i0 >= n) return;
  const uint32_t per = (n + kRankSplits - 1) / kRankSplits;
  const uint32_t j0 = min(n, blockIdx.y * per);
  const uint32_t m = min(n, j0 + per) - j0;
  uint64_t* flat = reinterpret_cast<uint64_t*>(sk);
  for (uint32_t t = threadIdx.x; t < m; t += kRankThreads) flat[t] = __ldg(in + j0 + t);
  if (threadIdx.x == 0) flat[m] = kEmpty;  // pad: no key is above the all-ones value
  __syncthreads();
  const uint32_t i = i0 + threadIdx.x;
  if (i >= n || m == 0) return;
  const uint64_t ki = __ldg(in + i);
  uint32_t c0 = 0, c1 = 0;
  const uint32_t pairs = (m + 1) / 2;
#pragma unroll 8
  for (uint32_t q = 0; q < pairs; ++q) {
    const ulonglong2 v = sk[q];
    c0 += v.x < ki;
    c1 += v.y < ki;
  }
  const uint32_t c = c0 + c1;
  if (c == 0) return;
  if (ki == kEmpty) {
    atomicAdd(&o.ctr->ones_rank, c);
  } else {
    const int64_t slot = small_find_slot(o.t.keys, o.t.mask, o.t.shift, ki);
    if (slot >= 0) atomicAdd(&o.t.vals[slot], c);
    else atomicOr(&o.ctr->error, 1u);
  }
}

__global__ void __launch_bounds__(kRankThreads)
    rank_place(const uint64_t* __restrict__ in, const unsigned int* n_dev, uint32_t max_n,
               ClusterSortOut o) {
  griddep_wait();
  griddep_release();
  const uint32_t n = *n_dev;
  if (!rank_applies(o, n, max_n)) return;
  const bool user = o.user_cells && int64_t(n) <= o.user_cap;
  for (uint32_t i = blockIdx.x * kRankThreads + threadIdx.x; i < n;
       i += gridDim.x * kRankThreads) {
    const uint64_t ki = in[i];
    uint32_t g;
    if (ki == kEmpty) {
      g = o.ctr->ones_rank;
    } else {
      const int64_t slot = small_find_slot(o.t.keys, o.t.mask, o.t.shift, ki);
      if (slot < 0) continue;  // reported by rank_count
      g = o.t.vals[slot];
    }
    if (g >= n) {
      atomicOr(&o.ctr->error, 1u);
      continue;
    }
    o.cells[g] = ki;
    if (user) {
      if (o.word_bits == 64) {
        static_cast<uint64_t*>(o.user_cells)[g] = ki;
      } else {
        const int wc = (o.ell + 31) / 32;
        uint32_t* u32 = static_cast<uint32_t*>(o.user_cells) + uint64_t(g) * wc;
        for (int c = 0; c < wc; ++c) u32[c] = uint32_t(ki >> (32 * c));
      }
    }
  }
}

// ------------------------- merge sort of wide rows -------------------------
//
// Rows of W = ceil(l / 64) words (l > 64), referenced by row number, are put in
// value order by a comparison merge sort: each item carries the 128 most
// significant bits of its row (bits [l - 128, l), zero-filled below bit 0) as
// a cached key, and only items with equal cached keys compare their whole
// rows (most significant word first); for l <= 128 the cached key is the whole
// row. Tiles of items are sorted in shared memory (bitonic network), then runs
// are merged pairwise (merge path: each block finds its diagonal split by
// binary search and merges one output tile); ceil(log2(U / tile)) passes.
//
// The kernels are generic over an order: Ord::Tag is the payload carried with
// each cached key, Ord::pad() a tag larger than every item, Ord::load(g)
// produces input item g and Ord::less compares two items. RowOrder sorts one
// scene's rows; BatchOrder (batch sort) sorts the distinct vectors of many
// scenes at once, scene by scene.

constexpr int kMThreads = 256;
constexpr uint32_t kPad = 0xffffffffu;

// Bits [off, off + 64) of a row (positions below 0 read as zero, off > -64).
struct RowOrder {
  using Tag = uint32_t;  // row number
  static constexpr int kItems = 8;
  static constexpr bool kPadAware = false;
  __device__ __forceinline__ static bool is_pad(const Tag&) { return false; }
  const uint64_t* rows;
  int w;
  int ell;
  bool full;                // the cached key is the whole row (l <= 128)
  const uint32_t* idx_in;   // input row numbers (nullable: item g is row g)
  __device__ __forceinline__ static Tag pad() { return kPad; }
  __device__ __forceinline__ void load(uint32_t g, ulonglong2* k, Tag* t) const {
    const uint32_t r = idx_in ? idx_in[g] : g;
    *t = r;
    *k = top128(rows + uint64_t(r) * w, ell);
  }
  // a < b; the padding item is larger than everything.
  __device__ __forceinline__ bool less(const ulonglong2& ka, Tag ia, const ulonglong2& kb,
                                       Tag ib) const {
    if (ia == kPad) return false;
    if (ib == kPad) return true;
    if (ka.x != kb.x) return ka.x < kb.x;
    if (ka.y != kb.y) return ka.y < kb.y;
    if (full) return ia < ib;
    const uint64_t* ra = rows + uint64_t(ia) * w;
    const uint64_t* rb = rows + uint64_t(ib) * w;
    for (int q = w - 1; q >= 0; --q)
      if (ra[q] != rb[q]) return ra[q] < rb[q];
    return ia < ib;
  }
};

struct BatchOrder {
  using Tag = uint2;  // (scene, index of the distinct vector within it)
  static constexpr int kItems = 4;
  const BatchSortScene* scenes;
  const ulonglong2* keys_in;
  const uint2* tags_in;
  __device__ __forceinline__ static Tag pad() { return make_uint2(kPad, kPad); }
  // Each scene's items sit at the front of its segment and padding after
  // them, in both buffers and after every pass: a tile or merge block whose
  // first position holds padding is all padding and has nothing to do.
  static constexpr bool kPadAware = true;
  __device__ __forceinline__ static bool is_pad(const Tag& t) { return t.x == kPad; }
  __device__ __forceinline__ void load(uint32_t g, ulonglong2* k, Tag* t) const {
    *k = keys_in[g];
    *t = tags_in[g];
  }
  __device__ __forceinline__ bool less(const ulonglong2& ka, Tag ta, const ulonglong2& kb,
                                       Tag tb) const {
    if (ta.x != tb.x) return ta.x < tb.x;  // scene first (padding has the largest)
    if (ta.x == kPad) return false;
    if (ka.x != kb.x) return ka.x < kb.x;
    if (ka.y != kb.y) return ka.y < kb.y;
    const BatchSortScene& sc = scenes[ta.x];
    if (sc.ell <= 128) return ta.y < tb.y;  // whole vector cached: distinct keys differ
    const uint64_t* ra = sc.keys64 + uint64_t(sc.idx[ta.y]) * sc.w;
    const uint64_t* rb = sc.keys64 + uint64_t(sc.idx[tb.y]) * sc.w;
    for (int q = sc.w - 1; q >= 0; --q)
      if (ra[q] != rb[q]) return ra[q] < rb[q];
    return ta.y < tb.y;
  }
};

// Segmented merge sorts (the batch sort): segments of 2^e positions, e = 10 ..
// 31, laid out largest first; classes[2 e], classes[2 e + 1] bound the
// positions of the segments of size 2^e.
constexpr int kSegClasses = 32;

// Segment size (2^e) at position g, from the class table.
__device__ __forceinline__ uint32_t seg_size_at(const uint32_t* classes, uint32_t g) {
  for (int e = kSegClasses - 1; e >= 10; --e)
    if (g >= classes[2 * e] && g < classes[2 * e + 1]) return 1u << e;
  return 0u;
}

// Tile sort: input items [b * tile, ...), with their cached keys.
template <class Ord>
__global__ void __launch_bounds__(kMThreads)
    msort_tiles(Ord ord, const unsigned int* n_dev, uint32_t max_n, ulonglong2* __restrict__ kout,
                typename Ord::Tag* __restrict__ tout, const unsigned int* skip) {
  constexpr int kTile = kMThreads * Ord::kItems;
  using Tag = typename Ord::Tag;
  __shared__ ulonglong2 sk[kTile];
  __shared__ Tag st[kTile];
  if (skip && *skip) return;
  const uint32_t n = min(*n_dev, max_n);
  const uint32_t base = blockIdx.x * kTile;
  if (base >= n) return;
  if constexpr (Ord::kPadAware) {
    // Sorted in place (the input is kout/tout): a padding tile stays as it is.
    if (Ord::is_pad(tout[base])) return;
  }
  for (int t = threadIdx.x; t < kTile; t += kMThreads) {
    const uint32_t g = base + t;
    if (g < n) {
      ord.load(g, &sk[t], &st[t]);
    } else {
      st[t] = Ord::pad();
      sk[t] = make_ulonglong2(~0ull, ~0ull);
    }
  }
  __syncthreads();
  for (int k = 2; k <= kTile; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kTile; t += kMThreads) {
        const int p = t ^ j;
        if (p > t) {
          const bool up = (t & k) == 0;
          const bool swap = up ? ord.less(sk[p], st[p], sk[t], st[t])
                               : ord.less(sk[t], st[t], sk[p], st[p]);
          if (swap) {
            const ulonglong2 tk = sk[t];
            sk[t] = sk[p];
            sk[p] = tk;
            const Tag tt = st[t];
            st[t] = st[p];
            st[p] = tt;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kTile; t += kMThreads) {
    const uint32_t g = base + t;
    if (g < n) {
      kout[g] = sk[t];
      tout[g] = st[t];
    }
  }
}

// Number of items of A among the first d items of merge(A, B).
template <class Ord>
__device__ __forceinline__ uint32_t merge_split(const Ord& ord, const ulonglong2* ka,
                                                const typename Ord::Tag* ia, uint32_t la,
                                                const ulonglong2* kb,
                                                const typename Ord::Tag* ib, uint32_t lb,
                                                uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0;
  uint32_t hi = d < la ? d : la;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t bj = d - 1 - mid;
    if (ord.less(kb[bj], ib[bj], ka[mid], ia[mid])) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// merge_split by one whole warp: 33-way search instead of a binary one (each
// round the lanes test 32 points of the remaining range along the diagonal),
// so a split over runs of millions of items costs about five dependent
// rounds of loads instead of twenty-odd. Every lane returns the result.
template <class Ord>
__device__ __forceinline__ uint32_t merge_split_warp(const Ord& ord, const ulonglong2* ka,
                                                     const typename Ord::Tag* ia, uint32_t la,
                                                     const ulonglong2* kb,
                                                     const typename Ord::Tag* ib, uint32_t lb,
                                                     uint32_t d) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lo = d > lb ? d - lb : 0;
  uint32_t hi = d < la ? d : la;
  // Answer: the first i in [lo, hi) with less(B[d - 1 - i], A[i]), else hi.
  while (lo < hi) {
    const uint32_t len = hi - lo;
    const bool few = len <= 32;
    const uint32_t p = few ? lo + lane : lo + uint32_t((uint64_t(len) * (lane + 1)) / 33);
    const bool live = few ? lane < len : true;
    const bool f = live && ord.less(kb[d - 1 - p], ib[d - 1 - p], ka[p], ia[p]);
    const uint32_t m = __ballot_sync(0xffffffffu, f);
    if (few) return m ? lo + uint32_t(__ffs(m) - 1) : hi;
    if (m == 0) {
      lo = __shfl_sync(0xffffffffu, p, 31) + 1;
    } else {
      const int j = __ffs(m) - 1;
      hi = __shfl_sync(0xffffffffu, p, j);
      if (j > 0) lo = __shfl_sync(0xffffffffu, p, j - 1) + 1;
    }
  }
  return lo;
}

// One merge pass: sorted runs of `width` items merged pairwise into runs of
// 2 * width; block b writes output items [b * tile, (b + 1) * tile). Warps 0
// and 1 find the block's two splits; every thread merges kItems outputs into
// registers, which go back through shared memory for coalesced stores.
template <class Ord>
__global__ void __launch_bounds__(kMThreads)
    msort_merge(Ord ord, const ulonglong2* __restrict__ kin,
                const typename Ord::Tag* __restrict__ iin, ulonglong2* __restrict__ kout,
                typename Ord::Tag* __restrict__ iout, const unsigned int* n_dev, uint32_t max_n,
                uint32_t width, const unsigned int* skip, const uint32_t* seg_classes) {
  constexpr int kTile = kMThreads * Ord::kItems;
  using Tag = typename Ord::Tag;
  __shared__ ulonglong2 sk[kTile];
  __shared__ Tag si[kTile];
  __shared__ uint32_t s_split[2];
  if (skip && *skip) return;
  const uint32_t n = min(*n_dev, max_n);
  const uint32_t out0 = blockIdx.x * kTile;
  if (out0 >= n) return;
  // Segmented sort: a segment no larger than the run width is sorted already.
  if (seg_classes && seg_size_at(seg_classes, out0) <= width) return;
  if constexpr (Ord::kPadAware) {
    // Padding from here to the end of the tile, and already in kout/iout.
    if (Ord::is_pad(iin[out0])) return;
  }
  const uint32_t s0 = (out0 / (2 * width)) * (2 * width);
  const uint32_t a_end = min(s0 + width, n);
  const uint32_t b_end = min(s0 + 2 * width, n);
  const uint32_t la = a_end - s0, lb = b_end - a_end;
  const uint32_t d0 = out0 - s0;
  const uint32_t d1 = min(d0 + uint32_t(kTile), la + lb);
  const ulonglong2* ka = kin + s0;
  const Tag* ia = iin + s0;
  const ulonglong2* kb = kin + a_end;
  const Tag* ib = iin + a_end;
  if (threadIdx.x < 64) {
    const uint32_t sp =
        merge_split_warp(ord, ka, ia, la, kb, ib, lb, threadIdx.x < 32 ? d0 : d1);
    if ((threadIdx.x & 31) == 0) s_split[threadIdx.x >> 5] = sp;
  }
  __syncthreads();
  const uint32_t a0 = s_split[0], a1 = s_split[1];
  const uint32_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t na = a1 - a0, nb = b1 - b0;
  for (uint32_t t = threadIdx.x; t < na + nb; t += kMThreads) {
    if (t < na) {
      sk[t] = ka[a0 + t];
      si[t] = ia[a0 + t];
    } else {
      sk[t] = kb[b0 + t - na];
      si[t] = ib[b0 + t - na];
    }
  }
  __syncthreads();
  // Each thread merges kItems consecutive outputs of this tile.
  const uint32_t dd = threadIdx.x * Ord::kItems;
  const uint32_t tot = na + nb;
  ulonglong2 ok[Ord::kItems];
  Tag ot[Ord::kItems];
  if (dd < tot) {
    uint32_t x = merge_split(ord, sk, si, na, sk + na, si + na, nb, dd);
    uint32_t y = dd - x;
#pragma unroll
    for (int o = 0; o < Ord::kItems; ++o) {
      if (dd + o >= tot) break;
      bool take_a;
      if (x >= na) take_a = false;
      else if (y >= nb) take_a = true;
      else take_a = !ord.less(sk[na + y], si[na + y], sk[x], si[x]);
      if (take_a) {
        ok[o] = sk[x];
        ot[o] = si[x];
        ++x;
      } else {
        ok[o] = sk[na + y];
        ot[o] = si[na + y];
        ++y;
      }
    }
  }
  __syncthreads();  // every thread is done reading the inputs
  if (dd < tot) {
#pragma unroll
    for (int o = 0; o < Ord::kItems; ++o) {
      if (dd + o >= tot) break;
      sk[dd + o] = ok[o];
      si[dd + o] = ot[o];
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < tot; t += kMThreads) {
    kout[out0 + t] = sk[t];
    iout[out0 + t] = si[t];
  }
}

// seg_classes (nullable): the segmented form; passes run while the run width
// is below max_width (the largest segment), and every segment ends in the
// buffer of the parity of its own pass count.
template <class Ord>
cudaError_t run_merge_sort(const Ord& ord, ulonglong2* k0, ulonglong2* k1,
                           typename Ord::Tag* t0, typename Ord::Tag* t1,
                           const unsigned int* n_dev, size_t max_n, cudaStream_t s,
                           bool* result_in_1, const unsigned int* skip,
                           const uint32_t* seg_classes = nullptr, size_t max_width = 0) {
  constexpr size_t kTile = size_t(kMThreads) * Ord::kItems;
  const unsigned tiles = unsigned((max_n + kTile - 1) / kTile);
  msort_tiles<Ord><<<tiles, kMThreads, 0, s>>>(ord, n_dev, uint32_t(max_n), k0, t0, skip);
  count_launch();
  bool in1 = false;
  const size_t limit = seg_classes ? max_width : max_n;
  for (size_t width = kTile; width < limit; width *= 2) {
    msort_merge<Ord><<<tiles, kMThreads, 0, s>>>(ord, in1 ? k1 : k0, in1 ? t1 : t0,
                                                 in1 ? k0 : k1, in1 ? t0 : t1, n_dev,
                                                 uint32_t(max_n), uint32_t(width), skip,
                                                 seg_classes);
    count_launch();
    in1 = !in1;
  }
  *result_in_1 = in1;
  return cudaGetLastError();
}

// Run fix-up after the key-only sort of rows longer than the cached key.
// A warp takes 32 sorted positions; for every run of equal keys that starts
// there (runs end where the key changes, so they are contiguous), it stages
// the run's rows in shared memory (stride w + 1 words, so that lanes reading
// the same word of different rows hit different banks), gives every row its
// rank among the run's rows by full comparison (rows are distinct, so the
// ranks are a permutation), and writes the row numbers back in that order.
// A run longer than the warp's share of shared memory holds clears *flag,
// which makes the full-row comparison sort run afterwards.
constexpr int kFixWarps = 8;
constexpr int kFixWords = 512;   // shared-memory words per warp
constexpr int kFixMaxRun = 64;   // at most two rows per lane

__device__ __forceinline__ bool same_key(const ulonglong2& a, const ulonglong2& b) {
  return a.x == b.x && a.y == b.y;
}

constexpr int kLongMax = 2048;  // longest run msort_fix_long sorts (rows <= 256 bits)

__global__ void __launch_bounds__(kFixWarps * 32)
    msort_fix_runs(const ulonglong2* __restrict__ keys, uint32_t* idx,
                   const uint64_t* __restrict__ rows, int w, const unsigned int* n_dev,
                   uint32_t max_n, unsigned int* flag, const unsigned int* skip,
                   uint2* __restrict__ long_runs, unsigned int* long_count) {
  extern __shared__ uint64_t fix_sm[];
  __shared__ int8_t hd_all[kFixWarps][kFixMaxRun];
  if (skip && *skip) return;
  const uint32_t n = min(*n_dev, max_n);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint64_t* sr = fix_sm + size_t(wid) * kFixWords;
  int8_t* hd_sm = hd_all[wid];
  const int stride = w + 1;
  const uint32_t max_run = uint32_t(min(kFixMaxRun, kFixWords / stride));
  const uint32_t chunks = (n + 31) / 32;
  for (uint32_t c = blockIdx.x * kFixWarps + wid; c < chunks; c += gridDim.x * kFixWarps) {
    const uint32_t t = c * 32 + lane;
    bool start = false;
    if (t < n) {
      const ulonglong2 k = keys[t];
      start = t + 1 < n && same_key(keys[t + 1], k) && !(t > 0 && same_key(keys[t - 1], k));
    }
    uint32_t starts = __ballot_sync(0xffffffffu, start);
    while (starts) {
      const uint32_t s0 = c * 32 + uint32_t(__ffs(starts) - 1);
      starts &= starts - 1;
      const ulonglong2 k0 = keys[s0];
      // Run = [s0, s0 + m). The scan stops once the run is too long for the
      // path that would take it: past max_run without the long-run list,
      // past kLongMax with it (whose block then needs the whole length).
      const uint32_t scan_limit = long_runs && w <= 4 ? uint32_t(kLongMax) : max_run;
      uint32_t m = 1;
      for (uint32_t base = s0 + 1;; base += 32) {
        const uint32_t p = base + lane;
        const uint32_t eq = __ballot_sync(0xffffffffu, p < n && same_key(keys[p], k0));
        const uint32_t lead = eq == 0xffffffffu ? 32u : uint32_t(__ffs(~eq) - 1);
        m += lead;
        if (lead < 32 || m > scan_limit) break;
      }
      if (m > max_run) {
        if (lane == 0) {
          // Rows of at most 256 bits: one block sorts the run by its low key
          // (msort_fix_long); longer rows or runs: the full-row pass.
          if (long_runs && w <= 4 && m <= uint32_t(kLongMax)) {
            const unsigned int k = atomicAdd(long_count, 1u);
            long_runs[k] = make_uint2(s0, m);
          } else {
            *flag = 0u;
          }
        }
        continue;
      }
      uint32_t mine[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t a = uint32_t(lane) + 32u * j;
        mine[j] = a < m ? idx[s0 + a] : 0u;
      }
      // Stage the rows: element e = base + lane = (row a, word q), advanced
      // by 32 elements per step without a division; row numbers come from
      // the lanes that loaded them (a uniform loop, so every lane shuffles).
      const uint32_t elems = m * uint32_t(w);
      uint32_t a = uint32_t(lane) / uint32_t(w), q = uint32_t(lane) - a * uint32_t(w);
      const uint32_t da = 32u / uint32_t(w), dq = 32u - da * uint32_t(w);
#pragma unroll 4
      for (uint32_t base = 0; base < elems; base += 32) {
        const bool live = base + uint32_t(lane) < elems;
        const uint32_t r0 = __shfl_sync(0xffffffffu, mine[0], int(a & 31u));
        const uint32_t r1 = __shfl_sync(0xffffffffu, mine[1], int(a & 31u));
        if (live) sr[a * stride + q] = rows[uint64_t(a < 32u ? r0 : r1) * w + q];
        a += da;
        q += dq;
        if (q >= uint32_t(w)) {
          q -= uint32_t(w);
          ++a;
        }
      }
      __syncwarp();
      // Each row's highest word that differs from the run's first row (the
      // pivot; -1 for the pivot). Two rows whose highest words differ are
      // ordered by the higher one alone (there the other row agrees with the
      // pivot); rows with the same highest word compare that word and, only
      // when it is equal too, the words below it.
      int hd[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t a = uint32_t(lane) + 32u * j;
        int q = -1;
        if (a < m && a > 0) {
          q = w - 1;
          while (q >= 0 && sr[a * stride + q] == sr[q]) --q;
        }
        hd[j] = q;
        if (a < m) hd_sm[a] = int8_t(q);
      }
      __syncwarp();
      uint32_t rank[2] = {0u, 0u};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t a = uint32_t(lane) + 32u * j;
        if (a < m) {
          const uint64_t* ra = sr + a * stride;
          const int da = hd[j];
          for (uint32_t b = 0; b < m; ++b) {
            if (b == a) continue;
            const uint64_t* rb = sr + b * stride;
            const int db = hd_sm[b];
            bool lt;
            if (db > da) {
              lt = rb[db] < sr[db];
            } else if (da > db) {
              lt = ra[da] > sr[da];
            } else if (rb[db] != ra[db]) {
              lt = rb[db] < ra[db];
            } else {
              lt = false;
              for (int q = db - 1; q >= 0; --q)
                if (rb[q] != ra[q]) {
                  lt = rb[q] < ra[q];
                  break;
                }
            }
            rank[j] += lt ? 1u : 0u;
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t a = uint32_t(lane) + 32u * j;
        if (a < m) idx[s0 + rank[j]] = mine[j];
      }
      __syncwarp();
    }
  }
}

// Long runs of rows of at most 256 bits (listed by msort_fix_runs): the rows
// of a run agree on their top 128 bits, so the remaining l - 128 <= 128 bits
// (the low key) order them exactly. One block per run: (low key, row) pairs
// in shared memory, padded to a power of two with keys above every real one,
// sorted by a bitonic network, row numbers written back in order.
constexpr int kLongThreads = 256;

__device__ __forceinline__ ulonglong2 low_key(const uint64_t* row, int ell) {
  const int L = ell - 128;  // 1 .. 128 bits below the top 128
  const uint64_t lo = L >= 64 ? row[0] : (row[0] & ((1ull << L) - 1));
  const uint64_t hi = L <= 64 ? 0ull : (L - 64 >= 64 ? row[1] : (row[1] & ((1ull << (L - 64)) - 1)));
  return make_ulonglong2(hi, lo);
}

// (key, row) order. A run's rows have distinct low keys, but at l = 256 a
// real key can equal the padding key (all ones): the padding's row number
// 0xffffffff keeps it after every real row.
__device__ __forceinline__ bool key_less(const ulonglong2& a, uint32_t ra, const ulonglong2& b,
                                         uint32_t rb) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  return ra < rb;
}

__global__ void __launch_bounds__(kLongThreads)
    msort_fix_long(const uint2* __restrict__ long_runs, const unsigned int* long_count,
                   uint32_t* idx, const uint64_t* __restrict__ rows, int w, int ell,
                   const unsigned int* skip) {
  __shared__ ulonglong2 sk[kLongMax];
  __shared__ uint32_t sr[kLongMax];
  if (skip && *skip) return;
  const unsigned int count = *long_count;
  for (unsigned int k = blockIdx.x; k < count; k += gridDim.x) {
    const uint2 run = long_runs[k];
    const uint32_t s0 = run.x, m = run.y;
    uint32_t p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (uint32_t t = threadIdx.x; t < p2; t += kLongThreads) {
      if (t < m) {
        const uint32_t r = idx[s0 + t];
        sr[t] = r;
        sk[t] = low_key(rows + uint64_t(r) * w, ell);
      } else {
        sr[t] = 0xffffffffu;
        sk[t] = make_ulonglong2(~0ull, ~0ull);
      }
    }
    __syncthreads();
    for (uint32_t size = 2; size <= p2; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t t = threadIdx.x; t < p2; t += kLongThreads) {
          const uint32_t o = t ^ stride;
          if (o > t) {
            const bool up = (t & size) == 0;
            if (key_less(sk[o], sr[o], sk[t], sr[t]) == up) {
              const ulonglong2 tk = sk[t];
              sk[t] = sk[o];
              sk[o] = tk;
              const uint32_t tr = sr[t];
              sr[t] = sr[o];
              sr[o] = tr;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t t = threadIdx.x; t < m; t += kLongThreads) idx[s0 + t] = sr[t];
    __syncthreads();
  }
}

// ------------------------------ batch sort ---------------------------------
//
// Every scene's distinct vectors are sorted by one merge sort, each scene in
// a segment of its own: scene s with u_s vectors gets P_s = max(1024,
// 2^ceil(log2 u_s)) positions (the rest padding items that sort last), and
// the segments are laid out largest first, so each one starts at a multiple
// of its size. A merge pass of run width w then only has work in segments
// larger than w: blocks over smaller (already sorted) segments return, and
// scene s is sorted after log2(P_s / 1024) passes, its result left in the
// buffer of that parity. The work is sum_s P_s log2(P_s / 1024) items instead
// of (sum_s u_s) log2(sum_s u_s / 1024), and the pass count follows the
// largest scene.

struct BatchSortWs {
  uint32_t* off;        // [n] segment start of each scene
  uint32_t* cnt;        // [n] its vectors
  uint32_t* order;      // [n] scenes by segment start
  uint32_t* starts;     // [n + 1] segment starts in that order; starts[n] = total
  uint32_t* classes;    // [2 * kSegClasses]: first and end position of the segments of size 2^e
  unsigned int* total;  // padded item count
  ulonglong2* k0;
  ulonglong2* k1;
  uint2* t0;
  uint2* t1;
  size_t bytes;
};

__device__ __forceinline__ uint32_t seg_exp(uint32_t u) {
  // log2 of max(1024, the next power of two >= u); 0 for an empty scene
  return u == 0 ? 0u : min(31u, max(10u, 32u - __clz(u - 1u)));
}

__global__ void __launch_bounds__(1024)
    bsort_layout(const BatchSortScene* __restrict__ sc, int n, BatchSortWs w) {
  __shared__ unsigned int count[kSegClasses];
  __shared__ unsigned int base[kSegClasses];
  __shared__ unsigned int first[kSegClasses];
  __shared__ unsigned int fill[kSegClasses];
  if (threadIdx.x < kSegClasses) {
    count[threadIdx.x] = 0;
    fill[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t u = sc[i].ctr->overflow ? 0u : min(sc[i].ctr->n_unique, sc[i].ucap);
    w.cnt[i] = u;
    atomicAdd(&count[seg_exp(u)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t pos = 0;
    unsigned int k = 0;
    for (int e = kSegClasses - 1; e >= 10; --e) {  // largest segments first
      base[e] = unsigned(pos);
      first[e] = k;
      pos += uint64_t(count[e]) << e;
      k += count[e];
      w.classes[2 * e] = base[e];
      w.classes[2 * e + 1] = unsigned(pos);
    }
    first[0] = k;  // empty scenes last (no positions)
    for (int e = 0; e < 10; ++e) w.classes[2 * e] = w.classes[2 * e + 1] = unsigned(pos);
    w.starts[n] = unsigned(pos);
    *w.total = unsigned(pos);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t e = seg_exp(w.cnt[i]);
    const unsigned int r = atomicAdd(&fill[e], 1u);
    const uint32_t o = e == 0 ? w.starts[n] : base[e] + uint32_t(uint64_t(r) << e);
    w.off[i] = o;
    w.order[first[e] + r] = uint32_t(i);
    w.starts[first[e] + r] = o;
  }
}

__device__ __forceinline__ int seg_index_at(const uint32_t* starts, int n, uint32_t g) {
  int lo = 0, hi = n - 1;  // last k with starts[k] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void bsort_items(const BatchSortScene* __restrict__ sc, int n, BatchSortWs w) {
  const uint32_t m = *w.total;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < m; g += gridDim.x * blockDim.x) {
    const int s = int(w.order[seg_index_at(w.starts, n, g)]);
    const uint32_t i = g - w.off[s];
    if (i < w.cnt[s]) {
      const BatchSortScene& c = sc[s];
      w.k0[g] = c.ell <= 64 ? make_ulonglong2(c.ulist[i], 0ull)
                            : top128(c.keys64 + uint64_t(c.idx[i]) * c.w, c.ell);
      w.t0[g] = make_uint2(uint32_t(s), i);
    } else {
      // Padding (sorts after every real item), in both buffers: the merge
      // passes skip the blocks that would only copy it.
      w.k0[g] = make_ulonglong2(~0ull, ~0ull);
      w.t0[g] = make_uint2(kPad, kPad);
      w.k1[g] = make_ulonglong2(~0ull, ~0ull);
      w.t1[g] = make_uint2(kPad, kPad);
    }
  }
}

__global__ void bsort_scatter(const BatchSortScene* __restrict__ sc, int n, BatchSortWs w) {
  const uint32_t m = *w.total;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < m; g += gridDim.x * blockDim.x) {
    const int s = int(w.order[seg_index_at(w.starts, n, g)]);
    const uint32_t rank = g - w.off[s];
    const uint32_t cnt = w.cnt[s];
    if (rank >= cnt) continue;
    // The segment's result is in the buffer of the parity of its pass count.
    const uint2 tg = (seg_exp(cnt) - 10u) & 1u ? w.t1[g] : w.t0[g];
    const BatchSortScene& c = sc[s];
    const bool user = c.user_cells && int64_t(cnt) <= c.user_cap;
    if (c.ell <= 64) {
      const uint64_t v = c.ulist[tg.y];
      c.cells[rank] = v;
      if (user) c.user_cells[rank] = v;
      if (c.t.keys) {
        if (v == kEmpty) {
          c.ctr->ones_rank = rank;
        } else {
          const int64_t slot = small_find_slot(c.t.keys, c.t.mask, c.t.shift, v);
          if (slot >= 0) c.t.vals[slot] = rank;
          else atomicOr(&c.ctr->error, 1u);
        }
      }
    } else {
      const uint64_t* row = c.keys64 + uint64_t(c.idx[tg.y]) * c.w;
      for (int q = 0; q < c.w; ++q) {
        c.cells[uint64_t(rank) * c.w + q] = row[q];
        if (user) c.user_cells[uint64_t(rank) * c.w + q] = row[q];
      }
    }
  }
}

BatchSortWs carve_bsort(void* base, size_t cap, int n) {
  BatchSortWs w{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = (o + 255) & ~size_t(255);
    void* p = base ? static_cast<char*>(base) + o : nullptr;
    o += bytes;
    return p;
  };
  const size_t c = cap > 0 ? cap : 1;
  const size_t sn = size_t(n) + 1;
  w.off = static_cast<uint32_t*>(take(sn * 4));
  w.cnt = static_cast<uint32_t*>(take(sn * 4));
  w.order = static_cast<uint32_t*>(take(sn * 4));
  w.starts = static_cast<uint32_t*>(take(sn * 4));
  w.classes = static_cast<uint32_t*>(take(2 * kSegClasses * 4));
  w.total = static_cast<unsigned int*>(take(4));
  w.k0 = static_cast<ulonglong2*>(take(c * 16));
  w.k1 = static_cast<ulonglong2*>(take(c * 16));
  w.t0 = static_cast<uint2*>(take(c * 8));
  w.t1 = static_cast<uint2*>(take(c * 8));
  w.bytes = o + 256;
  return w;
}

// ---------------------------------------------------------------------------
// Bucket sort of rows of l > 64 bits (the distinct vectors of step 2, §3.2,
// ordered as integers with bit l-1 the most significant). The top B bits of a
// row pick one of 2^B buckets (B from the capacity: about kBucketAvg rows a
// bucket when the distinct rows fill it). A histogram, one scan and one
// scatter put every (top 128 bits, row number) pair in its bucket's range;
// one block per bucket then orders the range in shared memory with a bitonic
// network on the top 128 bits, whole rows breaking ties. The plan kernel
// checks every bucket against kBucketMax before anything is written: when one
// is larger (top bits far from uniform, as the signs of a few planes are),
// the merge sort runs instead, so such inputs cost time, never correctness.
// ---------------------------------------------------------------------------
constexpr int kBucketAvg = 512;
constexpr int kBucketMax = 2048;
constexpr int kBucketThreads = 256;
constexpr int kBucketMaxBits = 14;

struct BucketWs {
  unsigned int* ok;       // 1: every bucket fits, the bucket sort runs
  unsigned int* fb_skip;  // nonzero: the merge sort's kernels return at once
  uint32_t* count;        // [2^bits]
  uint32_t* start;        // [2^bits + 1]
  uint32_t* cursor;       // [2^bits]
  int bits;
};

size_t bucket_ws_bytes(int bits) { return 16 + (3 * (size_t(1) << bits) + 1) * sizeof(uint32_t); }

BucketWs carve_bucket(void* scratch, int bits) {
  char* p = static_cast<char*>(scratch);
  const size_t nb = size_t(1) << bits;
  BucketWs b;
  b.ok = reinterpret_cast<unsigned int*>(p);
  b.fb_skip = b.ok + 1;
  b.count = reinterpret_cast<uint32_t*>(p + 16);
  b.start = b.count + nb;
  b.cursor = b.start + nb + 1;
  b.bits = bits;
  return b;
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t top, int bits) {
  return bits ? uint32_t(top >> (64 - bits)) : 0u;
}

__global__ void __launch_bounds__(kBucketThreads)
    bucket_hist(const uint64_t* __restrict__ rows, int w, int ell,
                const uint32_t* __restrict__ idx_in, const unsigned int* n_dev, uint32_t max_n,
                BucketWs b, const unsigned int* skip) {
  if (skip && *skip) return;
  const uint32_t u = min(*n_dev, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t r = idx_in ? idx_in[i] : i;
    atomicAdd(&b.count[bucket_of(bits64_at(rows + uint64_t(r) * w, ell - 64), b.bits)], 1u);
  }
}

// One block: bucket starts (exclusive scan of the counts), cursors cleared,
// and the decision between the bucket sort and the merge sort.
__global__ void __launch_bounds__(1024) bucket_plan(BucketWs b, const unsigned int* skip) {
  __shared__ uint32_t part[1024];
  __shared__ int too_big;
  if (skip && *skip) {
    if (threadIdx.x == 0) {
      *b.ok = 0u;
      *b.fb_skip = 1u;
    }
    return;
  }
  if (threadIdx.x == 0) too_big = 0;
  const uint32_t nb = 1u << b.bits;
  const uint32_t per = (nb + 1023) / 1024;
  const uint32_t j0 = threadIdx.x * per;
  const uint32_t j1 = min(j0 + per, nb);
  uint32_t sum = 0;
  bool big = false;
  for (uint32_t j = j0; j < j1; ++j) {
    const uint32_t c = b.count[j];
    sum += c;
    big |= c > uint32_t(kBucketMax);
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  if (big) too_big = 1;
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t v = int(threadIdx.x) >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (uint32_t j = j0; j < j1; ++j) {
    b.start[j] = run;
    run += b.count[j];
    b.cursor[j] = 0u;
  }
  if (threadIdx.x == 1023) b.start[nb] = part[1023];
  __syncthreads();
  if (threadIdx.x == 0) {
    *b.ok = too_big ? 0u : 1u;
    *b.fb_skip = too_big ? 0u : 1u;
  }
}

__global__ void __launch_bounds__(kBucketThreads)
    bucket_scatter(const uint64_t* __restrict__ rows, int w, int ell,
                   const uint32_t* __restrict__ idx_in, const unsigned int* n_dev, uint32_t max_n,
                   BucketWs b, const ulonglong2* __restrict__ ukeys,
                   ulonglong2* __restrict__ kout, uint32_t* __restrict__ xout) {
  if (!*b.ok) return;
  const uint32_t u = min(*n_dev, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t r = idx_in ? idx_in[i] : i;
    const ulonglong2 k = ukeys ? ukeys[i] : top128(rows + uint64_t(r) * w, ell);
    const uint32_t bk = bucket_of(k.x, b.bits);
    const uint32_t pos = b.start[bk] + atomicAdd(&b.cursor[bk], 1u);
    if (pos < b.start[bk + 1]) {  // always: the counts came from the same items
      kout[pos] = k;
      xout[pos] = r;
    }
  }
}

size_t bucket_local_smem() {
  return size_t(kBucketMax) * (sizeof(ulonglong2) + sizeof(uint32_t)) + 3 * 256 * sizeof(uint32_t);
}

// (key, row number) order of the bucket sort; padding items (key all ones,
// row number kPad) come after every real item.
__device__ __forceinline__ bool bkey_less(const ulonglong2& ka, uint32_t ia, const ulonglong2& kb,
                                          uint32_t ib) {
  if (ka.x != kb.x) return ka.x < kb.x;
  if (ka.y != kb.y) return ka.y < kb.y;
  return ia < ib;
}

// One block per bucket (grid-stride over buckets), ordered by (top 128 bits,
// row number); keys go to kout and row numbers to out in that order. Rows
// longer than 128 bits that share their top 128 bits are left in row-number
// order here, as the key-only merge sort leaves them; the run fix-up orders
// them afterwards. The usual case is a counting sort on the 8 bits below the
// bucket's own bits (256 sub-buckets, a few items each when the bits are
// spread), each sub-bucket then put in order by one thread's insertion sort;
// when some sub-bucket holds more than kSubMax items, the block sorts the
// whole bucket with a bitonic network instead.
constexpr uint32_t kSubMax = 32;

__global__ void __launch_bounds__(kBucketThreads)
    bucket_local(const uint64_t* __restrict__ rows, int w, int ell, BucketWs b,
                 const ulonglong2* kin, const uint32_t* xin, ulonglong2* kout, uint32_t* out) {
  static_assert(kBucketThreads == 256, "one thread per sub-bucket");
  extern __shared__ __align__(16) unsigned char bucket_sm[];
  ulonglong2* sk = reinterpret_cast<ulonglong2*>(bucket_sm);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + kBucketMax);
  uint32_t* hist = si + kBucketMax;  // [256]
  uint32_t* off = hist + 256;        // [256]
  uint32_t* cur = off + 256;         // [256]
  __shared__ uint32_t wsum[kBucketThreads / 32];
  __shared__ int big;
  (void)rows;
  (void)w;
  (void)ell;
  if (!*b.ok) return;
  const uint32_t nb = 1u << b.bits;
  const int dshift = 56 - b.bits;  // the 8 bits below the bucket's bits
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint32_t bk = blockIdx.x; bk < nb; bk += gridDim.x) {
    const uint32_t lo = b.start[bk];
    const uint32_t cnt = min(b.start[bk + 1] - lo, uint32_t(kBucketMax));
    if (cnt <= 1) {
      if (cnt == 1 && threadIdx.x == 0) {
        const ulonglong2 k = kin[lo];
        const uint32_t r = xin[lo];
        kout[lo] = k;
        out[lo] = r;
      }
      continue;
    }
    hist[threadIdx.x] = 0u;
    cur[threadIdx.x] = 0u;
    if (threadIdx.x == 0) big = 0;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x)
      atomicAdd(&hist[uint32_t(kin[lo + t].x >> dshift) & 0xffu], 1u);
    __syncthreads();
    {
      const uint32_t v = hist[threadIdx.x];
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      if (lane == 31) wsum[wid] = incl;
      __syncthreads();
      uint32_t before = 0;
      for (int k = 0; k < wid; ++k) before += wsum[k];
      off[threadIdx.x] = before + incl - v;
      if (v > kSubMax) big = 1;
    }
    __syncthreads();
    if (!big) {
      for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
        const ulonglong2 k = kin[lo + t];
        const uint32_t d = uint32_t(k.x >> dshift) & 0xffu;
        const uint32_t pos = off[d] + atomicAdd(&cur[d], 1u);
        sk[pos] = k;
        si[pos] = xin[lo + t];
      }
      __syncthreads();
      {
        const uint32_t s0 = off[threadIdx.x], c = hist[threadIdx.x];
        for (uint32_t i = s0 + 1; i < s0 + c; ++i) {
          const ulonglong2 k = sk[i];
          const uint32_t r = si[i];
          uint32_t j = i;
          while (j > s0 && bkey_less(k, r, sk[j - 1], si[j - 1])) {
            sk[j] = sk[j - 1];
            si[j] = si[j - 1];
            --j;
          }
          sk[j] = k;
          si[j] = r;
        }
      }
      __syncthreads();
    } else {
      uint32_t p2 = 2;
      while (p2 < cnt) p2 <<= 1;
      for (uint32_t t = threadIdx.x; t < p2; t += blockDim.x) {
        if (t < cnt) {
          sk[t] = kin[lo + t];
          si[t] = xin[lo + t];
        } else {
          sk[t] = make_ulonglong2(~0ull, ~0ull);
          si[t] = kPad;
        }
      }
      __syncthreads();
      for (uint32_t size = 2; size <= p2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t t = threadIdx.x; t < p2 / 2; t += blockDim.x) {
            const uint32_t i = 2 * t - (t & (stride - 1));
            const uint32_t j = i + stride;
            const bool up = (i & size) == 0;
            if (bkey_less(sk[j], si[j], sk[i], si[i]) == up) {
              const ulonglong2 tk = sk[i];
              sk[i] = sk[j];
              sk[j] = tk;
              const uint32_t tr = si[i];
              si[i] = si[j];
              si[j] = tr;
            }
          }
          __syncthreads();
        }
      }
    }
    for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
      kout[lo + t] = sk[t];
      out[lo + t] = si[t];
    }
    __syncthreads();  // the next bucket reuses the shared arrays
  }
}

}  // namespace

size_t scan_scratch_bytes(size_t max_n) {
  return ((max_n + kSTile - 1) / kSTile + 1) * sizeof(unsigned long long);
}

size_t radix_scratch_bytes(size_t max_n) {
  const size_t tiles = (max_n + kRTile - 1) / kRTile + 1;
  size_t bytes = 256 * tiles * sizeof(uint32_t);
  bytes = (bytes + 255) & ~size_t(255);
  if (tiles > kInlineTiles) {
    bytes += 256 * tiles * sizeof(unsigned long long);
    bytes = (bytes + 255) & ~size_t(255);
    bytes += scan_scratch_bytes(256 * tiles);
  }
  return bytes;
}

int bucket_sort_bits(size_t max_n) {
  int bits = 0;
  while (bits < kBucketMaxBits && (size_t(kBucketAvg) << bits) < max_n) ++bits;
  return bits;
}

uint32_t* bucket_sort_counts(void* scratch, size_t max_n) {
  return carve_bucket(scratch, bucket_sort_bits(max_n)).count;
}

cudaError_t scan_exclusive_u32(const uint32_t* in, unsigned long long* out,
                               const unsigned int* n_dev, size_t max_n,
                               unsigned long long* total, void* scratch, cudaStream_t s) {
  return scan_impl(in, out, Count{n_dev, 1, 1, max_n}, max_n, total, scratch, s);
}

cudaError_t radix_sort_u64(uint64_t* keys0, uint64_t* keys1, uint32_t* vals0, uint32_t* vals1,
                           const unsigned int* n_dev, size_t max_n, int bits, void* scratch,
                           cudaStream_t s, bool* result_in_1) {
  const int passes = (bits + 7) / 8;
  *result_in_1 = (passes & 1) != 0;
  if (max_n == 0 || passes == 0) {
    *result_in_1 = false;
    return cudaSuccess;
  }
  const size_t tiles = (max_n + kRTile - 1) / kRTile;
  char* sp = static_cast<char*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(sp);
  size_t off = (256 * (tiles + 1) * sizeof(uint32_t) + 255) & ~size_t(255);
  unsigned long long* scanned = nullptr;
  void* scan_scratch = nullptr;
  if (tiles > kInlineTiles) {
    scanned = reinterpret_cast<unsigned long long*>(sp + off);
    off += (256 * (tiles + 1) * sizeof(unsigned long long) + 255) & ~size_t(255);
    scan_scratch = sp + off;
  }
  uint64_t* kin = keys0;
  uint64_t* kout = keys1;
  uint32_t* vin = vals0;
  uint32_t* vout = vals1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    radix_hist<<<unsigned(tiles), kRThreads, 0, s>>>(kin, n_dev, uint32_t(max_n), shift, hist);
    count_launch();
    if (scanned) {
      cudaError_t e = scan_impl(hist, scanned, Count{n_dev, 256, kRTile, max_n}, 256 * tiles,
                                nullptr, scan_scratch, s);
      if (e != cudaSuccess) return e;
    }
    if (vals0) {
      radix_scatter<true><<<unsigned(tiles), kRThreads, 0, s>>>(
          kin, kout, vin, vout, n_dev, uint32_t(max_n), shift, hist, scanned);
    } else {
      radix_scatter<false><<<unsigned(tiles), kRThreads, 0, s>>>(
          kin, kout, nullptr, nullptr, n_dev, uint32_t(max_n), shift, hist, scanned);
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  return cudaSuccess;
}

}  // namespace cg

namespace cg {

cudaError_t cluster_sort(const uint64_t* in, const uint32_t* rows, const unsigned int* n_dev,
                         size_t max_n, int ell, const ClusterSortOut& o, cudaStream_t s,
                         bool* done, bool* tried) {
  *done = false;
  if (tried) *tried = false;
  const int w = (ell + 63) / 64;
  const int top = ell - 64 * (w - 1);
  if (w == 1 && !rows && max_n > 0 && o.t.keys) {
    // Decided on the device: a count above kRankMax leaves the work (and
    // o.ctr->sorted) to the cluster sort launched next.
    const uint32_t cap = uint32_t(std::min<size_t>(max_n, kRankMax));
    const dim3 grid((cap + kRankThreads - 1) / kRankThreads, kRankSplits);
    cudaError_t e = launch_dep(rank_count, grid, dim3(kRankThreads), 0, s, in, n_dev,
                               uint32_t(max_n), o);
    if (e == cudaSuccess)
      e = launch_dep(rank_place, dim3((cap + kRankThreads - 1) / kRankThreads),
                     dim3(kRankThreads), 0, s, in, n_dev, uint32_t(max_n), o);
    count_launch(2);
    if (e != cudaSuccess) return e;
    if (max_n <= kRankMax) {
      *done = true;
      return cudaSuccess;
    }
  }
  switch (w) {
    case 1: return cluster_sort_w<1>(in, rows, n_dev, max_n, top, o, s, done, tried);
    case 2: return cluster_sort_w<2>(in, rows, n_dev, max_n, top, o, s, done, tried);
    case 3: return cluster_sort_w<3>(in, rows, n_dev, max_n, top, o, s, done, tried);
    case 4: return cluster_sort_w<4>(in, rows, n_dev, max_n, top, o, s, done, tried);
    default: return cudaSuccess;  // longer vectors: multi-launch sort
  }
}

cudaError_t merge_sort_rows(const uint64_t* rows, int w64, int ell, const uint32_t* idx_in,
                            uint64_t* k0, uint64_t* k1, uint32_t* i0, uint32_t* i1,
                            const unsigned int* n_dev, size_t max_n, cudaStream_t s,
                            uint32_t** sorted_idx, const unsigned int* skip,
                            unsigned int* flag, void* scratch, size_t scratch_bytes,
                            const ulonglong2* ukeys) {
  *sorted_idx = i0;
  if (max_n == 0) return cudaSuccess;
  if (ell <= 64) return cudaErrorInvalidValue;
  ulonglong2* kk0 = reinterpret_cast<ulonglong2*>(k0);
  ulonglong2* kk1 = reinterpret_cast<ulonglong2*>(k1);
  bool in1 = false;
  const int bits = bucket_sort_bits(max_n);
  const unsigned int* ext_skip = skip;
  if (max_n < (1ull << 32) && scratch && bucket_ws_bytes(bits) <= scratch_bytes) {
    // The bucket sort first; the (key-only) merge sort below runs only when a
    // bucket is too large (b.fb_skip). Its keys and row numbers go to the
    // buffers the merge sort would end in, the row numbers through a buffer
    // other than idx_in, which the merge sort may still need.
    const BucketWs b = carve_bucket(scratch, bits);
    bool par = false;
    for (size_t width = size_t(kMThreads) * RowOrder::kItems; width < max_n; width *= 2)
      par = !par;
    uint32_t* out = par ? i1 : i0;
    uint32_t* x = out != idx_in ? out : (out == i0 ? i1 : i0);
    cudaError_t e;
    const int g = int(std::max<size_t>(
        1, std::min<size_t>((max_n + kBucketThreads - 1) / kBucketThreads,
                            size_t(sm_count()) * 8)));
    if (!ukeys) {  // counts from the rows (else the insert made them)
      e = cudaMemsetAsync(b.count, 0, (size_t(1) << bits) * sizeof(uint32_t), s);
      if (e != cudaSuccess) return e;
      bucket_hist<<<g, kBucketThreads, 0, s>>>(rows, w64, ell, idx_in, n_dev, uint32_t(max_n), b,
                                               skip);
      count_launch();
    }
    bucket_plan<<<1, 1024, 0, s>>>(b, skip);
    bucket_scatter<<<g, kBucketThreads, 0, s>>>(rows, w64, ell, idx_in, n_dev, uint32_t(max_n),
                                                b, ukeys, kk0, x);
    const size_t smem = bucket_local_smem();
    if ((e = ensure_smem_limit(reinterpret_cast<const void*>(bucket_local), smem)) != cudaSuccess)
      return e;
    int per_sm = 0;
    if ((e = blocks_per_sm(reinterpret_cast<const void*>(bucket_local), kBucketThreads, smem,
                           &per_sm)) != cudaSuccess)
      return e;
    const int gl = int(std::min<size_t>(size_t(1) << bits,
                                        size_t(sm_count()) * size_t(per_sm > 0 ? per_sm : 1)));
    bucket_local<<<gl, kBucketThreads, smem, s>>>(rows, w64, ell, b, kk0, x, par ? kk1 : kk0,
                                                  out);
    count_launch(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    skip = b.fb_skip;
  }
  if (ell <= 128 || !flag) {
    const RowOrder ord{rows, w64, ell, ell <= 128, idx_in};
    cudaError_t e = run_merge_sort(ord, kk0, kk1, i0, i1, n_dev, max_n, s, &in1, skip);
    *sorted_idx = in1 ? i1 : i0;
    return e;
  }
  // Rows longer than the cached key. Sorting on the key alone (ties in
  // row-number order) reads no row; each run of rows sharing their top 128
  // bits is then put in row order by one warp. Only when a run is too long
  // for that does the full-row comparison sort run (its kernels return at
  // once while *flag is nonzero). Both sorts make the same number of passes,
  // so their results land in the same buffer.
  cudaError_t e = cudaMemsetAsync(flag, 1, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const RowOrder by_key{rows, w64, ell, true, idx_in};
  e = run_merge_sort(by_key, kk0, kk1, i0, i1, n_dev, max_n, s, &in1, skip);
  if (e != cudaSuccess) return e;
  uint32_t* out = in1 ? i1 : i0;
  const size_t smem = size_t(kFixWarps) * kFixWords * sizeof(uint64_t);
  if ((e = ensure_smem_limit(reinterpret_cast<const void*>(msort_fix_runs), smem)) !=
      cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = blocks_per_sm(reinterpret_cast<const void*>(msort_fix_runs), kFixWarps * 32, smem,
                         &per_sm)) != cudaSuccess)
    return e;
  const size_t chunks = (max_n + 31) / 32;
  const int g = int(std::max<size_t>(
      1, std::min<size_t>((chunks + kFixWarps - 1) / kFixWarps,
                          size_t(sm_count()) * size_t(per_sm > 0 ? per_sm : 1))));
  // The list of long runs lives in the key buffer the sort did not end in:
  // its first 16 bytes hold the count.
  ulonglong2* spare = in1 ? kk0 : kk1;
  unsigned int* long_count = reinterpret_cast<unsigned int*>(spare);
  uint2* long_runs = reinterpret_cast<uint2*>(spare + 1);
  const bool use_long = w64 <= 4;
  if (use_long && (e = cudaMemsetAsync(long_count, 0, sizeof(ulonglong2), s)) != cudaSuccess)
    return e;
  msort_fix_runs<<<g, kFixWarps * 32, smem, s>>>(in1 ? kk1 : kk0, out, rows, w64, n_dev,
                                                 uint32_t(max_n), flag, ext_skip,
                                                 use_long ? long_runs : nullptr, long_count);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (use_long) {
    const unsigned lg = unsigned(std::max<size_t>(1, std::min<size_t>(
                                                         (max_n + kLongMax - 1) / kLongMax,
                                                         size_t(sm_count()) * 2)));
    msort_fix_long<<<lg, kLongThreads, 0, s>>>(long_runs, long_count, out, rows, w64, ell,
                                               ext_skip);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const RowOrder full{rows, w64, ell, false, out};
  bool in1b = false;
  e = run_merge_sort(full, kk0, kk1, i0, i1, n_dev, max_n, s, &in1b, flag);
  if (in1b != in1) return cudaErrorUnknown;  // the pass counts differ: cannot happen
  *sorted_idx = out;
  return e;
}

size_t batch_sort_seg_size(size_t ucap) {
  size_t p = 1024;
  while (p < ucap) p <<= 1;
  return p;
}

size_t batch_sort_bytes(size_t total_cap, int n_scenes) {
  return carve_bsort(nullptr, total_cap, n_scenes).bytes;
}

cudaError_t batch_sort(const BatchSortScene* scenes, int n_scenes, size_t total_cap,
                       size_t max_seg, void* scratch, cudaStream_t s) {
  if (n_scenes <= 0) return cudaSuccess;
  BatchSortWs w = carve_bsort(scratch, total_cap, n_scenes);
  bsort_layout<<<1, 1024, 0, s>>>(scenes, n_scenes, w);
  count_launch();
  const size_t cap = total_cap > 0 ? total_cap : 1;
  const int g = int(std::min<size_t>((cap + 255) / 256, size_t(sm_count()) * 8));
  bsort_items<<<g, 256, 0, s>>>(scenes, n_scenes, w);
  count_launch();
  // The padding items are in place, so the tile sort reads w.k0/w.t0 as they are.
  const BatchOrder ord{scenes, w.k0, w.t0};
  bool in1 = false;
  cudaError_t e = run_merge_sort(ord, w.k0, w.k1, w.t0, w.t1, w.total, cap, s, &in1, nullptr,
                                 w.classes, max_seg);
  if (e != cudaSuccess) return e;
  bsort_scatter<<<g, 256, 0, s>>>(scenes, n_scenes, w);
  count_launch();
  return cudaGetLastError();
}

// --------------------------- segmented key sort ----------------------------
//
// The lookup strategies that bucket cells by a key (PIVOT: distances to the
// pivots; HALVES: the low part) sort each scene's (key, cell) pairs. In a
// batch, hundreds of such small sorts are each a chain of latency-bound
// launches. Here the pairs of every scene are gathered into one array with
// the scene's number above the key bits, sorted by one LSD radix sort (so
// every scene's items end up contiguous, in key order, ties in input order),
// and scattered back into each scene's arrays.
namespace {

struct SegSortWs {
  unsigned int* off;  // [S + 1] item offsets; off[S] is the total
  uint64_t* k0;
  uint64_t* k1;
  uint32_t* v0;
  uint32_t* v1;
  void* radix;
  size_t bytes;
};

SegSortWs carve_segsort(void* base, size_t total_cap, int n_scenes) {
  SegSortWs w{};
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* r = p ? p + off : nullptr;
    off = (off + bytes + 255) & ~size_t(255);
    return r;
  };
  const size_t cap = total_cap > 0 ? total_cap : 1;
  w.off = reinterpret_cast<unsigned int*>(take((size_t(n_scenes) + 1) * sizeof(unsigned int)));
  w.k0 = reinterpret_cast<uint64_t*>(take(cap * sizeof(uint64_t)));
  w.k1 = reinterpret_cast<uint64_t*>(take(cap * sizeof(uint64_t)));
  w.v0 = reinterpret_cast<uint32_t*>(take(cap * sizeof(uint32_t)));
  w.v1 = reinterpret_cast<uint32_t*>(take(cap * sizeof(uint32_t)));
  w.radix = take(radix_scratch_bytes(cap));
  w.bytes = off;
  return w;
}

__global__ void __launch_bounds__(1024)
    segsort_offsets(const SegSortScene* __restrict__ sc, int n_scenes, unsigned int* off) {
  unsigned long long carry = 0;
  for (int base = 0; base < n_scenes; base += 1024) {
    const int i = base + int(threadIdx.x);
    const unsigned long long c =
        i < n_scenes && !sc[i].ctr->overflow ? min(sc[i].ctr->n_unique, sc[i].cap) : 0u;
    unsigned long long tot = 0;
    const unsigned long long ex = block_excl(c, &tot);
    if (i < n_scenes) off[i] = unsigned(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) off[n_scenes] = unsigned(carry);
}

// Scene of item g: the last s with off[s] <= g.
__device__ __forceinline__ int segsort_scene(const unsigned int* off, int n_scenes, uint32_t g) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void segsort_gather(const SegSortScene* __restrict__ sc, int n_scenes,
                               const unsigned int* __restrict__ off, int key_bits, uint64_t* k,
                               uint32_t* v) {
  const uint32_t total = off[n_scenes];
  const uint64_t mask = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1);
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += gridDim.x * blockDim.x) {
    const int s = segsort_scene(off, n_scenes, g);
    const uint32_t j = g - off[s];
    k[g] = (uint64_t(s) << key_bits) | (sc[s].keys[j] & mask);
    v[g] = sc[s].vals[j];
  }
}

__global__ void segsort_scatter(const SegSortScene* __restrict__ sc,
                                const unsigned int* __restrict__ off, int n_scenes, int key_bits,
                                const uint64_t* __restrict__ k, const uint32_t* __restrict__ v) {
  const uint32_t total = off[n_scenes];
  const uint64_t mask = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1);
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += gridDim.x * blockDim.x) {
    const uint64_t key = k[g];
    const uint64_t s = key_bits >= 64 ? 0 : key >> key_bits;
    if (s >= uint64_t(n_scenes)) continue;  // cannot happen: every item carries its scene
    const uint32_t j = g - off[s];  // scene s occupies [off[s], off[s + 1]) once sorted
    if (j >= sc[s].cap) continue;
    sc[s].keys[j] = key & mask;
    sc[s].vals[j] = v[g];
  }
}

}  // namespace

size_t seg_sort_bytes(size_t total_cap, int n_scenes) {
  return carve_segsort(nullptr, total_cap, n_scenes).bytes;
}

cudaError_t seg_sort(const SegSortScene* scenes, int n_scenes, size_t total_cap, int key_bits,
                     void* scratch, cudaStream_t s) {
  if (n_scenes <= 0 || total_cap == 0) return cudaSuccess;
  int scene_bits = 0;
  while ((1 << scene_bits) < n_scenes) ++scene_bits;
  if (key_bits < 1 || key_bits + scene_bits > 64) return cudaErrorInvalidValue;
  SegSortWs w = carve_segsort(scratch, total_cap, n_scenes);
  segsort_offsets<<<1, 1024, 0, s>>>(scenes, n_scenes, w.off);
  const int g = int(std::min<size_t>((total_cap + 255) / 256, size_t(sm_count()) * 8));
  segsort_gather<<<g, 256, 0, s>>>(scenes, n_scenes, w.off, key_bits, w.k0, w.v0);
  count_launch(2);
  bool in1 = false;
  cudaError_t e = radix_sort_u64(w.k0, w.k1, w.v0, w.v1, &w.off[n_scenes], total_cap,
                                 key_bits + scene_bits, w.radix, s, &in1);
  if (e != cudaSuccess) return e;
  segsort_scatter<<<g, 256, 0, s>>>(scenes, w.off, n_scenes, key_bits, in1 ? w.k1 : w.k0,
                                    in1 ? w.v1 : w.v0);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cg
