// Breadth-first search on the cell graph G_X. The paper's motivation (§1,
// §6): a path in the cell graph corresponds to an approximate solution of the
// motion-planning problem, and traversing large graphs on the GPU is named as
// the next problem. This file turns the edge list of cg_neighbors_h1 /
// cg_build (pairs i < j) into a compressed adjacency of both directions and
// searches it level by level from one cell.
//
//   adjacency: degree count (atomics over both endpoints of every edge), an
//              exclusive scan of the degrees, then a fill pass in which every
//              endpoint claims a slot of its row with an atomic cursor (rows
//              are unordered; distances do not depend on it);
//   levels:    level d reads the frontier f_in (cells at distance d) and, for
//              every neighbour v still at -1, claims it with a compare-and-
//              swap of dist[v] from -1 to d + 1; the winner records its parent
//              and appends v to f_out. Frontier sizes live in three rotating
//              device counters (level d reads cnt[d % 3], appends to
//              cnt[(d + 1) % 3] and clears cnt[(d + 2) % 3], which only level
//              d - 1 used), so levels are enqueued back to back without a host
//              round trip; a level whose frontier is empty returns at once
//              (the host looks at the frontier once per group of levels).
//
// Distances are unique; parents are one valid BFS tree among several (any
// neighbour one level closer). Work: O(U + E) per search.
//
// Single launch: the same levels in one cooperative launch (one block per
// SM, all co-resident), separated by a grid barrier of this file (an arrival
// counter and a generation word; the last block to arrive resets the counter
// and bumps the generation). Every barrier wait is bounded: when it runs out
// the block sets an error bit and leaves, and every other block leaves at its
// next barrier (which then cannot complete and runs out too), so the launch
// always ends. A level costs a barrier instead of a kernel launch.
#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;

int grid_for(size_t items) {
  const size_t want = (items + kThreads - 1) / kThreads;
  const size_t cap = size_t(sm_count()) * 8;
  size_t g = want < cap ? want : cap;
  return int(g < 1 ? 1 : g);
}

// dist = -1 except dist[source] = 0, parent = -1; counters of the first level.
__global__ void bfs_init(int32_t* __restrict__ dist, int32_t* __restrict__ parent, uint32_t n,
                         uint32_t source, uint32_t* __restrict__ f0, BfsCounters* c) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    dist[v] = v == source ? 0 : -1;
    if (parent) parent[v] = -1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    f0[0] = source;
    c->frontier[0] = 1;
    c->frontier[1] = 0;
    c->frontier[2] = 0;
    c->error = 0;
    c->n = n;
    c->reached = 0;  // each level adds its frontier's size
    c->depth = 0;
  }
}

__global__ void bfs_degree(const uint32_t* __restrict__ edges, uint64_t n_edges, uint32_t n,
                           uint32_t* __restrict__ deg, BfsCounters* c) {
  for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n_edges;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t i = edges[2 * e], j = edges[2 * e + 1];
    if (i >= n || j >= n || i == j) {
      atomicOr(&c->error, 1u);
      continue;
    }
    atomicAdd(&deg[i], 1u);
    atomicAdd(&deg[j], 1u);
  }
}

__global__ void bfs_fill(const uint32_t* __restrict__ edges, uint64_t n_edges, uint32_t n,
                         const unsigned long long* __restrict__ off, uint32_t* __restrict__ cur,
                         uint32_t* __restrict__ adj) {
  for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n_edges;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t i = edges[2 * e], j = edges[2 * e + 1];
    if (i >= n || j >= n || i == j) continue;
    adj[off[i] + atomicAdd(&cur[i], 1u)] = j;
    adj[off[j] + atomicAdd(&cur[j], 1u)] = i;
  }
}

// One level: the frontier cells f_in[0, cnt) at distance d claim their
// unvisited neighbours. Eight lanes take one frontier cell (lanes over its
// neighbours, so a cell's few neighbours are looked at in parallel, not one
// after the other); a warp appends the cells it claimed with one atomic.
// Loops are warp-uniform (the ballots need every lane).
constexpr int kLanesPerCell = 8;

__device__ __forceinline__ void expand_level(int d, uint32_t cnt,
                                             const unsigned long long* __restrict__ off,
                                             const uint32_t* __restrict__ deg,
                                             const uint32_t* __restrict__ adj, int32_t* dist,
                                             int32_t* __restrict__ parent,
                                             const uint32_t* __restrict__ f_in,
                                             uint32_t* __restrict__ f_out, unsigned int* out_cnt) {
  constexpr uint32_t kCellsPerWarp = 32 / kLanesPerCell;
  const int lane = threadIdx.x & 31;
  const int sub = lane % kLanesPerCell;
  const uint64_t warp0 = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
  const uint64_t warps = uint64_t(gridDim.x) * blockDim.x / 32;
  for (uint64_t k0 = warp0 * kCellsPerWarp; k0 < cnt; k0 += warps * kCellsPerWarp) {
    const uint64_t k = k0 + uint64_t(lane / kLanesPerCell);
    const bool live = k < cnt;
    const uint32_t u = live ? f_in[k] : 0u;
    const unsigned long long p0 = live ? off[u] : 0ull;
    const uint32_t m = live ? deg[u] : 0u;
    const uint32_t mmax = __reduce_max_sync(0xffffffffu, m);
    for (uint32_t r = 0; r < mmax; r += kLanesPerCell) {
      const uint32_t q = r + uint32_t(sub);
      bool won = false;
      uint32_t v = 0;
      if (q < m) {
        v = adj[p0 + q];
        won = reinterpret_cast<volatile int32_t*>(dist)[v] < 0 &&
              atomicCAS(&dist[v], -1, d + 1) == -1;
      }
      const uint32_t mask = __ballot_sync(0xffffffffu, won);
      if (mask == 0) continue;
      uint32_t base = 0;
      if (lane == __ffs(mask) - 1) base = atomicAdd(out_cnt, uint32_t(__popc(mask)));
      base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
      if (won) {
        if (parent) parent[v] = int32_t(u);
        f_out[base + uint32_t(__popc(mask & ((1u << lane) - 1)))] = v;
      }
    }
  }
}

__global__ void bfs_level(int d, const unsigned long long* __restrict__ off,
                          const uint32_t* __restrict__ deg, const uint32_t* __restrict__ adj,
                          int32_t* dist, int32_t* __restrict__ parent,
                          const uint32_t* __restrict__ f_in, uint32_t* __restrict__ f_out,
                          BfsCounters* c) {
  const uint32_t cnt = c->frontier[d % 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->frontier[(d + 2) % 3] = 0;
    if (cnt > 0) {
      c->depth = uint32_t(d);
      c->reached += cnt;  // the cells at distance d
    }
  }
  if (cnt == 0) return;
  expand_level(d, cnt, off, deg, adj, dist, parent, f_in, f_out, &c->frontier[(d + 1) % 3]);
}

// Grid barrier for a co-resident grid. Returns false when it gave up (or an
// earlier barrier did): the caller must then leave.
// The bound only has to end a wait that can never complete; a level of a
// legitimately huge frontier must not reach it: 2^26 polls of >= 64 ns.
constexpr unsigned kBarrierSpins = 1u << 26;

__device__ __forceinline__ bool grid_barrier(BfsCounters* c, uint32_t polls) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &c->bar_gen;
    volatile unsigned int* err = &c->error;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&c->bar_count, 1u) == gridDim.x - 1) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
      ok = 1;
    } else {
      ok = 0;
      for (uint32_t i = 0; i < polls; ++i) {  // 0 polls gives up at once
        if (*gen != g) {
          ok = 1;
          break;
        }
        if (*err & 2u) break;
        __nanosleep(64);
      }
      if (!ok) atomicOr(&c->error, 2u);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kThreads)
    bfs_all_levels(const unsigned long long* __restrict__ off, const uint32_t* __restrict__ deg,
                   const uint32_t* __restrict__ adj, int32_t* dist, int32_t* __restrict__ parent,
                   uint32_t* f0, uint32_t* f1, BfsCounters* c, uint32_t n, uint32_t polls) {
  for (int d = 0; d <= int(n); ++d) {
    const uint32_t cnt = *reinterpret_cast<volatile unsigned int*>(&c->frontier[d % 3]);
    if (cnt == 0) return;  // the same value in every block: all leave together
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->frontier[(d + 2) % 3] = 0;
      c->depth = uint32_t(d);
      c->reached += cnt;  // the cells at distance d
    }
    expand_level(d, cnt, off, deg, adj, dist, parent, (d & 1) ? f1 : f0, (d & 1) ? f0 : f1,
                 &c->frontier[(d + 1) % 3]);
    if (!grid_barrier(c, polls)) return;
  }
}

}  // namespace

cudaError_t launch_bfs_single(uint32_t n, int32_t* dist, int32_t* parent, const BfsWs& w,
                              cudaStream_t s, bool* launched) {
  *launched = false;
  int dev = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess) return e;
  if (!coop) return cudaSuccess;
  int per_sm = 0;
  e = blocks_per_sm(reinterpret_cast<const void*>(bfs_all_levels), kThreads, 0, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaSuccess;
  const unsigned grid = unsigned(sm_count());  // one block per SM: co-resident, cheap barrier
  e = cudaMemsetAsync(&w.ctr->bar_count, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const unsigned long long* off = w.off;
  const uint32_t* deg = w.deg;
  const uint32_t* adj = w.adj;
  uint32_t* f0 = w.f0;
  uint32_t* f1 = w.f1;
  BfsCounters* c = w.ctr;
  uint32_t polls = wait_limit(kBarrierSpins);
  void* args[] = {&off, &deg, &adj, &dist, &parent, &f0, &f1, &c, &n, &polls};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(bfs_all_levels), dim3(grid),
                                  dim3(kThreads), args, 0, s);
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
    cudaGetLastError();
    return cudaSuccess;
  }
  if (e != cudaSuccess) return e;
  count_launch();
  *launched = true;
  return cudaSuccess;
}

cudaError_t launch_bfs_adjacency(const uint32_t* edges, int64_t n_edges, uint32_t n,
                                 const BfsWs& w, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.deg, 0, size_t(n) * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.cur, 0, size_t(n) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (n_edges > 0) {
    bfs_degree<<<grid_for(size_t(n_edges)), kThreads, 0, s>>>(edges, uint64_t(n_edges), n, w.deg,
                                                               w.ctr);
    count_launch();
  }
  e = scan_exclusive_u32(w.deg, w.off, &w.ctr->n, n, w.total, w.scan, s);
  if (e != cudaSuccess) return e;
  if (n_edges > 0) {
    bfs_fill<<<grid_for(size_t(n_edges)), kThreads, 0, s>>>(edges, uint64_t(n_edges), n, w.off,
                                                             w.cur, w.adj);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_bfs_init(int32_t* dist, int32_t* parent, uint32_t n, uint32_t source,
                            const BfsWs& w, cudaStream_t s) {
  bfs_init<<<grid_for(n), kThreads, 0, s>>>(dist, parent, n, source, w.f0, w.ctr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bfs_levels(int first, int count, uint32_t n, int32_t* dist, int32_t* parent,
                              const BfsWs& w, cudaStream_t s) {
  // Frontiers are a small part of the graph on most levels: one block per SM
  // (grid-stride over the frontier) keeps an empty or short level cheap.
  const size_t want = (size_t(n) + kThreads - 1) / kThreads;
  const int g = int(want < size_t(sm_count()) ? (want < 1 ? 1 : want) : size_t(sm_count()));
  for (int d = first; d < first + count; ++d) {
    const uint32_t* f_in = (d & 1) ? w.f1 : w.f0;
    uint32_t* f_out = (d & 1) ? w.f0 : w.f1;
    bfs_level<<<g, kThreads, 0, s>>>(d, w.off, w.deg, w.adj, dist, parent, f_in, f_out, w.ctr);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace cg
