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
    c->reached = 1;
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

__global__ void bfs_level(int d, const unsigned long long* __restrict__ off,
                          const uint32_t* __restrict__ deg, const uint32_t* __restrict__ adj,
                          int32_t* dist, int32_t* __restrict__ parent,
                          const uint32_t* __restrict__ f_in, uint32_t* __restrict__ f_out,
                          BfsCounters* c) {
  const uint32_t cnt = c->frontier[d % 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->frontier[(d + 2) % 3] = 0;
    if (cnt > 0) c->depth = uint32_t(d);
  }
  if (cnt == 0) return;
  uint32_t* out_cnt = &c->frontier[(d + 1) % 3];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const uint32_t u = f_in[k];
    const unsigned long long p0 = off[u];
    const uint32_t m = deg[u];
    for (uint32_t q = 0; q < m; ++q) {
      const uint32_t v = adj[p0 + q];
      if (dist[v] >= 0) continue;
      if (atomicCAS(&dist[v], -1, d + 1) != -1) continue;
      if (parent) parent[v] = int32_t(u);
      f_out[atomicAdd(out_cnt, 1u)] = v;
      atomicAdd(&c->reached, 1u);
    }
  }
}

}  // namespace

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
