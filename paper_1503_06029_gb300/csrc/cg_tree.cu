// TREE lookup strategy: the search tree of §3.2 (Algorithm 3) over the sorted
// cells, built level by level on the device, one round of kernels per tree
// level (the paper's global synchronisation between levels).
//
// Layout and differences from the paper's tree (uncompressed, digits from
// x(0)):
//   * r = 8 (the paper's choice), digits read from the most significant end
//     of the value order, so that every node is a contiguous range of the
//     sorted cells (the paper sorts in its own digit order for the same
//     reason);
//   * leaf-valued: a node whose range holds a single cell is a leaf, and the
//     lookup compares the whole vector with that cell (the remaining digits
//     are not materialised);
//   * single-child chains are contracted: an internal node stores the level
//     lv on which its children differ (the first level where the digits of its
//     cells are not all equal); the digits above lv are checked by the final
//     comparison. The tree then has fewer than 2 U nodes instead of up to
//     U l / r.
//
// Build, one round per depth of the contracted tree (at most ceil(l / 8)):
//   dlv[i]  = first digit level on which cells i - 1 and i differ;
//   par[i]  = internal node of the current depth whose range holds cell i;
//   a. lv(node) = min dlv[i] over the node's range (minus its first cell);
//   b. a child starts at the node's first cell and at every i with dlv[i] = lv;
//   c. exclusive scan of those starts gives the children consecutive ids;
//   d. children are created, the parents' digit bitmaps and first-child ids set;
//   e. child sizes from the next start of the same parent;
//   f. par[i] moves to the child of i when that child has 2 or more cells.
#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kNone = 0xffffffffu;

struct TreeCtl {
  unsigned int base;                // next free node id
  unsigned int active;              // internal nodes created by the last round
  unsigned long long new_count;     // nodes created by this round (scan total)
};

int grid_for(size_t items, int per_block, int blocks_per_sm = 8) {
  const size_t want = (items + per_block - 1) / per_block;
  const size_t cap = size_t(sm_count()) * blocks_per_sm;
  size_t g = want < cap ? want : cap;
  return int(g < 1 ? 1 : g);
}

// Highest set bit of the 64-bit-word vector a xor b (W words), or -1.
__device__ __forceinline__ int top_diff(const uint64_t* a, const uint64_t* b, int w) {
  for (int q = w - 1; q >= 0; --q) {
    const uint64_t x = a[q] ^ b[q];
    if (x) return 64 * q + 63 - __clzll(static_cast<long long>(x));
  }
  return -1;
}

__device__ __forceinline__ uint32_t digit_of(const uint64_t* row, int ell, int lv) {
  int lo, hi;
  tree_digit_bits(ell, lv, &lo, &hi);
  const int q = lo >> 6, sh = lo & 63;
  uint64_t v = row[q] >> sh;
  if (sh + (hi - lo) > 64) v |= row[q + 1] << (64 - sh);
  return uint32_t(v & ((1ull << (hi - lo)) - 1ull));
}

__global__ void tree_init(const uint64_t* __restrict__ cells, int w, int ell,
                          const DevCounters* ctr, uint32_t max_n, TreeNode* nodes,
                          uint32_t* __restrict__ dlv, uint32_t* __restrict__ par, TreeCtl* ctl) {
  if (ctr->overflow) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    TreeNode root{};
    root.first = 0;
    root.lo = 0;
    root.cnt = u;
    root.lv = kNone;
    nodes[0] = root;
    ctl->base = 1;
    ctl->active = u >= 2 ? 1u : 0u;
    ctl->new_count = 0;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    par[i] = u >= 2 ? 0u : kNone;
    if (i == 0) {
      dlv[i] = kNone;
    } else {
      const int b = top_diff(cells + uint64_t(i - 1) * w, cells + uint64_t(i) * w, w);
      dlv[i] = b < 0 ? 0u : uint32_t((ell - 1 - b) >> 3);
    }
  }
}

// a. Branching level of every frontier node (and the id bookkeeping of the
//    previous round).
__global__ void tree_min(const DevCounters* ctr, uint32_t max_n, TreeNode* nodes,
                         const uint32_t* __restrict__ dlv, const uint32_t* __restrict__ par,
                         TreeCtl* ctl) {
  if (ctr->overflow || ctl->active == 0) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t p = par[i];
    if (p == kNone || i == nodes[p].lo) continue;
    atomicMin(&nodes[p].lv, dlv[i]);
  }
}

// b. Child starts.
__global__ void tree_flags(const DevCounters* ctr, uint32_t max_n, const TreeNode* nodes,
                           const uint32_t* __restrict__ dlv, const uint32_t* __restrict__ par,
                           uint32_t* __restrict__ flag, const TreeCtl* ctl) {
  if (ctr->overflow || ctl->active == 0) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t p = par[i];
    flag[i] = (p != kNone && (i == nodes[p].lo || dlv[i] == nodes[p].lv)) ? 1u : 0u;
  }
}

// d. Children: ids base + pos[i], parents' bitmaps and first-child ids.
__global__ void tree_make(const uint64_t* __restrict__ cells, int w, int ell,
                          const DevCounters* ctr, uint32_t max_n, TreeNode* nodes,
                          uint32_t node_cap, const uint32_t* __restrict__ par,
                          const uint32_t* __restrict__ flag,
                          const unsigned long long* __restrict__ pos, uint32_t* __restrict__ starts,
                          uint32_t* __restrict__ nparent, TreeCtl* ctl,
                          DevCounters* wctr) {
  if (ctr->overflow || ctl->active == 0) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint32_t base = ctl->base;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    const uint32_t p = par[i];
    const uint32_t q = uint32_t(pos[i]);
    const uint32_t c = base + q;
    if (c >= node_cap) {
      atomicOr(&wctr->error, 4u);  // cannot happen: fewer than 2 U nodes
      continue;
    }
    TreeNode nd{};
    nd.lo = i;
    nd.lv = kNone;
    nodes[c] = nd;
    starts[q] = i;
    nparent[q] = p;
    const uint32_t v = digit_of(cells + uint64_t(i) * w, ell, int(nodes[p].lv));
    atomicOr(&nodes[p].bm[v >> 5], 1u << (v & 31));
    if (i == nodes[p].lo) nodes[p].first = c;
  }
}

// e. Child sizes; counts the new internal nodes.
__global__ void tree_sizes(const DevCounters* ctr, TreeNode* nodes,
                           const uint32_t* __restrict__ starts,
                           const uint32_t* __restrict__ nparent, TreeCtl* ctl) {
  if (ctr->overflow || ctl->active == 0) return;
  const uint32_t base = ctl->base;
  const uint32_t m = uint32_t(ctl->new_count);
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    const uint32_t p = nparent[q];
    const uint32_t end =
        (q + 1 < m && nparent[q + 1] == p) ? starts[q + 1] : nodes[p].lo + nodes[p].cnt;
    nodes[base + q].cnt = end - starts[q];
  }
}

// f. Cells move to their child when it is internal.
__global__ void tree_descend(const DevCounters* ctr, uint32_t max_n, const TreeNode* nodes,
                             uint32_t* __restrict__ par, const uint32_t* __restrict__ flag,
                             const unsigned long long* __restrict__ pos, TreeCtl* ctl,
                             unsigned int* next_active) {
  if (ctr->overflow || ctl->active == 0) return;
  const uint32_t u = min(ctr->n_unique, max_n);
  const uint32_t base = ctl->base;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += gridDim.x * blockDim.x) {
    const uint32_t p = par[i];
    if (p == kNone) continue;
    const uint32_t c = base + uint32_t(pos[i]) + flag[i] - 1;
    const bool internal = nodes[c].cnt >= 2;
    par[i] = internal ? c : kNone;
    if (internal && flag[i]) atomicAdd(next_active, 1u);
  }
}

// g. Next round: ids move past this round's nodes.
__global__ void tree_advance(TreeCtl* ctl, unsigned int* next_active) {
  if (ctl->active == 0) return;
  ctl->base += uint32_t(ctl->new_count);
  ctl->new_count = 0;
  ctl->active = *next_active;
  *next_active = 0;
}

struct TreeScratch {
  TreeCtl* ctl;
  unsigned int* next_active;
  uint32_t* dlv;
  uint32_t* par;
  uint32_t* flag;
  unsigned long long* pos;
  uint32_t* starts;
  uint32_t* nparent;
  void* scan;
  size_t bytes;
};

TreeScratch carve_tree(void* base, size_t max_n) {
  TreeScratch t{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = base ? static_cast<char*>(base) + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t n = max_n > 0 ? max_n : 1;
  t.ctl = static_cast<TreeCtl*>(take(sizeof(TreeCtl)));
  t.next_active = static_cast<unsigned int*>(take(sizeof(unsigned int)));
  t.dlv = static_cast<uint32_t*>(take(n * 4));
  t.par = static_cast<uint32_t*>(take(n * 4));
  t.flag = static_cast<uint32_t*>(take(n * 4));
  t.pos = static_cast<unsigned long long*>(take(n * 8));
  t.starts = static_cast<uint32_t*>(take(n * 4));
  t.nparent = static_cast<uint32_t*>(take(n * 4));
  t.scan = take(scan_scratch_bytes(n));
  t.bytes = off + 256;
  return t;
}

}  // namespace

size_t tree_node_capacity(size_t max_n) { return 2 * (max_n > 0 ? max_n : 1) + 1; }

size_t tree_scratch_bytes(size_t max_n) { return carve_tree(nullptr, max_n).bytes; }

cudaError_t launch_tree_build(const uint64_t* cells, int w64, int ell, const DevCounters* ctr,
                              size_t max_n, TreeNode* nodes, void* scratch, cudaStream_t s) {
  if (max_n == 0) return cudaSuccess;
  TreeScratch t = carve_tree(scratch, max_n);
  const int g = grid_for(max_n, kThreads);
  DevCounters* wctr = const_cast<DevCounters*>(ctr);
  cudaError_t e = cudaMemsetAsync(t.next_active, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  tree_init<<<g, kThreads, 0, s>>>(cells, w64, ell, ctr, uint32_t(max_n), nodes, t.dlv, t.par,
                                   t.ctl);
  count_launch();
  const uint32_t node_cap = uint32_t(tree_node_capacity(max_n));
  const int levels = (ell + 7) / 8;
  for (int round = 0; round < levels; ++round) {
    tree_min<<<g, kThreads, 0, s>>>(ctr, uint32_t(max_n), nodes, t.dlv, t.par, t.ctl);
    tree_flags<<<g, kThreads, 0, s>>>(ctr, uint32_t(max_n), nodes, t.dlv, t.par, t.flag, t.ctl);
    count_launch(2);
    e = scan_exclusive_u32(t.flag, t.pos, &ctr->n_unique, max_n, &t.ctl->new_count, t.scan, s);
    if (e != cudaSuccess) return e;
    tree_make<<<g, kThreads, 0, s>>>(cells, w64, ell, ctr, uint32_t(max_n), nodes, node_cap,
                                     t.par, t.flag, t.pos, t.starts, t.nparent, t.ctl, wctr);
    tree_sizes<<<g, kThreads, 0, s>>>(ctr, nodes, t.starts, t.nparent, t.ctl);
    tree_descend<<<g, kThreads, 0, s>>>(ctr, uint32_t(max_n), nodes, t.par, t.flag, t.pos, t.ctl,
                                        t.next_active);
    tree_advance<<<1, 1, 0, s>>>(t.ctl, t.next_active);
    count_launch(4);
  }
  return cudaGetLastError();
}

}  // namespace cg
