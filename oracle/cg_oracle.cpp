// Plain CPU oracle for the cell-graph hot path.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or load
// this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
// use it. It shares no code with the CUDA library: no headers, no helpers, no
// tables. It is deliberately slow and written to be checked against the paper
// by eye: single-threaded, exact integer arithmetic, standard-library sort,
// unique and hash map.
//
// What it computes ("Massively Parallel Construction of the Cell Graph"):
//   1. Sign vectors (§2.1, Figure 1): bit i of point p's vector is 1 iff p
//      satisfies constraint c_i, here the closed half-space a_i . p >= b_i,
//      evaluated exactly (128-bit accumulation, so any int32 point/normal and
//      int64 offset is exact).
//   2. Cells (§3.2, tree-based algorithm, first step): sort the vectors and
//      remove duplicates; the remaining vectors are the cells (vertices of G_X).
//   3. Cell-graph edges (§2.2 definition; Algorithm 4 search): for every cell x
//      and every bit k, the vector x with bit k negated is looked up among the
//      cells; a hit is an edge. Each unordered pair is reported once (§2.2
//      asks for pairs i < j, duplicates in X must not repeat pairs).
//   4. The heuristic of §3.1 (Algorithms 1-2): distances to h pivot vectors,
//      inequality (⋆) to skip pairs, a segment-wise comparison of the rest; a
//      second, independent way to the same edges.
//   5. The search tree of §3.2 (Algorithm 3 build, Algorithm 4 walk): the
//      2^r-ary tree over the r-bit digit recoding of the cells, built level by
//      level from index ranges of the sorted digit sequences, and the edges it
//      finds by walking it once per flipped bit.
//   1b. Sign vectors for quadric constraints (curved boundaries, §2.1):
//      the same packing with bit i = [q_i(p) + a_i . p >= b_i], q_i a
//      quadratic form with integer coefficients, in exact 128-bit arithmetic.
//   6. Breadth-first search on G_X (§6: a path in the cell graph is an
//      approximate solution of the motion-planning problem): distances from
//      one cell by the textbook queue BFS over the undirected edge list.
//
// Conventions (the paper fixes none of them):
//   * bit i of a vector lives in word i / B, bit i % B, with B = 32 or 64
//     ("word_bits"); bits >= l of the last word are zero;
//   * vectors are ordered as the unsigned integers sum_i x(i) 2^i, so the last
//     word is the most significant one; cells are numbered in that order;
//   * an edge is the pair (i, j) of cell numbers with i < j; it is emitted from
//     the endpoint whose bit k is 0 (setting a zero bit raises the value, so
//     j > i), cells ascending and bits ascending within a cell, which is
//     lexicographic (i, j) order.
//
// Return codes: 0 ok, -1 bad argument, -2 output capacity too small (the
// required count is still written).

#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

// One packed vector, always held as 64-bit words internally (word j holds bits
// 64j .. 64j+63). Input and output may use 32-bit words; they are converted at
// the edges of each function.
using Vec = std::vector<uint64_t>;

int words_for(int ell, int word_bits) { return (ell + word_bits - 1) / word_bits; }

Vec load_vec(const void* base, int64_t row, int ell, int word_bits) {
  const int w64 = words_for(ell, 64);
  Vec v(w64, 0);
  if (word_bits == 64) {
    const uint64_t* p = static_cast<const uint64_t*>(base) + row * w64;
    for (int j = 0; j < w64; ++j) v[j] = p[j];
  } else {
    const int w32 = words_for(ell, 32);
    const uint32_t* p = static_cast<const uint32_t*>(base) + row * w32;
    for (int j = 0; j < w32; ++j) v[j / 2] |= uint64_t(p[j]) << (32 * (j % 2));
  }
  return v;
}

void store_vec(void* base, int64_t row, const Vec& v, int ell, int word_bits) {
  if (word_bits == 64) {
    const int w64 = words_for(ell, 64);
    uint64_t* p = static_cast<uint64_t*>(base) + row * w64;
    for (int j = 0; j < w64; ++j) p[j] = v[j];
  } else {
    const int w32 = words_for(ell, 32);
    uint32_t* p = static_cast<uint32_t*>(base) + row * w32;
    for (int j = 0; j < w32; ++j) p[j] = uint32_t(v[j / 2] >> (32 * (j % 2)));
  }
}

bool get_bit(const Vec& v, int k) { return (v[k / 64] >> (k % 64)) & 1u; }
void flip_bit(Vec& v, int k) { v[k / 64] ^= uint64_t(1) << (k % 64); }

// Value order: compare from the most significant word down.
bool value_less(const Vec& x, const Vec& y) {
  for (size_t j = x.size(); j-- > 0;) {
    if (x[j] != y[j]) return x[j] < y[j];
  }
  return false;
}

struct VecHash {
  size_t operator()(const Vec& v) const {
    size_t h = 1469598103934665603ull;
    for (uint64_t w : v) h = (h ^ std::hash<uint64_t>()(w)) * 1099511628211ull;
    return h;
  }
};

bool bad_words(int ell, int word_bits) {
  return ell < 1 || (word_bits != 32 && word_bits != 64);
}

// ---- The search tree of §3.2 --------------------------------------------
//
// Digit recoding: a vector of l bits is cut into L = ceil(l / r) segments.
// order = 0 (the paper's, Figure 2): segment h holds bits x(h r) ..
// x(min(l, (h + 1) r) - 1) and digit h is that bit string read as a binary
// number, its first bit the most significant (the last segment is shorter
// when r does not divide l). order = 1 (the library's value order): segment h
// holds bits [max(0, l - (h + 1) r), l - h r) and digit h is their value with
// the higher bit more significant, i.e. the same recoding of the vector read
// from bit l - 1 down.
std::vector<uint32_t> digits_of(const Vec& v, int ell, int r, int order) {
  const int L = (ell + r - 1) / r;
  std::vector<uint32_t> d(size_t(L), 0);
  for (int h = 0; h < L; ++h) {
    uint32_t val = 0;
    if (order == 0) {
      const int lo = h * r, hi = std::min(ell, (h + 1) * r);
      for (int k = lo; k < hi; ++k) val = 2 * val + (get_bit(v, k) ? 1u : 0u);
    } else {
      const int hi = ell - h * r, lo = std::max(0, ell - (h + 1) * r);
      for (int k = hi - 1; k >= lo; --k) val = 2 * val + (get_bit(v, k) ? 1u : 0u);
    }
    d[size_t(h)] = val;
  }
  return d;
}

// A node of the tree: the range [first, last] of the sorted digit sequences
// whose first `level` digits equal the node's path, and its children by digit.
struct TreeNode {
  int level;
  int64_t first, last;
  std::map<uint32_t, int64_t> child;
};

// Algorithm 3: level 0 is the root holding every sequence; for each level the
// sets vectors(C, v) are the maximal runs of equal digit h inside C's range
// (the sequences are sorted, so each set is a range), and every non-empty
// set becomes the v-child of C.
std::vector<TreeNode> build_tree(const std::vector<std::vector<uint32_t>>& seq, int L) {
  std::vector<TreeNode> nodes;
  nodes.push_back(TreeNode{0, 0, int64_t(seq.size()) - 1, {}});
  std::vector<int64_t> frontier{0};
  for (int h = 0; h < L && !seq.empty(); ++h) {
    std::vector<int64_t> next;
    for (int64_t c : frontier) {
      int64_t i = nodes[size_t(c)].first;
      const int64_t last = nodes[size_t(c)].last;
      while (i <= last) {
        int64_t j = i;
        while (j + 1 <= last && seq[size_t(j + 1)][size_t(h)] == seq[size_t(i)][size_t(h)]) ++j;
        const int64_t id = int64_t(nodes.size());
        nodes.push_back(TreeNode{h + 1, i, j, {}});
        nodes[size_t(c)].child[seq[size_t(i)][size_t(h)]] = id;
        next.push_back(id);
        i = j + 1;
      }
    }
    frontier.swap(next);
  }
  return nodes;
}

}  // namespace

extern "C" {

// Step 1 (§2.1): keys[p] = packed [a_i . p >= b_i] for i in [l].
// pts int32[n][d], a int32[l][d], b int64[l]; keys receives n * ceil(l/B) words.
int cgo_pack_signs(const int32_t* pts, int64_t n, int d, const int32_t* a, const int64_t* b,
                   int ell, int word_bits, void* keys) {
  if (n < 0 || d < 1 || bad_words(ell, word_bits)) return -1;
  for (int64_t p = 0; p < n; ++p) {
    Vec v(words_for(ell, 64), 0);
    for (int i = 0; i < ell; ++i) {
      __int128 s = 0;
      for (int k = 0; k < d; ++k) s += __int128(a[int64_t(i) * d + k]) * pts[p * d + k];
      s -= b[i];
      if (s >= 0) v[i / 64] |= uint64_t(1) << (i % 64);
    }
    store_vec(keys, p, v, ell, word_bits);
  }
  return 0;
}

// Step 1 for curved boundaries (§2.1: the constraints c_i are inequalities
// whose boundaries bound the cells; §2 notes that the method carries over to
// more complicated settings than lines): bit i of point p is
//   [ sum_{j<=k} q_i,jk p_j p_k + sum_k a_ik p_k >= b_i ],
// a quadric inequality with integer coefficients, evaluated exactly in 128-bit
// integers. q int32[l][d(d+1)/2] holds the coefficient of the monomial
// p_j p_k for j <= k, in the order (0,0), (0,1), ..., (0,d-1), (1,1), ...,
// (d-1,d-1); a int32[l][d]; b int64[l]. With q = 0 this is cgo_pack_signs.
int cgo_pack_signs_quadric(const int32_t* pts, int64_t n, int d, const int32_t* q,
                           const int32_t* a, const int64_t* b, int ell, int word_bits,
                           void* keys) {
  if (n < 0 || d < 1 || bad_words(ell, word_bits)) return -1;
  const int m = d * (d + 1) / 2;
  for (int64_t p = 0; p < n; ++p) {
    const int32_t* x = pts + p * d;
    Vec v(words_for(ell, 64), 0);
    for (int i = 0; i < ell; ++i) {
      __int128 s = 0;
      int t = 0;
      for (int j = 0; j < d; ++j) {
        for (int k = j; k < d; ++k, ++t) {
          const __int128 mono = __int128(int64_t(x[j]) * int64_t(x[k]));
          s += __int128(q[int64_t(i) * m + t]) * mono;
        }
      }
      for (int k = 0; k < d; ++k) s += __int128(a[int64_t(i) * d + k]) * x[k];
      s -= b[i];
      if (s >= 0) v[i / 64] |= uint64_t(1) << (i % 64);
    }
    store_vec(keys, p, v, ell, word_bits);
  }
  return 0;
}

// Step 2 (§3.2): sort the n vectors by value and drop duplicates. cells must
// hold n vectors; *n_cells receives U. point_cell (nullable) receives, for each
// input vector, the number of its cell.
int cgo_dedup(const void* keys, int64_t n, int ell, int word_bits, void* cells,
              int64_t* n_cells, uint32_t* point_cell) {
  if (n < 0 || bad_words(ell, word_bits) || !n_cells) return -1;
  std::vector<Vec> v;
  v.reserve(size_t(n));
  for (int64_t p = 0; p < n; ++p) v.push_back(load_vec(keys, p, ell, word_bits));
  std::vector<Vec> u = v;
  std::sort(u.begin(), u.end(), value_less);
  u.erase(std::unique(u.begin(), u.end()), u.end());
  for (size_t i = 0; i < u.size(); ++i) store_vec(cells, int64_t(i), u[i], ell, word_bits);
  *n_cells = int64_t(u.size());
  if (point_cell) {
    for (int64_t p = 0; p < n; ++p) {
      auto it = std::lower_bound(u.begin(), u.end(), v[size_t(p)], value_less);
      point_cell[p] = uint32_t(it - u.begin());
    }
  }
  return 0;
}

// Step 3 (§2.2, Algorithm 4): for cells listed in rows (all cells when rows is
// null), look up every single-bit change that sets a zero bit; each hit (i, j)
// is one edge. cells must be sorted and unique (the output of cgo_dedup).
// edges receives pairs (i, j) as uint32[E][2].
int cgo_neighbors_h1_rows(const void* cells, int64_t n_cells, int ell, int word_bits,
                          const int64_t* rows, int64_t n_rows, uint32_t* edges,
                          int64_t edges_cap, int64_t* n_edges) {
  if (n_cells < 0 || bad_words(ell, word_bits) || !n_edges) return -1;
  std::vector<Vec> u;
  u.reserve(size_t(n_cells));
  std::unordered_map<Vec, uint32_t, VecHash> index;
  index.reserve(size_t(n_cells) * 2);
  for (int64_t i = 0; i < n_cells; ++i) {
    u.push_back(load_vec(cells, i, ell, word_bits));
    index.emplace(u.back(), uint32_t(i));
  }
  const int64_t count = rows ? n_rows : n_cells;
  int64_t e = 0;
  for (int64_t r = 0; r < count; ++r) {
    const int64_t i = rows ? rows[r] : r;
    if (i < 0 || i >= n_cells) return -1;
    for (int k = 0; k < ell; ++k) {
      if (get_bit(u[size_t(i)], k)) continue;
      Vec y = u[size_t(i)];
      flip_bit(y, k);
      auto it = index.find(y);
      if (it == index.end()) continue;
      if (e < edges_cap) {
        edges[2 * e] = uint32_t(i);
        edges[2 * e + 1] = it->second;
      }
      ++e;
    }
  }
  *n_edges = e;
  return e > edges_cap ? -2 : 0;
}

int cgo_neighbors_h1(const void* cells, int64_t n_cells, int ell, int word_bits, uint32_t* edges,
                     int64_t edges_cap, int64_t* n_edges) {
  return cgo_neighbors_h1_rows(cells, n_cells, ell, word_bits, nullptr, 0, edges, edges_cap,
                               n_edges);
}

// The heuristic of §3.1 over the cells x_0 .. x_{n-1} (sorted and unique).
// Algorithm 1 (ComputeDist): dist(x_p, x_j) for every pivot p in [h] (the
// first h cells) and every cell j, the number of positions where their bits
// differ. Algorithm 2: every pair i < j is first tested against inequality
// (⋆) with the pivots; a pair passes when |dist(x_i, x_p) - dist(x_j, x_p)|
// <= 1 for every p (readings: the printed "> 1" test is inverted --
// as_printed = 1 applies it literally; pivots are ordinary vertices, so the
// pair loop starts at 0; dist is filled for every j). A pair that passes is
// compared the way a block of w threads does it: thread t counts the
// positions of its segment [t s, min((t + 1) s, l)), s = ceil(l / w), where
// the bits differ, stopping at 2; the counts are added in thread order,
// stopping at 2; a total of exactly 1 outputs (i, j). Pairs come out with i
// ascending, then j ascending. n_tested receives the number of pairs that
// passed the pivot test (with h = 0 every pair does: the naive method).
int cgo_heuristic(const void* cells, int64_t n_cells, int ell, int word_bits, int h, int w,
                  int as_printed, uint32_t* edges, int64_t edges_cap, int64_t* n_edges,
                  int64_t* n_tested) {
  if (n_cells < 0 || bad_words(ell, word_bits) || !n_edges || !n_tested || h < 0 || w < 1)
    return -1;
  std::vector<Vec> x;
  x.reserve(size_t(n_cells));
  for (int64_t i = 0; i < n_cells; ++i) x.push_back(load_vec(cells, i, ell, word_bits));
  const int64_t pivots = std::min<int64_t>(h, n_cells);
  // Algorithm 1.
  std::vector<std::vector<int>> dist(size_t(pivots), std::vector<int>(size_t(n_cells), 0));
  for (int64_t p = 0; p < pivots; ++p)
    for (int64_t j = 0; j < n_cells; ++j) {
      int c = 0;
      for (int k = 0; k < ell; ++k) c += get_bit(x[size_t(p)], k) != get_bit(x[size_t(j)], k);
      dist[size_t(p)][size_t(j)] = c;
    }
  // Algorithm 2.
  const int seg = (ell + w - 1) / w;
  int64_t e = 0, tested = 0;
  std::vector<int> results(static_cast<size_t>(w));
  for (int64_t i = 0; i < n_cells; ++i) {
    for (int64_t j = i + 1; j < n_cells; ++j) {
      bool pass = true;
      for (int64_t p = 0; p < pivots; ++p) {
        const int diff = std::abs(dist[size_t(p)][size_t(i)] - dist[size_t(p)][size_t(j)]);
        const bool ok = as_printed ? diff > 1 : diff <= 1;
        if (!ok) {
          pass = false;
          break;
        }
      }
      if (!pass) continue;
      ++tested;
      for (int t = 0; t < w; ++t) {
        int c = 0;
        for (int k = t * seg; k < std::min((t + 1) * seg, ell); ++k) {
          if (get_bit(x[size_t(i)], k) != get_bit(x[size_t(j)], k)) ++c;
          if (c >= 2) break;
        }
        results[size_t(t)] = c;
      }
      int count = 0;
      for (int t = 0; t < w; ++t) {
        count += results[size_t(t)];
        if (count >= 2) break;
      }
      if (count != 1) continue;
      if (e < edges_cap) {
        edges[2 * e] = uint32_t(i);
        edges[2 * e + 1] = uint32_t(j);
      }
      ++e;
    }
  }
  *n_edges = e;
  *n_tested = tested;
  return e > edges_cap ? -2 : 0;
}

// Breadth-first search (textbook FIFO queue) on the undirected graph with
// n_cells vertices and the edges (i, j) of the list: dist[v] = number of
// edges on a shortest path from source to v, -1 when v is unreachable.
int cgo_bfs(const uint32_t* edges, int64_t n_edges, int64_t n_cells, int64_t source,
            int32_t* dist) {
  if (n_edges < 0 || n_cells < 0 || source < 0 || source >= n_cells || !dist) return -1;
  std::vector<std::vector<uint32_t>> adj(static_cast<size_t>(n_cells));
  for (int64_t e = 0; e < n_edges; ++e) {
    const uint32_t i = edges[2 * e], j = edges[2 * e + 1];
    if (int64_t(i) >= n_cells || int64_t(j) >= n_cells) return -1;
    adj[i].push_back(j);
    adj[j].push_back(i);
  }
  for (int64_t v = 0; v < n_cells; ++v) dist[v] = -1;
  std::vector<uint32_t> queue;
  queue.reserve(size_t(n_cells));
  dist[source] = 0;
  queue.push_back(uint32_t(source));
  for (size_t head = 0; head < queue.size(); ++head) {
    const uint32_t u = queue[head];
    for (uint32_t v : adj[u])
      if (dist[v] < 0) {
        dist[v] = dist[u] + 1;
        queue.push_back(v);
      }
  }
  return 0;
}

// Node counts of the search tree per level (counts[0] = 1 for the root, up to
// counts[L]) and, when edges is non-null, the edges found by Algorithm 4's
// walk: for every cell and every zero bit k, the digits of the cell with bit
// k set are followed from the root; reaching the last level is a hit. cells
// must be sorted and unique (the output of cgo_dedup); edges as for
// cgo_neighbors_h1 (cell numbers in value order).
int cgo_tree(const void* cells, int64_t n_cells, int ell, int word_bits, int r, int order,
             int64_t* counts, int counts_cap, uint32_t* edges, int64_t edges_cap,
             int64_t* n_edges) {
  if (n_cells < 0 || bad_words(ell, word_bits) || r < 1 || r > 16 || (order != 0 && order != 1))
    return -1;
  const int L = (ell + r - 1) / r;
  if (counts_cap < L + 1) return -1;
  std::vector<Vec> u;
  for (int64_t i = 0; i < n_cells; ++i) u.push_back(load_vec(cells, i, ell, word_bits));
  // Sort the digit sequences lexicographically, remembering each one's cell.
  std::vector<std::pair<std::vector<uint32_t>, uint32_t>> tagged;
  for (int64_t i = 0; i < n_cells; ++i)
    tagged.emplace_back(digits_of(u[size_t(i)], ell, r, order), uint32_t(i));
  std::sort(tagged.begin(), tagged.end());
  std::vector<std::vector<uint32_t>> seq;
  for (auto& t : tagged) seq.push_back(t.first);
  const std::vector<TreeNode> nodes = build_tree(seq, L);
  for (int h = 0; h <= L; ++h) counts[h] = 0;
  for (const TreeNode& nd : nodes) ++counts[nd.level];
  if (!edges) return 0;
  int64_t e = 0;
  for (int64_t i = 0; i < n_cells; ++i) {
    for (int k = 0; k < ell; ++k) {
      if (get_bit(u[size_t(i)], k)) continue;
      Vec y = u[size_t(i)];
      flip_bit(y, k);
      const std::vector<uint32_t> dy = digits_of(y, ell, r, order);
      int64_t c = 0;
      bool found = true;
      for (int h = 0; h < L; ++h) {
        auto it = nodes[size_t(c)].child.find(dy[size_t(h)]);
        if (it == nodes[size_t(c)].child.end()) {
          found = false;
          break;
        }
        c = it->second;
      }
      if (!found) continue;
      const uint32_t j = tagged[size_t(nodes[size_t(c)].first)].second;
      if (e < edges_cap) {
        edges[2 * e] = uint32_t(i);
        edges[2 * e + 1] = j;
      }
      ++e;
    }
  }
  *n_edges = e;
  return e > edges_cap ? -2 : 0;
}

// Digit recoding of every cell (as used by cgo_tree): digits[i][h], L =
// ceil(l / r) digits per cell.
int cgo_tree_digits(const void* cells, int64_t n_cells, int ell, int word_bits, int r, int order,
                    uint32_t* digits) {
  if (n_cells < 0 || bad_words(ell, word_bits) || r < 1 || r > 16 || (order != 0 && order != 1))
    return -1;
  const int L = (ell + r - 1) / r;
  for (int64_t i = 0; i < n_cells; ++i) {
    const std::vector<uint32_t> d = digits_of(load_vec(cells, i, ell, word_bits), ell, r, order);
    for (int h = 0; h < L; ++h) digits[i * L + h] = d[size_t(h)];
  }
  return 0;
}

// Steps 1-3 for one scene: points -> cells and edges.
int cgo_build(const int32_t* pts, int64_t n, int d, const int32_t* a, const int64_t* b, int ell,
              int word_bits, void* cells, int64_t* n_cells, uint32_t* edges, int64_t edges_cap,
              int64_t* n_edges) {
  if (n < 0 || bad_words(ell, word_bits)) return -1;
  const int64_t row_bytes = int64_t(words_for(ell, word_bits)) * (word_bits / 8);
  std::vector<unsigned char> keys(size_t(n * row_bytes) + 1);
  int rc = cgo_pack_signs(pts, n, d, a, b, ell, word_bits, keys.data());
  if (rc) return rc;
  rc = cgo_dedup(keys.data(), n, ell, word_bits, cells, n_cells, nullptr);
  if (rc) return rc;
  return cgo_neighbors_h1(cells, *n_cells, ell, word_bits, edges, edges_cap, n_edges);
}

}  // extern "C"
