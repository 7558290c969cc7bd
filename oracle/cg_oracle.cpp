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
#include <cstdint>
#include <cstring>
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
