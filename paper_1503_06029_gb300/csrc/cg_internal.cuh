// Internal declarations shared by the CUDA translation units of libcellgraph.
// Nothing here is part of the C-ABI (include/cellgraph.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <algorithm>

namespace cg {

// Empty slot marker of the open-addressing tables. For vectors of l <= 64
// bits the table stores the vector itself, so the all-ones vector (possible
// only when l == 64) is tracked by a flag in DevCounters instead of a slot.
constexpr uint64_t kEmpty = ~0ull;

// Device-resident counters of one build. Zeroed by the first kernel of a build.
struct DevCounters {
  unsigned int n_unique;      // U: distinct vectors inserted
  unsigned int overflow;      // a table or list ran past its capacity
  unsigned long long n_edges; // E
  unsigned int ones_present;  // the all-ones vector (l == 64) is a cell
  unsigned int ones_rank;     // its cell number
  unsigned int error;         // device-side consistency failures (bit set)
  unsigned int ticket;        // work counter of the single-pass edge kernel
  unsigned int tc_spill;      // tiles the tensor-core sign kernel left to the fp32 one
  unsigned int sorted;        // 1: the one-cluster sort handled the distinct vectors
  unsigned int msort_done;    // wide-row merge sort: nonzero when every run of equal
                              // cached keys was ordered without the full-row pass
  unsigned int pad[5];
};

// Bits of DevCounters::error.
constexpr unsigned kErrTimeout = 64u;    // a bounded device-side wait ran out
constexpr unsigned kErrUnsorted = 128u;  // given cells are not ascending and unique
constexpr unsigned kErrHighBits = 256u;  // given cells have bits set at or above l
static_assert(sizeof(DevCounters) == 64, "DevCounters layout");

// ---------------------------------------------------------------------------
// Hashing (device). mix64 is the 64-bit finaliser of MurmurHash3 (Appleby,
// public domain); splitmix64 is the output function of SplitMix64 (Steele, Lea,
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// 64 bits of a row of 64-bit words starting at bit off (-64 < off <= l - 64;
// below bit 0 reads as zeros), and the top 128 bits of a row of l > 64 bits as
// (high, low): the cached sort key of the wide sorts (whole vector when
// l <= 128).
__device__ __forceinline__ uint64_t bits64_at(const uint64_t* row, int off) {
  if (off < 0) return row[0] << (-off);
  const int q = off >> 6, sh = off & 63;
  const uint64_t lo = row[q] >> sh;
  return sh ? (lo | (row[q + 1] << (64 - sh))) : lo;
}

__device__ __forceinline__ ulonglong2 top128(const uint64_t* row, int ell) {
  return make_ulonglong2(bits64_at(row, ell - 64), bits64_at(row, ell - 128));
}

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Random 64-bit value attached to bit k; the fingerprint of a vector is the XOR
// of the values of its set bits, so flipping bit k XORs the fingerprint with
// fp_bit(k) (a GF(2)-linear hash).
__host__ __device__ __forceinline__ uint64_t fp_bit(int k) {
  return splitmix64(0x5eed0c0ffee00000ull + uint64_t(k));
}

// ---------------------------------------------------------------------------
// Launch bookkeeping (cg_api.cu).
// ---------------------------------------------------------------------------
void count_launch(int n = 1);
void set_last_error(const char* msg);  // message returned by cg_last_error()
// Polls a bounded device-side wait of a kernel launched now may make before it
// gives up: `dflt`, or the smaller test limit set with cg_set_wait_limit.
uint32_t wait_limit(uint32_t dflt);
int sm_count();  // SMs of the current device (cached per device)
// Raises kern's dynamic shared memory limit on the current device to at least
// `bytes` (a runtime call only the first time a larger size is needed;
// thread-safe).
cudaError_t ensure_smem_limit(const void* kern, size_t bytes);
// Resident blocks per SM of kern for a block size and dynamic shared memory
// size, on the current device (computed once, then cached; thread-safe).
cudaError_t blocks_per_sm(const void* kern, int threads, size_t smem, int* out);

// ---------------------------------------------------------------------------
// Step 1: sign vectors (cg_pack.cu).
// ---------------------------------------------------------------------------
struct PackArgs {
  const int32_t* pts;
  int64_t n;
  int d;
  const int32_t* a;
  const int64_t* b;
  int ell;
  // Optional list of 128-point tiles to process (instead of all points):
  // tiles[0 .. *n_tiles) are tile numbers (points [128 t, 128 t + 128)).
  const uint32_t* tiles = nullptr;
  const unsigned int* n_tiles = nullptr;
};

// keys[n][W] in word_bits-bit words.
cudaError_t launch_pack_store(const PackArgs& pa, int word_bits, void* keys, cudaStream_t s);

// Open-addressing table for vectors of l <= 64 bits (the vector is the key).
// Home slot: Fibonacci hashing, the top log2(cap) bits of key * 2^64/phi
// (Knuth, TAOCP vol. 3, 6.4); linear probing.
struct SmallTable {
  uint64_t* keys;      // [cap], kEmpty = free
  uint32_t* vals;      // [cap], cell number of the key in the same slot
  uint32_t mask;       // cap - 1 (cap a power of two)
  int shift;           // 64 - log2(cap)
  uint64_t* ulist;     // [ucap] distinct vectors, in insertion order
  uint32_t ucap;
  DevCounters* ctr;
};

inline int table_shift(size_t cap) {
  int b = 0;
  while ((size_t(1) << b) < cap) ++b;
  return 64 - b;
}

// Fused steps 1-2 for l <= 64: every vector goes straight into the table
// (no vector is written to memory); distinct vectors are appended to ulist.
cudaError_t launch_pack_insert(const PackArgs& pa, const SmallTable& t, cudaStream_t s);

// Box grid over the points for the sign step (l <= 64): count[k] slabs of
// 2^shift[k] integers along axis k, starting at lo[k]. Cell (g_0 .. g_{d-1}),
// stored at g_0 + count[0] (g_1 + count[1] (g_2 + ...)), is the integer box
// of its slabs; `base` holds bit i when a_i . p >= b_i at every point of that
// box, `list` the constraints whose sign may change inside it (up to 7 of
// them; a count of 255 means more).
// A point's vector is then base plus the exact tests of its cell's crossing
// constraints only. lo and shift are chosen on the device from a sample of
// the points (a point outside the grid tests every constraint).
struct GridCell {
  uint64_t base;
  uint64_t list;  // crossing constraints: indices in bytes 0-6, their count in byte 7
};
constexpr int kGridMaxRows = 64;       // l <= 64
constexpr int kGridMaxQuads = 2;       // float4s per constraint row (d <= 4)
constexpr int kGridMaxCentres = 2304;  // slabs of all axes together
// The grid's placement and what its classification reads, written once per
// build by the placement kernel: slabs per axis, the constraint rows scaled
// for the grid's box with each row's threshold 2 + R, and the slab centres
// (axis k's from cen_off[k]).
struct GridGeom {
  int32_t lo[4];
  int32_t shift[4];
  int32_t count[4];
  int32_t cen_off[4];
  float4 rows[kGridMaxRows * kGridMaxQuads];
  float qlim[kGridMaxRows];
  float cen[kGridMaxCentres];
};
struct PackGrid {
  GridCell* cells;  // [2^total_bits] (the grid uses at most that many)
  GridGeom* geom;   // written by the placement kernel
  int total_bits;
};
// log2 of the cell budget of the grid for a scene of n points (0: no grid);
// `always` asks for one even where it does not pay (tests).
int pack_grid_bits(int64_t n, bool always);
// The grid's set-up (sample box, placement, cell classification), and the
// sign + insert kernel that reads it (enqueue it after the set-up on s).
cudaError_t launch_pack_grid_setup(const PackArgs& pa, const PackGrid& g, cudaStream_t s);
cudaError_t launch_pack_insert_grid(const PackArgs& pa, const SmallTable& t, const PackGrid& g,
                                    cudaStream_t s);
// The same for many scenes in one launch (a batch): scene s (device array)
// owns the 128-point warp tiles [tile0, next scene's tile0) of the batch's
// tile numbering, total_tiles in all; every scene has dimension d and at most
// 32 nch constraints (nch = 1 or 2). A warp takes a contiguous range of tiles
// and rebuilds its constraint rows when the scene or the tile bound changes.
struct SegPackScene {
  const int32_t* pts;
  int64_t n;
  const int32_t* a;
  const int64_t* b;
  int ell;
  SmallTable t;
  uint64_t tile0;
  uint64_t* keys64 = nullptr;  // 64 < l <= 256: the vectors are written here instead
};
cudaError_t launch_pack_insert_seg(const SegPackScene* scenes, int n_scenes, uint64_t total_tiles,
                                   int d, int nch, cudaStream_t s);
// Many scenes of 64 < l <= 256 (W = w64 = 2..4 words) and d <= 3 in one
// launch: each scene's sign vectors written to its keys64 (W words a point).
cudaError_t launch_pack_store_seg(const SegPackScene* scenes, int n_scenes, uint64_t total_tiles,
                                  int d, int w64, cudaStream_t s);
// Same on the tensor cores (cg_pack_tc.cu): l <= 64, d <= 4; tiles outside the
// exact-split ranges are evaluated in fp32 with exact re-evaluation.
// spill_tiles: ceil(n / 128) words of scratch.
cudaError_t launch_pack_tc_insert(const PackArgs& pa, const SmallTable& t, uint32_t* spill_tiles,
                                  cudaStream_t s);

// ---------------------------------------------------------------------------
// Programmatic dependent launch. Kernels of a build's chain are launched with
// launch_dep: the next kernel may be launched while the previous one still
// runs, and its blocks start with griddep_wait(), which returns once every
// earlier kernel of the stream has completed and its writes are visible (a
// no-op for a kernel launched without the attribute). griddep_release() lets
// the next kernel's launch begin early; it orders nothing.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
cudaError_t launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
#endif

// ---------------------------------------------------------------------------
// Device helpers used by several translation units.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t home_slot(uint64_t key, int shift) {
  return uint32_t((key * 0x9E3779B97F4A7C15ull) >> shift);
}

// Appends a newly inserted distinct vector to the table's list.
__device__ __forceinline__ void small_append(const SmallTable& t, uint64_t key) {
  const unsigned int idx = atomicAdd(&t.ctr->n_unique, 1u);
  if (idx < t.ucap) {
    t.ulist[idx] = key;
  } else {
    atomicOr(&t.ctr->overflow, 1u);
  }
}

// Inserts one vector (l <= 64) into the dedup table, starting at `slot` whose
// content `cur` the caller has already read; the first inserter of a value
// appends it to the list of cells (§3.2: duplicates are removed). A table that
// is full raises the overflow flag.
__device__ __forceinline__ void small_insert_from(const SmallTable& t, uint64_t key,
                                                  uint32_t slot, uint64_t cur) {
  if (key == kEmpty) {
    if (atomicExch(&t.ctr->ones_present, 1u) == 0u) small_append(t, key);
    return;
  }
  for (uint32_t probe = 0; probe <= t.mask; ++probe) {
    if (cur == key) return;
    if (cur == kEmpty) {
      const unsigned long long old =
          atomicCAS(reinterpret_cast<unsigned long long*>(t.keys + slot),
                    static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(key));
      if (old == kEmpty) {
        small_append(t, key);
        return;
      }
      if (old == key) return;
    }
    slot = (slot + 1) & t.mask;
    cur = t.keys[slot];
  }
  atomicOr(&t.ctr->overflow, 1u);
}

__device__ __forceinline__ void small_insert(const SmallTable& t, uint64_t key) {
  const uint32_t slot = home_slot(key, t.shift);
  small_insert_from(t, key, slot, key == kEmpty ? 0ull : t.keys[slot]);
}

// Slot holding `key` (known to be in the table), or -1.
__device__ __forceinline__ int64_t small_find_slot(const uint64_t* keys, uint32_t mask, int shift,
                                                   uint64_t key) {
  uint32_t slot = home_slot(key, shift);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint64_t cur = keys[slot];
    if (cur == key) return slot;
    if (cur == kEmpty) return -1;
    slot = (slot + 1) & mask;
  }
  return -1;
}
#endif

// ---------------------------------------------------------------------------
// Sorting and scanning (cg_sort.cu). Counts are read from device memory so
// that no host synchronisation is needed between steps.
// ---------------------------------------------------------------------------
// Scratch sizes (bytes) for up to `max_n` items.
size_t radix_scratch_bytes(size_t max_n);
size_t scan_scratch_bytes(size_t max_n);

// Stable LSD radix sort of keys (with optional uint32 payload) by bits
// [0, bits) of the keys, 8 bits per pass. Items: *n_dev (device). Buffers
// keys0/keys1 (and vals0/vals1) alternate; *result_in_1 tells where the sorted
// data ends up (host-known: depends only on the pass count).
cudaError_t radix_sort_u64(uint64_t* keys0, uint64_t* keys1, uint32_t* vals0, uint32_t* vals1,
                           const unsigned int* n_dev, size_t max_n, int bits, void* scratch,
                           cudaStream_t s, bool* result_in_1);

// Value order of U = min(*n_dev, max_n) rows of W = ceil(l / 64) words
// (l > 64): rows[idx_in[i]] (idx_in nullable: row i). Comparison merge sort
// on row numbers with the top 128 bits cached; k0/k1 (2 * max_n words each)
// and i0/i1 (max_n) are ping-pong buffers; *sorted_idx receives the buffer
// holding the sorted row numbers. With skip != nullptr, every kernel does
// nothing when *skip is nonzero. For l > 128 with flag != nullptr (a device
// word), the rows are sorted by the cached key alone and every short run of
// equal keys is then ordered by one warp; the full-row comparison sort runs
// only when some run is too long for that (flag records which). With scratch
// (scratch_bytes of device memory, radix_scratch_bytes(max_n) is enough) a
// bucket sort on the top bits runs first, and the merge sort only when some
// bucket is too large for it.
cudaError_t merge_sort_rows(const uint64_t* rows, int w64, int ell, const uint32_t* idx_in,
                            uint64_t* k0, uint64_t* k1, uint32_t* i0, uint32_t* i1,
                            const unsigned int* n_dev, size_t max_n, cudaStream_t s,
                            uint32_t** sorted_idx, const unsigned int* skip = nullptr,
                            unsigned int* flag = nullptr, void* scratch = nullptr,
                            size_t scratch_bytes = 0, const ulonglong2* ukeys = nullptr);

// Batch sort: the distinct vectors of many scenes sorted together, scene by
// scene (one merge sort on (scene, top 128 bits, whole vector)), then
// scattered into each scene's sorted cells, the caller's copy and, for
// l <= 64, the cell numbers in the scene's table. A scene whose table
// overflowed contributes nothing (the caller re-runs it).
struct BatchSortScene {
  DevCounters* ctr;        // n_unique (and overflow)
  uint32_t ucap;           // at most this many distinct vectors
  int w;                   // 64-bit words per vector
  int ell;
  const uint64_t* ulist;   // l <= 64: distinct vectors, insertion order
  const uint64_t* keys64;  // l > 64: vectors ...
  const uint32_t* idx;     // ... and the rows of the distinct ones
  uint64_t* cells;         // sorted cells, w words each
  uint64_t* user_cells;    // the caller's copy (64-bit words), nullable
  int64_t user_cap;        // cells
  SmallTable t;            // l <= 64: cell numbers into t.vals (t.keys nullable)
};
// Each scene is sorted in a segment of batch_sort_seg_size(ucap) positions
// (a power of two, at least 1024).
size_t batch_sort_seg_size(size_t ucap);
size_t batch_sort_bytes(size_t total_cap, int n_scenes);
// scenes: device array of n_scenes; total_cap >= the sum of their segment
// sizes, max_seg >= the largest.
cudaError_t batch_sort(const BatchSortScene* scenes, int n_scenes, size_t total_cap,
                       size_t max_seg, void* scratch, cudaStream_t s);

// Segmented key sort: many scenes' (key, value) arrays, each sorted by key
// (stable) in place, with one radix sort over all of them. Scene s holds
// min(ctr->n_unique, cap) items, none when its table overflowed (its keys were
// never written); only the low key_bits bits of a key take part.
struct SegSortScene {
  uint64_t* keys;
  uint32_t* vals;
  const DevCounters* ctr;
  uint32_t cap;
};
size_t seg_sort_bytes(size_t total_cap, int n_scenes);
// scenes: device array of n_scenes; total_cap >= the sum of their cap.
cudaError_t seg_sort(const SegSortScene* scenes, int n_scenes, size_t total_cap, int key_bits,
                     void* scratch, cudaStream_t s);

// out[i] = sum_{j<i} in[j] for i < *n_dev; *total = sum of all (device).
cudaError_t scan_exclusive_u32(const uint32_t* in, unsigned long long* out,
                               const unsigned int* n_dev, size_t max_n,
                               unsigned long long* total, void* scratch, cudaStream_t s);

// ---------------------------------------------------------------------------
// Cells and edges (cg_graph.cu).
// ---------------------------------------------------------------------------
cudaError_t launch_fill_u64(uint64_t* p, uint64_t v, size_t n, cudaStream_t s);
cudaError_t launch_zero_counters(DevCounters* c, cudaStream_t s);

// Insert stored vectors (l <= 64) into a SmallTable (dedup).
cudaError_t launch_insert_small(const void* keys, int64_t n, int word_bits, int ell,
                                const SmallTable& t, cudaStream_t s);
// vals[slot(cells[i])] = i for i < U; also records the all-ones cell.
cudaError_t launch_rank_small(const uint64_t* cells, const SmallTable& t, size_t max_n,
                              cudaStream_t s);
// Insert already-unique cells (internal rows, count ctr->n_unique) with their
// numbers; a repeated cell sets ctr->error.
cudaError_t launch_index_small(const uint64_t* cells, const SmallTable& t, size_t max_n,
                               cudaStream_t s);
// point_cell[p] = cell number of keys[p].
cudaError_t launch_point_cell_small(const void* keys, int64_t n, int word_bits, int ell,
                                    const SmallTable& t, uint32_t* point_cell, cudaStream_t s);
// Copy U cells (u64, internal) to the caller's layout when U <= cap.
cudaError_t launch_write_cells(const uint64_t* cells, int ell, int word_bits, void* out,
                               int64_t cap, const DevCounters* ctr, size_t max_n, cudaStream_t s,
                               const unsigned int* skip = nullptr);
// Load caller-layout cells into internal u64 rows; sets ctr->n_unique = n.
cudaError_t launch_load_cells(const void* cells, int64_t n, int word_bits, int ell,
                              uint64_t* out, DevCounters* ctr, cudaStream_t s);

// Sets kErrUnsorted unless the U = ctr->n_unique rows of w64 words are
// strictly ascending in value order.
cudaError_t launch_check_sorted(const uint64_t* cells, int w64, DevCounters* ctr, size_t max_n,
                                cudaStream_t s);
// For a caller's 64-bit cells used in place: sets ctr->n_unique = n, and
// kErrUnsorted / kErrHighBits unless the rows are strictly ascending and
// have no bit set at or above l.
cudaError_t launch_adopt_cells(const uint64_t* cells, int64_t n, int ell, DevCounters* ctr,
                               cudaStream_t s);
// Copies *ctr to host_ctr (mapped pinned memory, device address), then, after
// a system-wide fence, writes seq to *host_flag: a host thread that reads
// seq from the flag (with acquire ordering) sees the counters.
cudaError_t launch_publish_done(const DevCounters* ctr, DevCounters* host_ctr,
                                unsigned int* host_flag, unsigned int seq, cudaStream_t s);
// The same for several requests in one launch (one block per entry).
struct PublishEntry {
  const DevCounters* ctr;
  DevCounters* host_ctr;
  unsigned int* host_flag;
  unsigned int seq;
};
cudaError_t launch_publish_group(const PublishEntry* e, int n, cudaStream_t s);
// out[0] = U, out[1] = E, out[2] = status (CG_OK, CG_ERR_CAPACITY when a count
// exceeds its cap, CG_ERR_TIMEOUT / CG_ERR_INTERNAL on device-side failures).
cudaError_t launch_publish_counts(const DevCounters* ctr, int64_t* out, int64_t cells_cap,
                                  int64_t edges_cap, cudaStream_t s);

// Batches: the single-pass edge kernel over many scenes of l <= 64 in one
// launch (HASH lookups in each scene's table, or SORTED binary search in its
// cells). scratch: n_scenes + 2 words (chunk offsets, total, ticket).
struct SegSearchScene {
  const uint64_t* cells;  // sorted cells
  SmallTable t;           // the scene's table (HASH) and counters (t.ctr)
  unsigned long long* status;
  uint32_t* edges;
  int64_t edges_cap;
  int ell;
  uint32_t ucap;
};
cudaError_t launch_neighbors_seg_small(const SegSearchScene* scenes, int n_scenes,
                                       size_t total_chunks, bool sorted_lookup,
                                       unsigned int* scratch, cudaStream_t s);
// Batches: the clears of many l <= 64 scenes in one launch (one block each).
struct SegClear {
  uint64_t* keys;
  uint32_t* vals;  // nullable
  size_t cap;
  unsigned long long* status;
  size_t n_status;
  DevCounters* ctr;
  uint64_t* keys2 = nullptr;  // a second table (kEmpty), cap2 slots
  size_t cap2 = 0;
};
cudaError_t launch_clear_seg(const SegClear* scenes, int n_scenes, cudaStream_t s);

// Clears a build's table (kEmpty), the look-back status words and the counters.
// (A second table, table2/cap2, and an array of 32-bit words to be zeroed,
// zero32/n_zero32, may be cleared in the same launch.)
cudaError_t launch_clear_build(uint64_t* table, size_t cap, unsigned long long* status,
                               size_t n_status, DevCounters* ctr, cudaStream_t s,
                               uint64_t* table2 = nullptr, size_t cap2 = 0,
                               uint32_t* zero32 = nullptr, size_t n_zero32 = 0);

// Sorts U = min(*n_dev, max_n) distinct vectors of W = ceil(l/64) <= 4 words
// inside one thread-block cluster (keys held in distributed shared memory),
// then writes the sorted cells, the caller's copy (when U <= user_cap, in
// word_bits words) and, for l <= 64 with a table, the cell numbers into the
// table. Row i of the input is in[rows[i]] (rows nullable: in[i]). Sets *done
// to false when max_n or l is too large for one cluster.
struct ClusterSortOut {
  uint64_t* cells;
  void* user_cells;
  int64_t user_cap;
  int word_bits;
  int ell;
  SmallTable t;  // t.keys == nullptr: no numbering
  DevCounters* ctr;
};
// *done: the cluster sort certainly handles all vectors (max_n fits). When it
// does not and *tried is set, the cluster kernel was launched at its full
// capacity anyway: it sorts when the actual count fits and records the
// outcome in o.ctr->sorted, which the fallback steps then read (skip flag).
cudaError_t cluster_sort(const uint64_t* in, const uint32_t* rows, const unsigned int* n_dev,
                         size_t max_n, int ell, const ClusterSortOut& o, cudaStream_t s,
                         bool* done, bool* tried = nullptr);

// Steps 3-4 in one kernel for l <= 64: hit search, scan with decoupled
// look-back (status: ceil(max_n / 32) words, zeroed) and edge output.
size_t ne_status_words(size_t max_n);
cudaError_t launch_neighbors_emit_small(const uint64_t* cells, const SmallTable& t, int ell,
                                        int strategy, unsigned long long* status,
                                        uint32_t* edges, int64_t edges_cap, size_t max_n,
                                        cudaStream_t s);

// Neighbour search. masks: [U][ceil(l/32)] hit bits; counts: [U].
cudaError_t launch_neighbors_small(const uint64_t* cells, const SmallTable& t, int ell,
                                   int strategy, uint32_t* masks, uint32_t* counts,
                                   size_t max_n, cudaStream_t s);
cudaError_t launch_emit_small(const uint64_t* cells, const SmallTable& t, int ell, int strategy,
                              const uint32_t* masks, const unsigned long long* offsets,
                              uint32_t* edges, int64_t edges_cap, size_t max_n, cudaStream_t s);

// Vectors of l > 64 bits (W = ceil(l/64) words).
struct WideTable {
  uint64_t* slots;  // [cap]: (tag << 32) | index, kEmpty = free
  uint32_t mask;
  uint32_t* ulist;  // [ucap] representative input rows, insertion order
  uint32_t ucap;
  DevCounters* ctr;
  // Optional (insert only): the top 128 bits of each representative, in
  // ulist order, and counts of the representatives per value of their top
  // bucket_bits bits (the bucket sort's histogram, cleared beforehand).
  ulonglong2* ukeys = nullptr;
  uint32_t* bucket_count = nullptr;
  int bucket_bits = 0;
  int ell = 0;
};
cudaError_t launch_insert_wide(const uint64_t* keys, int64_t n, int w64, const WideTable& t,
                               cudaStream_t s);
// Batches: the dedup inserts of many scenes of l > 64 in one launch (their
// vectors written by launch_pack_store_seg); p0 numbers the points of all
// scenes in order.
struct SegInsertWide {
  const uint64_t* keys64;
  int64_t n;
  int w;
  WideTable t;
  uint64_t p0;
};
cudaError_t launch_insert_wide_seg(const SegInsertWide* scenes, int n_scenes,
                                   uint64_t total_points, cudaStream_t s);
// Sort representatives by value: idx0/idx1 permuted, kw0/kw1 word scratch.
cudaError_t sort_wide(const uint64_t* keys, int w64, int ell, uint32_t* idx0, uint32_t* idx1,
                      uint64_t* kw0, uint64_t* kw1, const unsigned int* n_dev, size_t max_n,
                      void* scratch, cudaStream_t s, uint32_t** sorted_idx,
                      const unsigned int* skip = nullptr, unsigned int* flag = nullptr,
                      const void* ukeys = nullptr);
// The bucket sort inside sort_wide / merge_sort_rows (scratch of
// radix_scratch_bytes(max_n) bytes): its bucket bits and its count array,
// which an insert can fill (WideTable::bucket_count, cleared first) together
// with the top-128-bit keys in ulist order (WideTable::ukeys, passed on as
// ukeys) so that the sort reads neither from the rows.
int bucket_sort_bits(size_t max_n);
uint32_t* bucket_sort_counts(void* scratch, size_t max_n);
// out_cap >= 0: out is a caller's buffer of that many rows, written only when
// all U rows fit.
cudaError_t launch_gather_rows(const uint64_t* keys, int w64, const uint32_t* idx,
                               const unsigned int* n_dev, size_t max_n, uint64_t* out,
                               cudaStream_t s, const unsigned int* skip = nullptr,
                               int64_t out_cap = -1);
cudaError_t launch_rank_by_row(const uint32_t* idx, const unsigned int* n_dev, size_t max_n,
                               uint32_t* rank_by_row, cudaStream_t s);
cudaError_t launch_point_cell_wide(const uint64_t* keys, int64_t n, int w64, const WideTable& t,
                                   const uint32_t* rank_by_row, uint32_t* point_cell,
                                   cudaStream_t s);
// Fingerprint table over sorted cells: fp[i] and slots (tag, i).
cudaError_t launch_index_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                              uint64_t* fp, size_t max_n, cudaStream_t s);
cudaError_t launch_neighbors_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                                  const uint64_t* fp, int strategy, uint32_t* masks,
                                  uint32_t* counts, size_t max_n, cudaStream_t s);
cudaError_t launch_emit_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                             const uint64_t* fp, int strategy, const uint32_t* masks,
                             const unsigned long long* offsets, uint32_t* edges,
                             int64_t edges_cap, size_t max_n, cudaStream_t s);

// Single-pass steps 3-4 for W-word vectors (status: ne_status_words(max_n)
// zeroed words); needs the fingerprint index (launch_index_wide) for HASH.
cudaError_t launch_neighbors_emit_wide(const uint64_t* cells, int w64, int ell, const WideTable& t,
                                       const uint64_t* fp, int strategy,
                                       unsigned long long* status, uint32_t* edges,
                                       int64_t edges_cap, size_t max_n, cudaStream_t s);

// PIVOT strategy (cg_pivot.cu): keys of h distances to pivot cells, sorted
// (radix_sort_u64 over pivot_sort_bits bits), bucket table, then the
// neighbour search and edge output.
int pivot_max_h(int ell);
int pivot_sort_bits(int ell, int h);
cudaError_t launch_pivot_keys(const uint64_t* cells, int w64, int ell, int h,
                              const DevCounters* ctr, size_t max_n, uint64_t* key_by_cell,
                              uint64_t* skeys, uint32_t* sidx, cudaStream_t s);
// Bucket table of pivot_table_slots(max_n) 16-byte entries (filled with
// all-ones words before use).
size_t pivot_table_slots(size_t max_n);
cudaError_t launch_pivot_index(const uint64_t* skeys, const DevCounters* ctr, size_t max_n,
                               void* table, size_t tcap, DevCounters* wctr, cudaStream_t s);
// Search + scan + edge output (ctr->n_edges = E); hbuf: pivot_hit_words(max_n)
// words; scan: scan_scratch_bytes(max_n).
size_t pivot_hit_words(size_t max_n);

// Breadth-first search on G_X (cg_bfs.cu).
struct BfsCounters {
  unsigned int frontier[3];  // rotating frontier sizes (level d reads [d % 3])
  unsigned int error;        // 1: an edge with an endpoint >= n or a self-loop;
                             // 2: a grid-barrier wait ran out (single-launch search)
  unsigned int n;            // number of cells (device copy, for the scan)
  unsigned int reached;      // cells with a distance
  unsigned int depth;        // last level with a non-empty frontier
  unsigned int bar_count;    // grid barrier of the single-launch search:
  unsigned int bar_gen;      //   arrivals, generation
  unsigned int pad[3];
};
struct BfsWs {
  uint32_t* deg;              // n
  unsigned long long* off;    // n (row starts)
  uint32_t* cur;              // n (fill cursors)
  uint32_t* adj;              // 2 E
  uint32_t* f0;               // n
  uint32_t* f1;               // n
  BfsCounters* ctr;
  unsigned long long* total;  // 2 E
  void* scan;                 // scan_scratch_bytes(n)
};
cudaError_t launch_bfs_adjacency(const uint32_t* edges, int64_t n_edges, uint32_t n,
                                 const BfsWs& w, cudaStream_t s);
cudaError_t launch_bfs_init(int32_t* dist, int32_t* parent, uint32_t n, uint32_t source,
                            const BfsWs& w, cudaStream_t s);
// Enqueues levels first .. first + count - 1.
cudaError_t launch_bfs_levels(int first, int count, uint32_t n, int32_t* dist, int32_t* parent,
                              const BfsWs& w, cudaStream_t s);
// All levels in one cooperative launch (grid barriers between levels). Sets
// *launched = false, with nothing enqueued, when the device or the launch
// does not allow it (the caller then enqueues levels).
cudaError_t launch_bfs_single(uint32_t n, int32_t* dist, int32_t* parent, const BfsWs& w,
                              cudaStream_t s, bool* launched);

// ALLPAIRS strategy (cg_pivot.cu): keys from launch_pivot_keys, then every
// pair i < j tested; at most kAllPairsMaxCells cells.
constexpr int64_t kAllPairsMaxCells = int64_t(1) << 18;
cudaError_t launch_allpairs_edges(const uint64_t* cells, int w64, int ell, int h,
                                  DevCounters* ctr, size_t max_n, const uint64_t* key_by_cell,
                                  uint32_t* counts, uint32_t* hbuf, unsigned long long* offsets,
                                  uint32_t* fill, void* scan, uint32_t* edges, int64_t edges_cap,
                                  cudaStream_t s);

// HALVES strategy (cg_pivot.cu): the l bits split at s = halves_split(l);
// keys, a stable sort of (L key, cell) over halves_sort_bits(l) bits, then the
// search and edge output. Uses the PIVOT workspace: hkey in key_by_cell, the
// folds fl and fh in the bucket-table memory, sfh in the sort's spare key
// buffer.
int halves_split(int ell);
int halves_sort_bits(int ell);
// adopt_n >= 0 (2 <= w64 <= 16 only): cells are a caller's rows used in place;
// U = adopt_n is written to ctr->n_unique and the rows are checked as
// launch_adopt_cells checks them, in the same pass.
cudaError_t launch_halves_keys(const uint64_t* cells, int w64, int ell, DevCounters* ctr,
                               size_t max_n, uint64_t* hkey, uint64_t* fl, uint64_t* fh,
                               uint64_t* lkey, uint32_t* idx, cudaStream_t s,
                               int64_t adopt_n = -1);
// Whether launch_halves_keys can check adopted rows of w64 words itself.
inline bool halves_keys_can_adopt(int w64) { return w64 >= 2 && w64 <= 16; }
cudaError_t launch_halves_edges(const uint64_t* cells, int w64, int ell, DevCounters* ctr,
                                size_t max_n, const uint64_t* hkey, const uint64_t* fl,
                                const uint64_t* fh, const uint64_t* skey, const uint32_t* sidx,
                                uint64_t* sfh, uint32_t* counts, uint32_t* hbuf,
                                unsigned long long* offsets, uint32_t* fill, void* scan,
                                uint32_t* edges, int64_t edges_cap, cudaStream_t s);
cudaError_t launch_pivot_edges(const uint64_t* cells, int w64, int ell, int h, DevCounters* ctr,
                               size_t max_n, const uint64_t* key_by_cell, const uint32_t* sidx,
                               const void* table, size_t tcap, uint32_t* counts, uint32_t* hbuf,
                               unsigned long long* offsets, uint32_t* fill, void* scan,
                               uint32_t* edges, int64_t edges_cap, cudaStream_t s);

// TREE strategy (cg_tree.cu): the 2^r-ary search tree of §3.2 (r = 8) over
// the sorted cells, digits taken from the most significant end of the value
// order (digit h = bits [max(0, l - 8 (h + 1)), l - 8 h)). Leaf-valued (a node
// whose range holds one cell is a leaf; the lookup then compares the whole
// vector) and with single-child chains contracted: an internal node records
// the level its children branch on. Children of a node are consecutive node
// ids in digit order; bm marks the digits present.
struct TreeNode {
  uint32_t bm[8];
  uint32_t first;  // id of the first child
  uint32_t lo;     // first cell of the node's range
  uint32_t cnt;    // cells in the range (1: leaf of cell lo)
  uint32_t lv;     // branching level (internal nodes)
};
static_assert(sizeof(TreeNode) == 48, "TreeNode layout");

#ifdef __CUDACC__
__device__ __forceinline__ int tree_levels(int ell) { return (ell + 7) >> 3; }
// [lo, hi) bit range of digit h.
__device__ __forceinline__ void tree_digit_bits(int ell, int h, int* lo, int* hi) {
  *hi = ell - 8 * h;
  *lo = *hi > 8 ? *hi - 8 : 0;
}
// Child of node nd for digit v, or -1.
__device__ __forceinline__ int64_t tree_child(const TreeNode& nd, uint32_t v) {
  const uint32_t wv = nd.bm[v >> 5];
  if (!((wv >> (v & 31)) & 1u)) return -1;
  uint32_t rank = __popc(wv & ((1u << (v & 31)) - 1u));
  for (uint32_t q = 0; q < (v >> 5); ++q) rank += __popc(nd.bm[q]);
  return int64_t(nd.first) + rank;
}
#endif

// Workspace of the tree build for up to max_n cells (bytes), and the build
// itself: nodes (tree_node_capacity(max_n) entries) end up holding the tree,
// node 0 the root.
size_t tree_node_capacity(size_t max_n);
size_t tree_scratch_bytes(size_t max_n);
cudaError_t launch_tree_build(const uint64_t* cells, int w64, int ell, const DevCounters* ctr,
                              size_t max_n, TreeNode* nodes, void* scratch, cudaStream_t s);
// Steps 3-4 with TREE lookups: single pass (like launch_neighbors_emit_*)
// when neighbors_emit_tree_fits(w64, l), else hit masks + scan + emit.
bool neighbors_emit_tree_fits(int w64, int ell);
cudaError_t launch_neighbors_tree_masks(const uint64_t* cells, int w64, int ell,
                                        const TreeNode* nodes, DevCounters* ctr, uint32_t* masks,
                                        uint32_t* counts, size_t max_n, cudaStream_t s);
cudaError_t launch_emit_tree(const uint64_t* cells, int w64, int ell, const TreeNode* nodes,
                             DevCounters* ctr, const uint32_t* masks,
                             const unsigned long long* offsets, uint32_t* edges,
                             int64_t edges_cap, size_t max_n, cudaStream_t s);
cudaError_t launch_neighbors_emit_tree(const uint64_t* cells, int w64, int ell,
                                       const TreeNode* nodes, DevCounters* ctr,
                                       unsigned long long* status, uint32_t* edges,
                                       int64_t edges_cap, size_t max_n, cudaStream_t s);

// Batch gather: per scene, its counters, internal cells (w words per cell,
// up to ucap cells) and internal edges (up to ecap).
struct BatchEntry {
  const DevCounters* ctr;
  const uint64_t* cells;
  const uint32_t* edges;
  uint32_t w;
  uint32_t ucap;
  unsigned long long ecap;
};
// cells_off / edges_off: n + 1 words each; *ok = all scenes fitted.
cudaError_t launch_batch_gather(const BatchEntry* tab, int n, long long* cells_off,
                                long long* edges_off, int* ok, uint64_t* out_cells,
                                int64_t cells_cap, uint32_t* out_edges, int64_t edges_cap,
                                cudaStream_t s);

// Convert caller-layout keys ([n][W] of word_bits) to internal u64 rows.
cudaError_t launch_keys_to_u64(const void* keys, int64_t n, int word_bits, int ell,
                               uint64_t* out, cudaStream_t s);

}  // namespace cg
