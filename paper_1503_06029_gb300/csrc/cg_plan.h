// Host-side planning and enqueueing of one scene's build (steps 1-4), shared by
// the single-scene, batch and server entry points.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/cellgraph.h"
#include "cg_internal.cuh"

namespace cg {

// Library defaults of the tunables: HASH lookups, 4 pivots, fp32 sign kernel.
// The library's default setting for bucket b (CG_TUNE_BUCKETS): HASH for
// l <= 128, HALVES above (measured faster from l = 200 on: l * U probes grow
// with l, HALVES' work does not).
cg_tune_params default_tune(int bucket);
// The lookup strategy CG_STRATEGY_AUTO stands for at length l.
int auto_strategy(int ell);
// Valid, clamped copy of p for vectors of l bits (h within 1..pivot_max_h(l)).
cg_tune_params sanitize_tune(const cg_tune_params& p, int ell);

// One scene's build: sizes and strategy.
struct ScenePlan {
  int64_t n;
  int ell;
  size_t cap;   // table slots (power of two)
  size_t ucap;  // distinct-vector capacity
  bool small;   // l <= 64
  bool single;  // wide, single-pass neighbour kernel and cluster sort
  int grid_bits;  // log2 cells of the sign step's box grid (0: none)
  cg_tune_params tp;
};

ScenePlan plan_scene(int64_t n, int ell, size_t cap, const cg_tune_params& tp);

// Device workspace of one scene (without its counters and outputs).
size_t scene_ws_bytes(const ScenePlan& p);

// First table capacity tried for a scene of n points, d dimensions and l
// constraints (from the arrangement bound), and the capacity that always fits.
size_t initial_cap(int64_t n, int d, int ell);
size_t full_cap(int64_t n);

// Points that arrive in pieces: piece k (points [k * per, min(n, (k + 1) *
// per))) may be read once `ready[k]` has completed. The sign + dedup step of
// vectors of l <= 64 bits then runs one launch per piece into the same
// table; other steps wait for all pieces.
struct PackPieces {
  int count;
  int64_t per;
  const cudaEvent_t* ready;
};

// Enqueues one scene's build into workspace `ws` with counters at `ctr`;
// nothing is read back. Cells go to `cells` (word_bits words, when
// U <= cells_cap), edges to `edges` (up to edges_cap). ctx (nullable) only
// receives stage-timing marks.
// Phases: the whole build, or (for batches whose sort runs across scenes)
// everything up to the dedup insert, and everything after the sort.
// kPhaseSearchKeys / kPhaseSearchRest split kPhaseSearch of a PIVOT or HALVES
// scene around a batch-wide sort of its (key, cell) pairs (seg_sort).
enum ScenePhase {
  kPhaseAll = 0,
  kPhaseInsert = 1,
  kPhaseSearch = 2,
  kPhaseSearchKeys = 3,
  kPhaseSearchRest = 4
};

cg_status enqueue_scene(cg_ctx* ctx, char* ws, DevCounters* ctr, const ScenePlan& plan,
                        const PackArgs& pa, int word_bits, void* cells, int64_t cells_cap,
                        uint32_t* edges, int64_t edges_cap, cudaStream_t s,
                        const PackPieces* pieces = nullptr, int phase = kPhaseAll);

// Whether a scene can be split into kPhaseInsert / kPhaseSearch around a
// batch sort, and its sort descriptor (device pointers into workspace ws,
// counters ctr, the caller's cells user_cells of capacity user_cap).
bool scene_batch_sortable(const ScenePlan& plan);
BatchSortScene scene_sort_desc(char* ws, DevCounters* ctr, const ScenePlan& plan,
                               uint64_t* user_cells, int64_t user_cap);

// Descriptors of a scene of l <= 64 (plan.small) for the segmented kernels:
// its clear, its sign + insert (tiles numbered from tile0 in its launch), and
// its single-pass search (HASH or SORTED; edges to `edges`, at most
// edges_cap). Null outputs are skipped.
void scene_small_descs(char* ws, DevCounters* ctr, const ScenePlan& plan, const PackArgs& pa,
                       uint64_t tile0, uint32_t* edges, int64_t edges_cap, SegClear* clr,
                       SegPackScene* pk, SegSearchScene* se);

// Whether a strategy sorts (key, cell) pairs (PIVOT, HALVES), the key width of
// a scene's pairs, and the descriptor of those pairs in workspace ws.
bool keysort_strategy(int strategy);
int scene_key_bits(const ScenePlan& plan);
SegSortScene scene_keysort_desc(char* ws, DevCounters* ctr, const ScenePlan& plan);

}  // namespace cg
