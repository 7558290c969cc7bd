/*
 * cellgraph.h -- C-ABI of libcellgraph.so, a CUDA (sm_103a) implementation of
 * the cell-graph construction of "Massively Parallel Construction of the Cell
 * Graph" (Kaczmarski, Rzazewski, Wolant).
 *
 * The method, in the paper's terms:
 *   - a scene is a system of l constraints c_0..c_{l-1}; a sampled point P is
 *     represented by the l-bit vector v_P whose bit i is 1 iff P satisfies c_i
 *     (§2.1, Figure 1). Here every constraint is the closed half-space
 *     a_i . p >= b_i with integer a_i, p, b_i, evaluated exactly;
 *   - the cells are the distinct vectors (§2.1); the multiset X of sampled
 *     vectors is sorted and its duplicates removed (§3.2);
 *   - the cell graph G_X has an edge between two cells iff their Hamming
 *     distance is exactly 1 (§2.2); each unordered pair is reported once, even
 *     when X holds duplicates (§2.2). The search flips each bit of each cell and
 *     looks the result up (Algorithm 4).
 *
 * Conventions shared by every call:
 *   - Packing: bit i of a vector lives in word i / B at bit position i % B,
 *     with B = word_bits (32 or 64). A vector takes W = ceil(l / B) words; the
 *     bits >= l of the last word are zero. Arrays of vectors are row-major
 *     [count][W].
 *   - Order: vectors compare as the unsigned integers sum_i x(i) 2^i (the last
 *     word is the most significant). Cells are numbered 0..U-1 in that order.
 *   - Edges: pairs (i, j) of cell numbers with i < j, stored as uint32[E][2], in
 *     lexicographic (i, j) order. Every edge is found from its endpoint i, whose
 *     bit k is 0 while j's is 1.
 *   - Memory: every array argument is DEVICE memory owned by the caller, except
 *     where a parameter says "host". The library never frees caller memory.
 *   - Streams: work is enqueued on `stream` (a cudaStream_t; 0 is the legacy
 *     default stream). Calls that return counts through host pointers wait for
 *     their own work on that stream before returning.
 *   - Capacities: when an output array is too small the call returns
 *     CG_ERR_CAPACITY, still writes the required count(s), and writes nothing
 *     past the given capacity.
 *   - Errors: every call returns a cg_status; cg_last_error() gives a message
 *     for the calling thread's last failure. Invalid arguments are rejected
 *     before any work is enqueued.
 *   - Sizes: n < 2^32 - 1 points/vectors (cell numbers are uint32), 1 <= d <= 4,
 *     1 <= l <= 4096. Coordinates, normals (int32) and offsets (int64) may take
 *     any value of their type: the sign tests are exact.
 */
#ifndef CELLGRAPH_H
#define CELLGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cg_status;
#define CG_OK 0
#define CG_ERR_INVALID_ARG 1 /* bad pointer, size, word_bits, strategy, unsorted
                                cells given to cg_neighbors_h1, ... */
#define CG_ERR_RANGE 2       /* reserved: never returned, every int32 coordinate and
                                normal and int64 offset is evaluated exactly */
#define CG_ERR_CAPACITY 3    /* an output array is too small; counts were written */
#define CG_ERR_OOM 4         /* a library-owned allocation failed */
#define CG_ERR_CUDA 5        /* a CUDA runtime call or kernel launch failed */
#define CG_ERR_TIMEOUT 6     /* a bounded device-side wait ran out */
#define CG_ERR_INTERNAL 7    /* a device-side consistency check failed */

/* Lookup strategies for the neighbour search (cg_neighbors_h1). */
#define CG_STRATEGY_AUTO 0   /* library choice: HASH for l <= 128, HALVES above */
#define CG_STRATEGY_HASH 1   /* open-addressing table keyed on the vector (l <= 64)
                                or on a GF(2)-linear 64-bit fingerprint (l > 64);
                                every candidate is verified against the full vector */
#define CG_STRATEGY_SORTED 2 /* binary search in the sorted cell array */
#define CG_STRATEGY_PIVOT 3  /* distance-to-pivot bucketing by inequality (⋆) of §3.1:
                                cells are grouped by their Hamming distances to h
                                pivot cells, and only the 2^h buckets whose
                                distances differ by +-1 in every coordinate are
                                compared, word by word (XOR + popcount) */
#define CG_STRATEGY_TREE 4   /* the 2^r-ary search tree of §3.2 (Algorithms 3-4),
                                r = 8, built level by level over the sorted
                                cells and walked once per flipped bit */
#define CG_STRATEGY_HALVES 5 /* the O(n l) search named in §6, as two-part
                                multi-index hashing: with the bits split at
                                s = floor(l/2), partners that differ below s
                                share the high part (contiguous in the sorted
                                cells), partners that differ above s share the
                                low part (grouped by one stable sort); each
                                group is compared within itself */
#define CG_STRATEGY_ALLPAIRS 6 /* the heuristic of §3.1 in its all-pairs form
                                (Algorithms 1-2): every pair i < j whose
                                distances to h pivot cells pass inequality (⋆)
                                is compared; quadratic, so cg_neighbors_h1
                                accepts it for at most 2^18 cells (else
                                CG_ERR_INVALID_ARG) and tuning does not offer it */

/* Message describing the calling thread's last failed call ("" if none). */
const char* cg_last_error(void);

/* Library version string. */
const char* cg_version(void);

/* Number of kernels this library has launched in this process (all devices,
 * all threads). Host-side counter; used to report launches per step. */
uint64_t cg_launch_count(void);

/* Test control of the library's bounded device-side waits (the paper has no
 * counterpart): every wait on another block's progress -- the edge kernels'
 * look-back for their output offset, the BFS grid barrier, the tensor-core
 * sign kernel's wait for its MMA -- gives up after a fixed number of polls,
 * sets an error bit and returns, so a wait that
 * can never end yields CG_ERR_TIMEOUT instead of a hung GPU. cg_set_wait_limit
 * lowers that number for kernels launched afterwards by any thread of the
 * process: `polls` = 0 makes every such wait give up before its first poll
 * (the call then returns CG_ERR_TIMEOUT whenever the wait was needed);
 * `polls` < 0 restores the built-in limits. Outputs of a call that timed out
 * are unspecified (but stay within their capacities). A CUDA graph the library
 * captured (repeated cg_build / cg_build_batch calls) keeps the limit it was
 * captured with. For tests only. */
cg_status cg_set_wait_limit(int64_t polls);

/* ---------------------------------------------------------------------------
 * Step 1 -- sign vectors (§2.1, Figure 1).
 * keys[p] = packed [a_i . pts[p] >= b_i] for i = 0..l-1, evaluated exactly.
 *   pts   int32[n][d] row-major, device.
 *   a     int32[l][d] row-major (constraint normals), device.
 *   b     int64[l] (constraint offsets), device.
 *   keys  [n][W] words of word_bits bits, device, written entirely.
 * n = 0 is allowed (nothing is written). No workspace; asynchronous.
 * ------------------------------------------------------------------------- */
cg_status cg_pack_signs(const int32_t* pts, int64_t n, int d, const int32_t* a,
                        const int64_t* b, int ell, int word_bits, void* keys,
                        void* stream);

/* ---------------------------------------------------------------------------
 * Step 1 for curved boundaries -- sign vectors of quadric constraints (§2.1:
 * the constraints are inequalities whose boundaries partition the space into
 * cells; the paper's figure uses lines, motion-planning scenes need curves).
 * keys[p] = packed [ sum_{j<=k} q_i,jk p_j p_k + a_i . pts[p] >= b_i ] for
 * i = 0..l-1, evaluated exactly for every int32 input and int64 offset.
 *   pts   int32[n][d] row-major, device.
 *   q     int32[l][d(d+1)/2] row-major, device: coefficient of the monomial
 *         p_j p_k (j <= k), in the order (0,0), (0,1), ..., (0,d-1), (1,1),
 *         ..., (d-1,d-1). A sphere |p - c|^2 >= r^2 is q = 1 on the squares,
 *         0 elsewhere, a = -2c, b = r^2 - |c|^2.
 *   a     int32[l][d] row-major, device.    b  int64[l], device.
 *   keys  [n][W] words of word_bits bits, device, written entirely.
 * 1 <= d <= 4, 1 <= l <= 4096. n = 0 is allowed. No workspace; asynchronous.
 * The keys feed cg_dedup_cells and cg_neighbors_h1 unchanged.
 * ------------------------------------------------------------------------- */
cg_status cg_pack_signs_quadric(const int32_t* pts, int64_t n, int d, const int32_t* q,
                                const int32_t* a, const int64_t* b, int ell, int word_bits,
                                void* keys, void* stream);

/* ---------------------------------------------------------------------------
 * Step 2 -- cells: sort the multiset of vectors and remove duplicates (§3.2).
 *   keys        [n][W] words (word_bits), device, read only.
 *               Bits at or above l in a key are ignored.
 *   cells       [cells_cap][W] words, device: the U distinct vectors in order.
 *   n_cells     host: receives U.
 *   point_cell  nullable, uint32[n], device: cell number of every input vector.
 *   ws          device workspace of *ws_bytes bytes. With ws == NULL the call
 *               only writes the required size to *ws_bytes and returns.
 * Blocks until the work on `stream` is done (U is returned through a host
 * pointer). U > cells_cap gives CG_ERR_CAPACITY with *n_cells = U.
 * ------------------------------------------------------------------------- */
cg_status cg_dedup_cells(const void* keys, int64_t n, int ell, int word_bits, void* cells,
                         int64_t cells_cap, int64_t* n_cells, uint32_t* point_cell,
                         void* ws, size_t* ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Steps 3-4 -- Hamming-1 neighbour search and edge compaction (§2.2,
 * Algorithm 4): for every cell i and every bit k with x_i(k) = 0, the vector
 * x_i with bit k set is looked up among the cells; each hit j gives edge (i, j).
 *   cells      [n_cells][W] words, device: sorted ascending and unique (the
 *              output of cg_dedup_cells), bits at or above l zero; other
 *              input is detected on the device and gives CG_ERR_INVALID_ARG.
 *              With word_bits = 64 and l > 64 the rows are read in place
 *              (never written); otherwise they are first converted into the
 *              workspace.
 *   edges      uint32[edges_cap][2], device.
 *   n_edges    host: receives E.
 *   strategy   CG_STRATEGY_* (PIVOT and ALLPAIRS use h = 4 pivots, or the
 *              value of the environment variable CG_PIVOTS when it is set).
 *   ws, ws_bytes  as for cg_dedup_cells.
 * Blocks until done. E > edges_cap gives CG_ERR_CAPACITY with *n_edges = E.
 * ------------------------------------------------------------------------- */
cg_status cg_neighbors_h1(const void* cells, int64_t n_cells, int ell, int word_bits,
                          uint32_t* edges, int64_t edges_cap, int64_t* n_edges, int strategy,
                          void* ws, size_t* ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Context: owns a device memory pool that grows on demand, the pinned host
 * words used to return counts, and the table-size hints learned from earlier
 * calls. One context serves one device; calls on one context must not overlap
 * (use one context per host thread).
 * ------------------------------------------------------------------------- */
typedef struct cg_ctx cg_ctx;

/* Creates a context on `device` (a CUDA device ordinal). */
cg_status cg_ctx_create(cg_ctx** out, int device);
/* Frees the context and its pool. Waits for nothing; the caller must make
 * sure no work that uses the pool is still running. */
cg_status cg_ctx_destroy(cg_ctx* ctx);
/* Bytes of device memory the context currently holds. */
cg_status cg_ctx_pool_bytes(const cg_ctx* ctx, size_t* bytes);

/* Stage timing: with timing enabled, cg_build records CUDA events on its
 * stream between its stages and, once the build has finished, adds each
 * stage's duration to a per-stage total. cg_ctx_set_timing resets the totals.
 * cg_ctx_stage_times returns the number of stages in *n, the number of timed
 * builds in *builds (nullable) and, for the first `cap` stages, the total ms
 * (nullable) and the stage names (nullable; static strings owned by the
 * library). The stage "pack_dedup" holds exactly the fused sign+dedup kernel. */
cg_status cg_ctx_set_timing(cg_ctx* ctx, int enable);
cg_status cg_ctx_stage_times(cg_ctx* ctx, double* ms, const char** names, int cap, int* n,
                             int64_t* builds);

/* ---------------------------------------------------------------------------
 * Tuning. The paper's tunables are the pivot count h of the heuristic and the
 * digit width of the tree (§3, §5); here a context keeps, per bucket of l,
 * the lookup strategy of the neighbour search, the pivot count for PIVOT and
 * the sign kernel, and uses them for cg_build and cg_build_batch (AUTO in
 * cg_neighbors_h1 uses the library defaults). Every setting gives the same
 * output; only the speed differs.
 * Buckets: 0: l <= 16, 1: <= 32, 2: <= 64, 3: <= 128, 4: <= 256, 5: <= 1024,
 * 6: <= 4096.
 * Defaults: HASH for l <= 128 and HALVES above (the AUTO choice), h = 4, the
 * fp32 sign kernel.
 * ------------------------------------------------------------------------- */
#define CG_TUNE_BUCKETS 7
typedef struct cg_tune_params {
  int strategy;    /* CG_STRATEGY_HASH, _SORTED, _PIVOT, _TREE or _HALVES */
  int pivots;      /* h for PIVOT: 1 <= h <= min(8, 64 / bits(l)) (clamped) */
  int sign_kernel; /* 0: the library's choice of the fp32 forms below: 2
                         for l <= 64, n >= 2^18 and points in device memory,
                         else 3;
                      1: tensor cores (tcgen05, l <= 64 only; ignored above);
                      2: fp32 FMA filter with exact fallback behind a box grid
                         over the points (l <= 64: each point tests only the
                         constraints that cross its grid cell);
                      3: fp32 FMA filter with exact fallback on every
                         constraint (also what points read in place from host
                         memory by cg_build_host get under 0 or 2) */
} cg_tune_params;

int cg_tune_bucket(int ell); /* bucket of l, or -1 when l is out of range */
cg_status cg_ctx_tune_get(const cg_ctx* ctx, int bucket, cg_tune_params* out);
cg_status cg_ctx_tune_set(cg_ctx* ctx, int bucket, const cg_tune_params* p);


/* ---------------------------------------------------------------------------
 * Steps 1-4 for one scene: points -> cells -> edges (§2.1, §3.2, §2.2,
 * Algorithm 4), with the vectors never written to memory when l <= 64.
 *   pts, a, b   as for cg_pack_signs (device).
 *   cells       [cells_cap][W] words (word_bits), device.
 *   edges       uint32[edges_cap][2], device.
 *   n_cells, n_edges   host: receive U and E.
 * Blocks until done. Returns CG_ERR_CAPACITY (with both counts written) when
 * either output is too small; nothing is written past a capacity.
 * ------------------------------------------------------------------------- */
cg_status cg_build(cg_ctx* ctx, const int32_t* pts, int64_t n, int d, const int32_t* a,
                   const int64_t* b, int ell, int word_bits, void* cells, int64_t cells_cap,
                   int64_t* n_cells, uint32_t* edges, int64_t edges_cap, int64_t* n_edges,
                   void* stream);

/* Same as cg_build, but nothing waits and nothing is read back: the build is
 * enqueued on `stream`, followed by a kernel that writes counts[0] = U,
 * counts[1] = E and counts[2] = a status (CG_OK; CG_ERR_CAPACITY when U >
 * cells_cap or E > edges_cap, with nothing written past either cap;
 * CG_ERR_INTERNAL when the dedup table overflowed its first size guess -- run
 * cg_build once to grow it -- or a device check failed; CG_ERR_TIMEOUT).
 * counts: device int64[3]. The enqueued work can be captured into a CUDA
 * graph by the caller; a call that has to grow the context's pool allocates,
 * so make the first call with a given size outside stream capture. Calls on
 * one context must be ordered on one stream (they share its pool). */
cg_status cg_build_dev(cg_ctx* ctx, const int32_t* pts, int64_t n, int d, const int32_t* a,
                       const int64_t* b, int ell, int word_bits, void* cells, int64_t cells_cap,
                       uint32_t* edges, int64_t edges_cap, int64_t* counts, void* stream);

/* Same as cg_build with every array in HOST memory (pinned or pageable): the
 * call copies the inputs to the context's device pool, builds, and copies the
 * cells and edges back. Blocks until the copies are done. Points in pinned
 * host memory are read by the sign kernel in place, over the host link,
 * overlapping the transfer with the arithmetic. The environment variable
 * CG_HOST_INPUT=pieces copies them in pieces on a second stream instead (each
 * piece processed as it arrives), CG_HOST_INPUT=copy in one piece first. */
cg_status cg_build_host(cg_ctx* ctx, const int32_t* pts, int64_t n, int d, const int32_t* a,
                        const int64_t* b, int ell, int word_bits, void* cells,
                        int64_t cells_cap, int64_t* n_cells, uint32_t* edges,
                        int64_t edges_cap, int64_t* n_edges, void* stream);

/* ---------------------------------------------------------------------------
 * Batched build of many independent scenes (§2.1-§2.2 per scene; the paper
 * treats one scene at a time). All scenes are enqueued without host
 * synchronisation on a pool of streams (each scene's steps 1-4 on one stream,
 * scenes running concurrently), their results are gathered into contiguous
 * outputs by device-side offsets, and all counts are read back once. A batch
 * repeated with the same scenes and outputs is replayed from a captured CUDA
 * graph. Cells use 64-bit words (W_s = ceil(l_s / 64) words per cell); edges
 * hold scene-local cell numbers.
 *   scenes     host array of n_scenes descriptors (device arrays inside).
 *   out->cells       device, capacity out->cells_cap 64-bit words: the cells
 *                    of scene 0, then scene 1, ...
 *   out->edges       device, capacity out->edges_cap edges: scene after scene.
 *   out->n_cells, out->n_edges     host int64[n_scenes]: U_s and E_s.
 *   out->cells_offset, out->edges_offset  host int64[n_scenes + 1], nullable:
 *                    first word / first edge of each scene (prefix sums).
 * Blocks until done. Totals above the capacities give CG_ERR_CAPACITY with all
 * counts written and nothing written to the outputs.
 * ------------------------------------------------------------------------- */
typedef struct cg_scene {
  const int32_t* pts; /* int32[n][d], device */
  int64_t n;
  int d;
  const int32_t* a;   /* int32[l][d], device */
  const int64_t* b;   /* int64[l], device */
  int ell;
} cg_scene;

typedef struct cg_batch_out {
  uint64_t* cells;
  int64_t cells_cap;
  uint32_t* edges;
  int64_t edges_cap;
  int64_t* n_cells;
  int64_t* n_edges;
  int64_t* cells_offset;
  int64_t* edges_offset;
} cg_batch_out;

cg_status cg_build_batch(cg_ctx* ctx, const cg_scene* scenes, int n_scenes, cg_batch_out* out,
                         void* stream);

/* Autotuner: for every bucket of l present among the scenes (device arrays,
 * as for cg_build_batch), times those scenes (at most 16 per bucket) under
 * each candidate setting -- HASH, SORTED, TREE, HALVES, PIVOT with h in
 * {2, 3, 4}, and for l <= 64 both sign kernels -- and keeps the fastest
 * setting in the context. Several scenes of a bucket are timed as one
 * cg_build_batch, `reps` replays after two warm-up calls (device work under
 * concurrency, as a batch runs them); a lone scene is timed with cg_build,
 * `reps` times after one warm-up. chosen_ms (nullable, host
 * double[CG_TUNE_BUCKETS]) receives the best time per bucket (0 for buckets
 * without scenes). Blocks until done. */
cg_status cg_ctx_autotune(cg_ctx* ctx, const cg_scene* scenes, int n_scenes, int reps,
                          double* chosen_ms);

/* ---------------------------------------------------------------------------
 * Paths in the cell graph.
 * ------------------------------------------------------------------------- */
/* Breadth-first search on the cell graph G_X (§1 and §6: a path in the cell
 * graph is an approximate solution of the motion-planning problem; traversing
 * the graph on the GPU is the paper's next step).
 *   edges      device uint32[n_edges][2], undirected pairs (i, j) with i != j,
 *              both < n_cells -- the output of cg_neighbors_h1 / cg_build
 *              (any order is accepted);
 *   source     the start cell, 0 <= source < n_cells;
 *   dist       device int32[n_cells] (caller-owned, written): number of edges
 *              on a shortest path from source, -1 when unreachable;
 *   parent     device int32[n_cells] or NULL: the predecessor of every cell
 *              on one shortest path (a BFS tree; several are valid, any
 *              neighbour one level closer may be chosen), -1 for the source
 *              and unreachable cells;
 *   n_reached, depth  host out-params (nullable): cells reached (source
 *              included) and the largest finite distance.
 * Workspace: query with ws = NULL (O(n_cells + n_edges) bytes). The call
 * builds an adjacency of both directions, then searches level by level: all
 * levels in one cooperative launch with grid barriers between them where the
 * device allows it, else one launch per level with a look at the host once
 * per 16 levels (the environment variable CG_BFS_LEVELS=1 selects the latter);
 * it returns when the search is done. A grid-barrier wait that runs out (it
 * cannot in a co-resident grid) gives CG_ERR_TIMEOUT. Errors: CG_ERR_INVALID_ARG for bad sizes, a source out of range, or an
 * edge with an endpoint >= n_cells or i == j (detected on the device; dist is
 * then unspecified). */
cg_status cg_bfs(const uint32_t* edges, int64_t n_edges, int64_t n_cells, int64_t source,
                 int32_t* dist, int32_t* parent, int64_t* n_reached, int64_t* depth, void* ws,
                 size_t* ws_bytes, void* stream);


/* ---------------------------------------------------------------------------
 * Serving: a request loop that builds independent scenes (§2.1-§2.2 per scene)
 * as they arrive. The paper has no counterpart; this is the deployment form of
 * cg_build for a stream of requests.
 *
 * Continuous batching: a scheduler thread owned by the server admits queued
 * requests in arrival order as soon as a slot (one of max_inflight streams)
 * and enough of the HBM budget are free, and enqueues each admitted scene's
 * steps 1-4 on its slot's stream, so the work of requests that arrived at
 * different times runs on the device at the same time. A request is charged
 * its whole device footprint (copied inputs, workspace, cells and edges at
 * capacity) from admission; the workspace is returned when it completes, the
 * cells and edges stay on the device (charged) until cg_server_release. The
 * budget therefore bounds everything the server holds. Admission never
 * changes a result: each request's output is exactly what cg_build gives for
 * the same scene (64-bit words), alone or in any mix.
 *
 * A request whose table or edge capacity turns out too small is re-run with
 * larger capacities before it completes (it is re-queued at the head).
 * Results: cells uint64[U][ceil(l/64)] in value order and edges uint32[E][2]
 * in (i, j) order, as for cg_build.
 * ------------------------------------------------------------------------- */
typedef struct cg_server cg_server;

/* Request states reported by cg_server_poll. */
#define CG_REQ_QUEUED 0
#define CG_REQ_RUNNING 1
#define CG_REQ_DONE 2
#define CG_REQ_FAILED 3

typedef struct cg_server_result {
  cg_status status;       /* CG_OK, or why the request failed */
  int64_t n_cells;        /* U */
  int64_t n_edges;        /* E */
  int words;              /* 64-bit words per cell, ceil(l / 64) */
  const uint64_t* cells;  /* device, valid until cg_server_release */
  const uint32_t* edges;  /* device, valid until cg_server_release */
  double submit_us;       /* host steady clock, microseconds since server creation: */
  double admit_us;        /*   submitted, admitted (first time), and the moment the */
  double done_us;         /*   scheduler saw the request's completion flag */
  int retries;            /* re-runs after a capacity overflow */
} cg_server_result;

typedef struct cg_server_stats {
  int64_t submitted, completed, failed, retried;
  int64_t queued, running;        /* now */
  size_t bytes_in_use;            /* charged against the budget now */
  size_t peak_bytes;              /* maximum of bytes_in_use so far */
  int max_running;                /* most requests running at once so far */
  int64_t groups;                 /* launches of admitted requests together ... */
  int64_t grouped;                /* ... and the requests started that way */
} cg_server_stats;

/* Creates a server on `device` that holds at most hbm_budget_bytes of device
 * memory for requests and runs at most max_inflight requests at once
 * (1..64). The budget is reserved on the device at creation (one arena,
 * sub-allocated by the server; CG_ERR_OOM when it cannot be reserved).
 * Starts the scheduler threads. */
cg_status cg_server_create(int device, size_t hbm_budget_bytes, int max_inflight,
                           cg_server** out);

/* Queues one scene. inputs_on_host != 0: pts/a/b are HOST arrays (pinned for
 * asynchronous copies), copied to the request's device memory after
 * admission; 0: they are device arrays used in place. Either way they must
 * stay valid and unchanged until the request is DONE or FAILED. Writes the
 * request's ticket (> 0). Invalid scenes are rejected here
 * (CG_ERR_INVALID_ARG); a scene whose footprint exceeds the whole budget is
 * accepted and then FAILED with CG_ERR_CAPACITY. */
cg_status cg_server_submit(cg_server* srv, const cg_scene* scene, int inputs_on_host,
                           int64_t* ticket);

/* Writes the request's state (CG_REQ_*). Unknown or released tickets give
 * CG_ERR_INVALID_ARG. */
cg_status cg_server_poll(cg_server* srv, int64_t ticket, int* state);

/* Waits until the request is DONE or FAILED, at most timeout_s seconds
 * (< 0: no limit). Returns CG_OK when it finished (check the result's status),
 * CG_ERR_TIMEOUT when the time ran out first. */
cg_status cg_server_wait(cg_server* srv, int64_t ticket, double timeout_s);

/* Result of a DONE or FAILED request (CG_ERR_INVALID_ARG while it is still
 * queued or running). */
cg_status cg_server_result_get(cg_server* srv, int64_t ticket, cg_server_result* out);

/* Copies a DONE request's cells and edges to caller memory (host or device;
 * nullable when the capacity is 0); blocks until copied. Caps smaller than
 * U*words words / E edges give CG_ERR_CAPACITY and copy nothing. */
cg_status cg_server_copy(cg_server* srv, int64_t ticket, uint64_t* cells, int64_t cells_cap,
                         uint32_t* edges, int64_t edges_cap);

/* Frees a finished request's device result and forgets the ticket. */
cg_status cg_server_release(cg_server* srv, int64_t ticket);

cg_status cg_server_get_stats(cg_server* srv, cg_server_stats* out);

/* Copies the context's tuning (cg_ctx_tune_set / cg_ctx_autotune) into the
 * server; requests admitted afterwards use it. */
cg_status cg_server_use_tuning(cg_server* srv, const cg_ctx* ctx);

/* Host-side fault injection for tests: the next `count` device allocations the
 * scheduler makes report failure, so the requests that needed them FAIL with
 * CG_ERR_OOM while the server keeps serving the others. No GPU fault is made. */
cg_status cg_server_inject_alloc_failures(cg_server* srv, int count);

/* Stops admitting, lets running requests finish, fails queued ones, frees all
 * device memory of the server (results included) and joins its thread. */
cg_status cg_server_destroy(cg_server* srv);

/* ---------------------------------------------------------------------------
 * Allocation-free neighbour search. The paper has no counterpart: this is a
 * deployment variant of cg_neighbors_h1 (HASH strategy, 1 <= l <= 64) for
 * callers that cannot allocate device memory at the point of the call (fixed
 * memory budgets, real-time loops, hosts whose allocator belongs to another
 * framework). All scratch (hash table, look-back words, counters) lives in one
 * fixed array of about 2.1 MB compiled into the library, present on every
 * device that loads it until the process exits; the call itself allocates
 * nothing. Arguments, outputs, ordering and errors are those of
 * cg_neighbors_h1, plus:
 *   - at most CG_NOALLOC_MAX_CELLS cells; more gives CG_ERR_INVALID_ARG before
 *     any work is enqueued;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - like cg_neighbors_h1 it blocks until its work on `stream` is done (E is
 *     returned through a host pointer); unsorted or repeated rows and rows
 *     with bits at or above l give CG_ERR_INVALID_ARG, as there;
 *   - every call reuses the same array (each call clears what must start at
 *     zero); calls whose work overlaps on the GPU race and give undefined
 *     results, so serialise them.
 * ------------------------------------------------------------------------- */
#define CG_NOALLOC_MAX_CELLS 65536
cg_status cg_neighbors_h1_noalloc(const void* cells, int64_t n_cells, int ell, int word_bits,
                                  uint32_t* edges, int64_t edges_cap, int64_t* n_edges,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CELLGRAPH_H */
