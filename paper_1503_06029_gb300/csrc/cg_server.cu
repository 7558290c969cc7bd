// Request server (cg_server_*): continuous batching of independent scene
// builds (§2.1-§2.2 per scene) under a device-memory budget.
//
// Threads:
//   * callers submit, poll, wait, copy and release under `mu`;
//   * up to kSchedThreads scheduler threads, each owning a share of the slot
//     streams, admit queued requests (arrival order, from one shared queue)
//     whenever one of their slots and enough of the budget are free, enqueue
//     each admitted scene on its slot's stream, and settle completions;
//   * a one-warp kernel at the end of each request's stream work copies its
//     counters into mapped pinned host memory and then writes the request's
//     sequence number to its slot's host flag; the scheduler thread that owns
//     the slot polls the flag (a plain memory read, no driver call) and
//     settles the request (the completion time is taken when it is seen).
// No CUDA call is ever made while `mu` is held: some runtime calls may wait
// for earlier work in a stream.
//
// Memory: one device arena of the budget's size is reserved at creation and
// sub-allocated on the host (first fit in address order, 256-byte blocks,
// neighbours merged on free), so admitting and settling a request makes no
// allocation call. Each request owns two blocks: a work block (counters,
// copied inputs, build workspace) that is freed when the request completes,
// and a result block (cells and edges at capacity) that is freed by
// cg_server_release; blocks are freed only after the device work that used
// them has finished. A request that fits the budget but not the arena's free
// blocks (fragmentation) waits, like one that does not fit the budget, until a
// block is freed.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cg_plan.h"

using namespace cg;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 64;
constexpr int kSchedThreads = 4;  // scheduler threads (enqueueing is host-bound)
// Requests admitted in one pass that the segmented kernels can take (l <= 64,
// HASH or SORTED lookups, fp32 sign kernel) start together when there are at
// least kGroupMin of them: about 10 launches and one upload for the group
// instead of about 7 launches and 3 copies per request. Admission itself is
// not held back to form groups (measured: waiting for free slots cost more
// than the launches it saved), so groups form when requests arrive in bursts.
constexpr int kGroupMin = 4;
constexpr int kGroupMax = 64;

thread_local std::string t_msg;

cg_status srv_fail(cg_status st, const std::string& msg) {
  t_msg = msg;
  cg::set_last_error(t_msg.c_str());
  return st;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Req {
  int64_t id = 0;
  cg_scene sc{};
  bool on_host = false;
  int state = CG_REQ_QUEUED;
  cg_status status = CG_OK;
  std::string err;
  // plan
  size_t cap = 0;
  size_t ecap = 0;
  cg_tune_params tp{};
  ScenePlan plan{};
  int w = 1;
  size_t in_bytes = 0;  // copied inputs (host inputs only)
  size_t work_bytes = 0;
  size_t result_bytes = 0;
  size_t edges_off = 0;  // edges inside the result block
  // device memory and slot while admitted
  char* work = nullptr;
  char* result = nullptr;
  int slot = -1;
  int worker = -1;
  int run_slot = -1;  // the slot whose stream carries the work (own, or its group's)
  struct Group* group = nullptr;        // the group it ran in, if any
  unsigned int seq = 0;  // value its completion writes to the slot's host flag
  bool stream_error = false;
  // outcome
  int64_t n_cells = 0, n_edges = 0;
  double t_submit = 0, t_admit = -1, t_done = 0;
  int retries = 0;
  cg_server* srv = nullptr;
};

// Requests started together through the segmented kernels share one device
// block (descriptors, constraint arrays, sort scratch), freed when the last
// of them is settled.
struct Group {
  char* block = nullptr;
  size_t bytes = 0;
  int pending = 0;            // members not yet settled (changed under the server's mu)
  std::vector<char> staging;  // host copy of the uploaded descriptors
};

}  // namespace

struct cg_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  Clock::time_point t0;
  std::vector<cudaStream_t> streams;
  DevCounters* hctr = nullptr;    // mapped pinned, one per slot (host address)
  DevCounters* dctr = nullptr;    // the same memory, device address
  unsigned int* hflag = nullptr;  // mapped pinned completion flags, one per slot
  unsigned int* dflag = nullptr;
  std::vector<unsigned int> slot_seq;
  cudaStream_t copy_stream = nullptr;
  char* arena = nullptr;                  // device memory of the budget's size
  std::map<size_t, size_t> free_blocks;   // offset -> size, address order
  uint64_t free_gen = 0;                  // bumped on every free
  uint64_t blocked_gen = ~uint64_t(0);    // free_gen when an allocation last failed
  std::mutex mu;
  std::condition_variable cv_sched;
  std::condition_variable cv_done;
  std::deque<Req*> queue;
  // Scheduler threads: thread k owns the slots k, k + T, k + 2T, ... and
  // settles the requests that ran on them.
  struct Worker {
    std::thread th;
    std::vector<int> free_slots;
    std::vector<Req*> active;  // enqueued, completion not yet seen (this thread only)
    int running = 0;
  };
  std::vector<Worker> workers;
  std::unordered_map<int64_t, Req*> reqs;
  size_t in_use = 0, peak = 0;
  int running = 0, max_running = 0;
  int64_t next_id = 1;
  int64_t submitted = 0, completed = 0, failed = 0, retried = 0;
  int64_t groups = 0, grouped = 0;
  int inject_alloc_fail = 0;
  cg_tune_params tune[CG_TUNE_BUCKETS];
  bool stop = false;
};

namespace {

double now_us(const cg_server* s) {
  return std::chrono::duration<double, std::micro>(Clock::now() - s->t0).count();
}

// Whether the segmented kernels can take a request (see kGroupMin), before
// and after it has its blocks.
bool group_candidate(const Req* r) {
  const ScenePlan& p = r->plan;
  static const bool tc_forced = [] {
    const char* sk = std::getenv("CG_SIGN_KERNEL");
    return sk && std::strcmp(sk, "tc") == 0;
  }();
  return r->sc.n > 0 && p.small && scene_batch_sortable(p) && p.tp.sign_kernel != 1 &&
         !tc_forced && (p.tp.strategy == CG_STRATEGY_HASH || p.tp.strategy == CG_STRATEGY_SORTED);
}

bool group_eligible(const Req* r) { return r->work && r->result && group_candidate(r); }

// Sizes of a request's two blocks for its current capacities.
void plan_request(Req* r) {
  const cg_scene& sc = r->sc;
  r->plan = plan_scene(sc.n, sc.ell, r->cap, r->tp);
  // A served request's sign step stays one launch: the server's rate is set
  // by the CUDA calls each request start makes, and the box grid adds two.
  if (r->tp.sign_kernel != 2) r->plan.grid_bits = 0;
  r->w = (sc.ell + 63) / 64;
  if (r->ecap == 0) r->ecap = std::max<size_t>(1024, 4 * r->plan.ucap + 64);
  r->in_bytes = r->on_host ? align256(size_t(sc.n) * sc.d * 4) + align256(size_t(sc.ell) * sc.d * 4) +
                                 align256(size_t(sc.ell) * 8)
                           : 0;
  r->work_bytes = align256(sizeof(DevCounters)) + r->in_bytes + align256(scene_ws_bytes(r->plan));
  r->edges_off = align256(r->plan.ucap * size_t(r->w) * 8);
  r->result_bytes = r->edges_off + align256(r->ecap * 8);
}

// Arena blocks (mu held). First fit in address order.
bool arena_alloc(cg_server* s, size_t bytes, char** out) {
  bytes = align256(bytes > 0 ? bytes : 1);
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second < bytes) continue;
    const size_t off = it->first, size = it->second;
    s->free_blocks.erase(it);
    if (size > bytes) s->free_blocks.emplace(off + bytes, size - bytes);
    *out = s->arena + off;
    return true;
  }
  return false;
}

void arena_free(cg_server* s, char* p, size_t bytes) {
  if (!p) return;
  bytes = align256(bytes > 0 ? bytes : 1);
  size_t off = size_t(p - s->arena);
  auto next = s->free_blocks.lower_bound(off);
  if (next != s->free_blocks.end() && off + bytes == next->first) {
    bytes += next->second;
    next = s->free_blocks.erase(next);
  }
  ++s->free_gen;
  if (next != s->free_blocks.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      prev->second += bytes;
      return;
    }
  }
  s->free_blocks.emplace(off, bytes);
}

// Enqueues an admitted request on its slot's stream. No lock held.
cg_status start_request(cg_server* s, Req* r) {
  cudaStream_t st = s->streams[size_t(r->slot)];
  if (!r->work || !r->result)
    return srv_fail(CG_ERR_OOM, "request blocks: injected allocation failure");
  cudaError_t e = cudaSuccess;
  const cg_scene& sc = r->sc;
  char* base = r->work;
  DevCounters* ctr = reinterpret_cast<DevCounters*>(base);
  size_t off = align256(sizeof(DevCounters));
  const int32_t* pts = sc.pts;
  const int32_t* a = sc.a;
  const int64_t* b = sc.b;
  auto undo = [&](cudaError_t err, const char* what) {
    return srv_fail(CG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
  };
  if (r->on_host) {
    int32_t* dp = reinterpret_cast<int32_t*>(base + off);
    off += align256(size_t(sc.n) * sc.d * 4);
    int32_t* da = reinterpret_cast<int32_t*>(base + off);
    off += align256(size_t(sc.ell) * sc.d * 4);
    int64_t* db = reinterpret_cast<int64_t*>(base + off);
    off += align256(size_t(sc.ell) * 8);
    if (sc.n > 0 && (e = cudaMemcpyAsync(dp, sc.pts, size_t(sc.n) * sc.d * 4,
                                         cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return undo(e, "copying points");
    if ((e = cudaMemcpyAsync(da, sc.a, size_t(sc.ell) * sc.d * 4, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return undo(e, "copying normals");
    if ((e = cudaMemcpyAsync(db, sc.b, size_t(sc.ell) * 8, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return undo(e, "copying offsets");
    pts = dp;
    a = da;
    b = db;
  }
  PackArgs pa{pts, sc.n, sc.d, a, b, sc.ell};
  const cg_status cs =
      enqueue_scene(nullptr, base + off, ctr, r->plan, pa, 64, r->result, int64_t(r->plan.ucap),
                    reinterpret_cast<uint32_t*>(r->result + r->edges_off), int64_t(r->ecap), st);
  if (cs != CG_OK) return cs;
  if ((e = launch_publish_done(ctr, s->dctr + r->slot, s->dflag + r->slot, r->seq, st)) !=
      cudaSuccess)
    return undo(e, "completion flag");
  return CG_OK;
}

// Device layout of a group's block: descriptors, the constraint arrays of
// host-input requests, the searches' scratch and the sort's scratch.
struct GroupLayout {
  size_t clr, pk, sort, se, pub, scr, bs, desc_bytes, bytes;
  std::vector<size_t> a, b;
  size_t sort_cap, sort_seg;
};

GroupLayout group_layout(const std::vector<Req*>& g) {
  GroupLayout L{};
  const size_t K = g.size();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + (bytes > 0 ? bytes : 1));
    return o;
  };
  L.clr = take(K * sizeof(SegClear));
  L.pk = take(K * sizeof(SegPackScene));
  L.sort = take(K * sizeof(BatchSortScene));
  L.se = take(K * sizeof(SegSearchScene));
  L.pub = take(K * sizeof(PublishEntry));
  L.scr = take(2 * (K + 2) * sizeof(unsigned int));
  L.a.assign(K, 0);
  L.b.assign(K, 0);
  for (size_t i = 0; i < K; ++i)
    if (g[i]->on_host) {
      L.a[i] = take(size_t(g[i]->sc.ell) * g[i]->sc.d * 4);
      L.b[i] = take(size_t(g[i]->sc.ell) * 8);
    }
  L.desc_bytes = off;
  L.sort_cap = 0;
  L.sort_seg = 1024;
  for (const Req* r : g) {
    const size_t seg = batch_sort_seg_size(r->plan.ucap);
    L.sort_cap += seg;
    L.sort_seg = std::max(L.sort_seg, seg);
  }
  L.bs = take(batch_sort_bytes(L.sort_cap, int(K)));
  L.bytes = off;
  return L;
}

// Starts the requests of g (admitted, blocks and slots assigned, each with
// run_slot = g[0]->slot) together on g[0]'s slot stream: one upload of their
// descriptors and constraint arrays (staged in `staging`, which must live
// until the work is done), host points copied into each request's work
// block; then the clears, a sign + insert launch per (d,
// constraint chunks), one sort of every request's distinct vectors, the
// searches (HASH, then SORTED) and one completion launch. No lock held.
cg_status start_group(cg_server* s, const std::vector<Req*>& g, char* block,
                      const GroupLayout& L, std::vector<char>& staging) {
  const int K = int(g.size());
  cudaStream_t st = s->streams[size_t(g[0]->slot)];
  auto undo = [&](cudaError_t err, const char* what) {
    return srv_fail(CG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
  };
  staging.assign(L.desc_bytes, 0);
  char* hb = staging.data();
  SegClear* hclr = reinterpret_cast<SegClear*>(hb + L.clr);
  SegPackScene* hpk = reinterpret_cast<SegPackScene*>(hb + L.pk);
  BatchSortScene* hsort = reinterpret_cast<BatchSortScene*>(hb + L.sort);
  SegSearchScene* hse = reinterpret_cast<SegSearchScene*>(hb + L.se);
  PublishEntry* hpub = reinterpret_cast<PublishEntry*>(hb + L.pub);
  std::vector<PackArgs> pa(size_t(K), PackArgs{nullptr, 0, 0, nullptr, nullptr, 0});
  std::vector<char*> ws(static_cast<size_t>(K), nullptr);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < K; ++i) {
    Req* r = g[size_t(i)];
    const cg_scene& sc = r->sc;
    const int32_t* pts = sc.pts;
    const int32_t* a = sc.a;
    const int64_t* b = sc.b;
    const size_t off0 = align256(sizeof(DevCounters));
    if (r->on_host) {
      // Copied, not read in place from pinned memory: copies by the copy
      // engines served more scenes per second than sign kernels reading the
      // host link (31.1 k against 27.4 k scenes/s at half load).
      int32_t* dp = reinterpret_cast<int32_t*>(r->work + off0);
      if ((e = cudaMemcpyAsync(dp, sc.pts, size_t(sc.n) * sc.d * 4, cudaMemcpyHostToDevice,
                               st)) != cudaSuccess)
        return undo(e, "copying points");
      pts = dp;
      std::memcpy(hb + L.a[size_t(i)], sc.a, size_t(sc.ell) * sc.d * 4);
      std::memcpy(hb + L.b[size_t(i)], sc.b, size_t(sc.ell) * 8);
      a = reinterpret_cast<const int32_t*>(block + L.a[size_t(i)]);
      b = reinterpret_cast<const int64_t*>(block + L.b[size_t(i)]);
    }
    pa[size_t(i)] = PackArgs{pts, sc.n, sc.d, a, b, sc.ell};
    ws[size_t(i)] = r->work + off0 + r->in_bytes;
    DevCounters* ctr = reinterpret_cast<DevCounters*>(r->work);
    scene_small_descs(ws[size_t(i)], ctr, r->plan, pa[size_t(i)], 0, nullptr, 0, &hclr[i],
                      nullptr, nullptr);
    hsort[i] = scene_sort_desc(ws[size_t(i)], ctr, r->plan, reinterpret_cast<uint64_t*>(r->result),
                               int64_t(r->plan.ucap));
    hpub[i] = PublishEntry{ctr, s->dctr + r->slot, s->dflag + r->slot, r->seq};
  }
  // Sign + insert descriptors grouped by (d, constraint chunks), each group
  // numbering its 128-point tiles from 0; searches HASH first.
  struct PackGroup {
    int d, nch, first, count;
    uint64_t tiles;
  };
  std::vector<PackGroup> pgroups;
  int n_pk = 0;
  for (int d = 1; d <= 4; ++d)
    for (int nch = 1; nch <= 2; ++nch) {
      PackGroup gr{d, nch, n_pk, 0, 0};
      for (int i = 0; i < K; ++i) {
        const Req* r = g[size_t(i)];
        if (r->sc.d != d || (r->sc.ell > 32 ? 2 : 1) != nch) continue;
        scene_small_descs(ws[size_t(i)], reinterpret_cast<DevCounters*>(r->work), r->plan,
                          pa[size_t(i)], gr.tiles, nullptr, 0, nullptr, &hpk[n_pk], nullptr);
        ++n_pk;
        ++gr.count;
        gr.tiles += uint64_t((r->sc.n + 127) / 128);
      }
      if (gr.count) pgroups.push_back(gr);
    }
  int n_se[2] = {0, 0};
  size_t chunks[2] = {0, 0};
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < K; ++i) {
      const Req* r = g[size_t(i)];
      if ((r->plan.tp.strategy == CG_STRATEGY_SORTED) != (pass == 1)) continue;
      scene_small_descs(ws[size_t(i)], reinterpret_cast<DevCounters*>(r->work), r->plan,
                        pa[size_t(i)], 0, reinterpret_cast<uint32_t*>(r->result + r->edges_off),
                        int64_t(r->ecap), nullptr, nullptr, &hse[n_se[0] + n_se[1]]);
      ++n_se[pass];
      chunks[pass] += (r->plan.ucap + 31) / 32;
    }
  if ((e = cudaMemcpyAsync(block, hb, L.desc_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return undo(e, "uploading the group's descriptors");
  const SegClear* dclr = reinterpret_cast<const SegClear*>(block + L.clr);
  const SegPackScene* dpk = reinterpret_cast<const SegPackScene*>(block + L.pk);
  const BatchSortScene* dsort = reinterpret_cast<const BatchSortScene*>(block + L.sort);
  const SegSearchScene* dse = reinterpret_cast<const SegSearchScene*>(block + L.se);
  const PublishEntry* dpub = reinterpret_cast<const PublishEntry*>(block + L.pub);
  unsigned int* dscr = reinterpret_cast<unsigned int*>(block + L.scr);
  if ((e = launch_clear_seg(dclr, K, st)) != cudaSuccess) return undo(e, "clearing");
  for (const PackGroup& gr : pgroups)
    if ((e = launch_pack_insert_seg(dpk + gr.first, gr.count, gr.tiles, gr.d, gr.nch, st)) !=
        cudaSuccess)
      return undo(e, "sign vectors + dedup");
  if ((e = batch_sort(dsort, K, L.sort_cap, L.sort_seg, block + L.bs, st)) != cudaSuccess)
    return undo(e, "sorting cells");
  if (n_se[0] && (e = launch_neighbors_seg_small(dse, n_se[0], chunks[0], false, dscr, st)) !=
                     cudaSuccess)
    return undo(e, "neighbour search");
  if (n_se[1] && (e = launch_neighbors_seg_small(dse + n_se[0], n_se[1], chunks[1], true,
                                                 dscr + (K + 2), st)) != cudaSuccess)
    return undo(e, "neighbour search");
  if ((e = launch_publish_group(dpub, K, st)) != cudaSuccess) return undo(e, "completion flags");
  return CG_OK;
}


// Settles a request whose stream work has finished. No lock held on entry.
void finish_request(cg_server* s, Req* r) {
  const DevCounters h = s->hctr[r->slot];
  enum { kOk, kRetry, kFail } what = kOk;
  cg_status fst = CG_OK;
  std::string msg;
  if (r->stream_error) {
    what = kFail;
    fst = CG_ERR_CUDA;
    msg = "the request's stream reported an error";
  } else if (h.error & kErrTimeout) {
    what = kFail;
    fst = CG_ERR_TIMEOUT;
    msg = "a bounded device-side wait ran out";
  } else if (h.error) {
    what = kFail;
    fst = CG_ERR_INTERNAL;
    msg = "device-side consistency check failed";
  } else if (h.overflow) {
    if (r->cap >= full_cap(r->sc.n)) {
      what = kFail;
      fst = CG_ERR_INTERNAL;
      msg = "table overflow at full capacity";
    } else {
      what = kRetry;
    }
  } else if (h.n_edges > r->ecap) {
    what = kRetry;
  }
  const size_t freed_work = r->work_bytes;
  const size_t freed_result = what == kOk ? 0 : r->result_bytes;
  char* work = r->work;
  char* result = what == kOk ? nullptr : r->result;
  r->work = nullptr;
  if (what != kOk) r->result = nullptr;
  const size_t work_bytes = r->work_bytes, result_bytes = r->result_bytes;
  if (what == kRetry) {
    if (h.overflow) r->cap = std::min(full_cap(r->sc.n), r->cap * 4);
    else r->ecap = size_t(h.n_edges) + 64;
    plan_request(r);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    arena_free(s, work, work_bytes);
    arena_free(s, result, result_bytes);
    s->in_use -= freed_work + freed_result;
    if (Group* G = r->group) {
      r->group = nullptr;
      if (--G->pending == 0) {
        arena_free(s, G->block, G->bytes);
        s->in_use -= G->bytes;
        delete G;
      }
    }
    s->workers[size_t(r->worker)].free_slots.push_back(r->slot);
    --s->workers[size_t(r->worker)].running;
    r->slot = -1;
    --s->running;
    if (what == kRetry) {
      ++r->retries;
      ++s->retried;
      r->state = CG_REQ_QUEUED;
      s->queue.push_front(r);
    } else if (what == kFail) {
      r->state = CG_REQ_FAILED;
      r->status = fst;
      r->err = msg;
      ++s->failed;
    } else {
      r->n_cells = int64_t(h.n_unique);
      r->n_edges = int64_t(h.n_edges);
      r->state = CG_REQ_DONE;
      ++s->completed;
    }
  }
  s->cv_done.notify_all();
  s->cv_sched.notify_all();  // memory and a slot are free again
}

// True when the head of the queue can be admitted now by scheduler k (or must
// be failed).
bool admissible(const cg_server* s, int k) {
  const cg_server::Worker& me = s->workers[size_t(k)];
  if (s->queue.empty() || me.free_slots.empty()) return false;
  if (s->blocked_gen == s->free_gen) return false;  // the arena had no room; no free since
  const Req* r = s->queue.front();
  const size_t need = r->work_bytes + r->result_bytes;
  return need > s->budget || s->in_use + need <= s->budget;
}

// Scheduler thread k: settles the requests of its slots whose completion flag
// has been written (a read of mapped host memory: neither a host callback,
// whose single driver thread capped completions, nor an event query per
// request and poll, which competed with launches for the driver), then admits
// queued requests while the head fits; sleeps on the condition variable when
// idle, or for about 10 us while requests of its own are in flight. When no
// request of its own has finished for 100 ms, it asks the driver about their
// streams, so that a request whose stream failed is settled as failed.
void scheduler(cg_server* s, int k) {
  cudaSetDevice(s->device);
  cg_server::Worker& me = s->workers[size_t(k)];
  // An admitted request whose start failed part-way (after its stream has
  // drained): blocks and slot back, request failed. No lock held on entry.
  auto fail_started = [&](Req* r, cg_status st, const std::string& err) {
    std::lock_guard<std::mutex> lk(s->mu);
    arena_free(s, r->work, r->work_bytes);
    arena_free(s, r->result, r->result_bytes);
    r->work = r->result = nullptr;
    s->in_use -= r->work_bytes + r->result_bytes;
    me.free_slots.push_back(r->slot);
    --me.running;
    r->slot = -1;
    --s->running;
    r->state = CG_REQ_FAILED;
    r->status = st;
    r->err = err;
    ++s->failed;
    s->cv_done.notify_all();
  };
  auto start_one = [&](Req* r) {
    const cg_status st = start_request(s, r);
    if (st == CG_OK) {
      me.active.push_back(r);
      return;
    }
    // Part of the request may have been enqueued: its blocks are reused only
    // after that work has drained.
    const std::string err = cg_last_error();
    cudaStreamSynchronize(s->streams[size_t(r->slot)]);
    cudaGetLastError();
    fail_started(r, st, err);
  };
  // Admitted requests for the segmented kernels, started together (or one
  // by one when fewer than kGroupMin, or when the arena has no room for the
  // group's block).
  std::vector<Req*> pend;
  auto flush_group = [&]() {
    if (pend.empty()) return;
    if (int(pend.size()) >= kGroupMin) {
      const GroupLayout L = group_layout(pend);
      char* blk = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (arena_alloc(s, L.bytes, &blk)) {
          s->in_use += L.bytes;
          if (s->in_use > s->peak) s->peak = s->in_use;
        } else {
          blk = nullptr;
        }
      }
      if (blk) {
        Group* G = new Group();
        G->block = blk;
        G->bytes = L.bytes;
        G->pending = int(pend.size());
        for (Req* r : pend) {
          r->group = G;
          r->run_slot = pend[0]->slot;
        }
        const cg_status st = start_group(s, pend, blk, L, G->staging);
        if (st == CG_OK) {
          for (Req* r : pend) me.active.push_back(r);
          {
            std::lock_guard<std::mutex> lk(s->mu);
            ++s->groups;
            s->grouped += int64_t(pend.size());
          }
          pend.clear();
          return;
        }
        const std::string err = cg_last_error();
        cudaStreamSynchronize(s->streams[size_t(pend[0]->slot)]);
        cudaGetLastError();
        for (Req* r : pend) {
          r->group = nullptr;
          fail_started(r, st, err);
        }
        {
          std::lock_guard<std::mutex> lk(s->mu);
          arena_free(s, blk, L.bytes);
          s->in_use -= L.bytes;
        }
        delete G;
        pend.clear();
        return;
      }
    }
    for (Req* r : pend) start_one(r);
    pend.clear();
  };
  Clock::time_point last_progress = Clock::now();
  for (;;) {
    std::vector<Req*> fin;
    const bool check_streams =
        !me.active.empty() && Clock::now() - last_progress > std::chrono::milliseconds(100);
    for (size_t q = 0; q < me.active.size();) {
      Req* r = me.active[q];
      if (__atomic_load_n(&s->hflag[r->slot], __ATOMIC_ACQUIRE) != r->seq) {
        if (check_streams) {
          const cudaError_t e = cudaStreamQuery(s->streams[size_t(r->run_slot)]);
          if (e != cudaSuccess && e != cudaErrorNotReady) r->stream_error = true;
        }
        if (!r->stream_error) {
          ++q;
          continue;
        }
      }
      r->t_done = now_us(s);
      fin.push_back(r);
      me.active[q] = me.active.back();
      me.active.pop_back();
    }
    if (check_streams) last_progress = Clock::now();
    if (!fin.empty()) last_progress = Clock::now();
    for (Req* r : fin) finish_request(s, r);
    // Admit in arrival order while the head fits.
    bool admitted = false;
    for (;;) {
      Req* r = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop || !admissible(s, k)) break;
        r = s->queue.front();
        const size_t need = r->work_bytes + r->result_bytes;
        if (need <= s->budget) {
          bool injected = false;
          if (s->inject_alloc_fail > 0) {
            --s->inject_alloc_fail;
            injected = true;
          }
          char* wp = nullptr;
          char* rp = nullptr;
          if (!injected) {
            if (!arena_alloc(s, r->work_bytes, &wp)) {
              s->blocked_gen = s->free_gen;
              break;
            }
            if (!arena_alloc(s, r->result_bytes, &rp)) {
              arena_free(s, wp, r->work_bytes);
              s->blocked_gen = s->free_gen;
              break;
            }
          }
          r->work = wp;
          r->result = rp;
        }
        s->queue.pop_front();
        if (need > s->budget) {
          r->state = CG_REQ_FAILED;
          r->status = CG_ERR_CAPACITY;
          r->err = "request needs " + std::to_string(need) + " bytes, budget is " +
                   std::to_string(s->budget);
          ++s->failed;
          s->cv_done.notify_all();
          continue;
        }
        r->worker = k;
        r->slot = me.free_slots.back();
        me.free_slots.pop_back();
        r->seq = ++s->slot_seq[size_t(r->slot)];
        ++me.running;
        s->in_use += need;
        if (s->in_use > s->peak) s->peak = s->in_use;
        ++s->running;
        if (s->running > s->max_running) s->max_running = s->running;
        r->state = CG_REQ_RUNNING;
        if (r->t_admit < 0) r->t_admit = now_us(s);
      }
      r->run_slot = r->slot;
      admitted = true;
      if (group_eligible(r)) {
        pend.push_back(r);
        if (int(pend.size()) >= kGroupMax) flush_group();
        continue;
      }
      start_one(r);
    }
    flush_group();
    if (!fin.empty() || admitted) continue;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return (!s->stop && admissible(s, k)) || (s->stop && me.active.empty()); };
    if (me.active.empty()) s->cv_sched.wait(lk, ready);
    else s->cv_sched.wait_for(lk, std::chrono::microseconds(10), ready);
    if (s->stop && me.active.empty()) return;
  }
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

Req* find_locked(cg_server* s, int64_t ticket) {
  auto it = s->reqs.find(ticket);
  return it == s->reqs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

cg_status cg_server_create(int device, size_t hbm_budget_bytes, int max_inflight,
                           cg_server** out) {
  if (!out) return srv_fail(CG_ERR_INVALID_ARG, "out is NULL");
  if (max_inflight < 1 || max_inflight > kMaxSlots)
    return srv_fail(CG_ERR_INVALID_ARG, "max_inflight must be 1..64");
  if (hbm_budget_bytes == 0) return srv_fail(CG_ERR_INVALID_ARG, "budget is 0");
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
    cudaGetLastError();
    return srv_fail(CG_ERR_INVALID_ARG, "no such device");
  }
  DevGuard g(device);
  cg_server* s = new cg_server();
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_inflight;
  s->t0 = Clock::now();
  for (int b = 0; b < CG_TUNE_BUCKETS; ++b) s->tune[b] = default_tune(b);
  auto bail = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->hctr) cudaFreeHost(s->hctr);
    if (s->hflag) cudaFreeHost(s->hflag);
    if (s->arena) cudaFree(s->arena);
    delete s;
    return srv_fail(CG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  const int n_threads = max_inflight < kSchedThreads ? max_inflight : kSchedThreads;
  s->workers = std::vector<cg_server::Worker>(static_cast<size_t>(n_threads));
  for (int k = 0; k < max_inflight; ++k) {
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(e, "creating a slot stream");
    s->streams.push_back(st);
  }
  s->slot_seq.assign(size_t(max_inflight), 0u);
  for (int k = max_inflight - 1; k >= 0; --k) {
    s->workers[size_t(k % n_threads)].free_slots.push_back(k);
  }
  if ((e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "creating the copy stream");
  if ((e = cudaHostAlloc(reinterpret_cast<void**>(&s->hctr),
                         sizeof(DevCounters) * size_t(max_inflight), cudaHostAllocMapped)) !=
      cudaSuccess)
    return bail(e, "pinned counters");
  if ((e = cudaHostAlloc(reinterpret_cast<void**>(&s->hflag),
                         sizeof(unsigned int) * size_t(max_inflight), cudaHostAllocMapped)) !=
      cudaSuccess)
    return bail(e, "pinned completion flags");
  std::memset(s->hflag, 0, sizeof(unsigned int) * size_t(max_inflight));
  if ((e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->dctr), s->hctr, 0)) !=
          cudaSuccess ||
      (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->dflag), s->hflag, 0)) !=
          cudaSuccess)
    return bail(e, "device addresses of the pinned words");
  const size_t arena_bytes = align256(hbm_budget_bytes);
  if ((e = cudaMalloc(reinterpret_cast<void**>(&s->arena), arena_bytes)) != cudaSuccess) {
    cudaGetLastError();
    for (auto st : s->streams) cudaStreamDestroy(st);
    cudaStreamDestroy(s->copy_stream);
    cudaFreeHost(s->hctr);
    cudaFreeHost(s->hflag);
    delete s;
    return srv_fail(CG_ERR_OOM, "cannot reserve the budget (" + std::to_string(hbm_budget_bytes) +
                                    " bytes) on the device");
  }
  s->free_blocks.emplace(size_t(0), arena_bytes);
  for (int k = 0; k < n_threads; ++k) s->workers[size_t(k)].th = std::thread(scheduler, s, k);
  *out = s;
  return CG_OK;
}

cg_status cg_server_submit(cg_server* srv, const cg_scene* scene, int inputs_on_host,
                           int64_t* ticket) {
  if (!srv || !scene || !ticket) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  const cg_scene& sc = *scene;
  if (sc.n < 0 || uint64_t(sc.n) >= 0xffffffffull)
    return srv_fail(CG_ERR_INVALID_ARG, "n must satisfy 0 <= n < 2^32 - 1");
  if (sc.ell < 1 || sc.ell > 4096) return srv_fail(CG_ERR_INVALID_ARG, "l must be 1..4096");
  if (sc.d < 1 || sc.d > 4) return srv_fail(CG_ERR_INVALID_ARG, "d must be 1..4");
  if ((sc.n > 0 && !sc.pts) || !sc.a || !sc.b)
    return srv_fail(CG_ERR_INVALID_ARG, "NULL input array");
  Req* r = new Req();
  r->sc = sc;
  r->on_host = inputs_on_host != 0;
  r->srv = srv;
  r->cap = std::min(initial_cap(sc.n, sc.d, sc.ell), full_cap(sc.n));
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->tp = srv->tune[cg_tune_bucket(sc.ell)];
  }
  plan_request(r);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) {
      delete r;
      return srv_fail(CG_ERR_INVALID_ARG, "server is shutting down");
    }
    r->id = srv->next_id++;
    r->t_submit = now_us(srv);
    srv->reqs[r->id] = r;
    srv->queue.push_back(r);
    ++srv->submitted;
    *ticket = r->id;
  }
  srv->cv_sched.notify_all();
  return CG_OK;
}

cg_status cg_server_poll(cg_server* srv, int64_t ticket, int* state) {
  if (!srv || !state) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  Req* r = find_locked(srv, ticket);
  if (!r) return srv_fail(CG_ERR_INVALID_ARG, "unknown ticket");
  *state = r->state;
  return CG_OK;
}

cg_status cg_server_wait(cg_server* srv, int64_t ticket, double timeout_s) {
  if (!srv) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  if (!find_locked(srv, ticket)) return srv_fail(CG_ERR_INVALID_ARG, "unknown ticket");
  bool gone = false;
  auto settled = [&] {
    Req* r = find_locked(srv, ticket);
    if (!r) {
      gone = true;
      return true;
    }
    return r->state == CG_REQ_DONE || r->state == CG_REQ_FAILED;
  };
  bool ok;
  if (timeout_s < 0) {
    srv->cv_done.wait(lk, settled);
    ok = true;
  } else {
    ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), settled);
  }
  if (gone) return srv_fail(CG_ERR_INVALID_ARG, "ticket released while waiting");
  return ok ? CG_OK : srv_fail(CG_ERR_TIMEOUT, "request not finished within the timeout");
}

cg_status cg_server_result_get(cg_server* srv, int64_t ticket, cg_server_result* out) {
  if (!srv || !out) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  Req* r = find_locked(srv, ticket);
  if (!r) return srv_fail(CG_ERR_INVALID_ARG, "unknown ticket");
  if (r->state != CG_REQ_DONE && r->state != CG_REQ_FAILED)
    return srv_fail(CG_ERR_INVALID_ARG, "request not finished");
  out->status = r->status;
  out->n_cells = r->n_cells;
  out->n_edges = r->n_edges;
  out->words = r->w;
  out->cells = r->state == CG_REQ_DONE ? reinterpret_cast<const uint64_t*>(r->result) : nullptr;
  out->edges = r->state == CG_REQ_DONE
                   ? reinterpret_cast<const uint32_t*>(r->result + r->edges_off)
                   : nullptr;
  out->submit_us = r->t_submit;
  out->admit_us = r->t_admit;
  out->done_us = r->t_done;
  out->retries = r->retries;
  if (r->state == CG_REQ_FAILED) cg::set_last_error(r->err.c_str());
  return CG_OK;
}

cg_status cg_server_copy(cg_server* srv, int64_t ticket, uint64_t* cells, int64_t cells_cap,
                         uint32_t* edges, int64_t edges_cap) {
  if (!srv) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (cells_cap < 0 || edges_cap < 0 || (cells_cap > 0 && !cells) || (edges_cap > 0 && !edges))
    return srv_fail(CG_ERR_INVALID_ARG, "bad output array or capacity");
  const char* src = nullptr;
  size_t cell_words = 0, n_edges = 0, edges_off = 0;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    Req* r = find_locked(srv, ticket);
    if (!r) return srv_fail(CG_ERR_INVALID_ARG, "unknown ticket");
    if (r->state != CG_REQ_DONE) return srv_fail(CG_ERR_INVALID_ARG, "request not done");
    src = r->result;
    cell_words = size_t(r->n_cells) * size_t(r->w);
    n_edges = size_t(r->n_edges);
    edges_off = r->edges_off;
  }
  if (int64_t(cell_words) > cells_cap || int64_t(n_edges) > edges_cap)
    return srv_fail(CG_ERR_CAPACITY, "output capacity too small");
  DevGuard g(srv->device);
  cudaError_t e = cudaSuccess;
  if (cell_words)
    e = cudaMemcpyAsync(cells, src, cell_words * 8, cudaMemcpyDefault, srv->copy_stream);
  if (e == cudaSuccess && n_edges)
    e = cudaMemcpyAsync(edges, src + edges_off, n_edges * 8, cudaMemcpyDefault, srv->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(srv->copy_stream);
  if (e != cudaSuccess)
    return srv_fail(CG_ERR_CUDA, std::string("copying a result: ") + cudaGetErrorString(e));
  return CG_OK;
}

cg_status cg_server_release(cg_server* srv, int64_t ticket) {
  if (!srv) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    r = find_locked(srv, ticket);
    if (!r) return srv_fail(CG_ERR_INVALID_ARG, "unknown ticket");
    if (r->state != CG_REQ_DONE && r->state != CG_REQ_FAILED)
      return srv_fail(CG_ERR_INVALID_ARG, "request not finished");
    srv->reqs.erase(ticket);
    if (r->result) {
      srv->in_use -= r->result_bytes;
      arena_free(srv, r->result, r->result_bytes);
      r->result = nullptr;
    }
  }
  delete r;
  srv->cv_sched.notify_all();
  srv->cv_done.notify_all();
  return CG_OK;
}

cg_status cg_server_get_stats(cg_server* srv, cg_server_stats* out) {
  if (!srv || !out) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->failed = srv->failed;
  out->retried = srv->retried;
  out->queued = int64_t(srv->queue.size());
  out->running = srv->running;
  out->bytes_in_use = srv->in_use;
  out->peak_bytes = srv->peak;
  out->max_running = srv->max_running;
  out->groups = srv->groups;
  out->grouped = srv->grouped;
  return CG_OK;
}

cg_status cg_server_use_tuning(cg_server* srv, const cg_ctx* ctx) {
  if (!srv || !ctx) return srv_fail(CG_ERR_INVALID_ARG, "NULL argument");
  cg_tune_params t[CG_TUNE_BUCKETS];
  for (int b = 0; b < CG_TUNE_BUCKETS; ++b) {
    const cg_status st = cg_ctx_tune_get(ctx, b, &t[b]);
    if (st) return st;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  for (int b = 0; b < CG_TUNE_BUCKETS; ++b) srv->tune[b] = t[b];
  return CG_OK;
}

cg_status cg_server_inject_alloc_failures(cg_server* srv, int count) {
  if (!srv || count < 0) return srv_fail(CG_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->inject_alloc_fail = count;
  return CG_OK;
}

cg_status cg_server_destroy(cg_server* srv) {
  if (!srv) return CG_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_sched.notify_all();
  for (auto& w : srv->workers)
    if (w.th.joinable()) w.th.join();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    for (Req* r : srv->queue) {
      r->state = CG_REQ_FAILED;
      r->status = CG_ERR_INVALID_ARG;
      r->err = "server shut down before the request was admitted";
      ++srv->failed;
    }
    srv->queue.clear();
  }
  srv->cv_done.notify_all();
  DevGuard g(srv->device);
  for (auto& kv : srv->reqs) delete kv.second;
  srv->reqs.clear();
  cudaStreamSynchronize(srv->copy_stream);
  for (auto st : srv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaStreamDestroy(srv->copy_stream);
  cudaFree(srv->arena);
  cudaFreeHost(srv->hctr);
  cudaFreeHost(srv->hflag);
  delete srv;
  return CG_OK;
}

}  // extern "C"
