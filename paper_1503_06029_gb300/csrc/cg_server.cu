// Request server (cg_server_*): continuous batching of independent scene
// builds (§2.1-§2.2 per scene) under a device-memory budget.
//
// Threads:
//   * callers submit, poll, wait, copy and release under `mu`;
//   * up to kSchedThreads scheduler threads, each owning a share of the slot
//     streams, admit queued requests (arrival order, from one shared queue)
//     whenever one of their slots and enough of the budget are free, enqueue
//     each admitted scene on its slot's stream, and settle completions;
//   * an event recorded after each request's last operation marks its
//     completion; the scheduler thread that owns the slot polls it and
//     settles the request (the completion time is taken when it is seen).
// No CUDA call is ever made while `mu` is held: some runtime calls may wait
// for earlier work in a stream.
//
// Memory: each request owns two stream-ordered allocations from the server's
// memory pool: a work block (counters, copied inputs, build workspace) that is
// freed when the request completes, and a result block (cells and edges at
// capacity) that is freed by cg_server_release. Both are charged against the
// budget from admission until they are freed.
#include <chrono>
#include <condition_variable>
#include <deque>
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
  // outcome
  int64_t n_cells = 0, n_edges = 0;
  double t_submit = 0, t_admit = -1, t_done = 0;
  int retries = 0;
  cg_server* srv = nullptr;
};

}  // namespace

struct cg_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  Clock::time_point t0;
  std::vector<cudaStream_t> streams;
  DevCounters* hctr = nullptr;  // pinned, one per slot
  cudaStream_t copy_stream = nullptr;
  cudaMemPool_t pool = nullptr;
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
  std::vector<cudaEvent_t> done_ev;  // per slot: recorded after a request's last operation
  std::vector<Worker> workers;
  std::unordered_map<int64_t, Req*> reqs;
  size_t in_use = 0, peak = 0;
  int running = 0, max_running = 0;
  int64_t next_id = 1;
  int64_t submitted = 0, completed = 0, failed = 0, retried = 0;
  int inject_alloc_fail = 0;
  cg_tune_params tune[CG_TUNE_BUCKETS];
  bool stop = false;
};

namespace {

double now_us(const cg_server* s) {
  return std::chrono::duration<double, std::micro>(Clock::now() - s->t0).count();
}

// Sizes of a request's two blocks for its current capacities.
void plan_request(Req* r) {
  const cg_scene& sc = r->sc;
  r->plan = plan_scene(sc.n, sc.ell, r->cap, r->tp);
  r->w = (sc.ell + 63) / 64;
  if (r->ecap == 0) r->ecap = std::max<size_t>(1024, 4 * r->plan.ucap + 64);
  r->in_bytes = r->on_host ? align256(size_t(sc.n) * sc.d * 4) + align256(size_t(sc.ell) * sc.d * 4) +
                                 align256(size_t(sc.ell) * 8)
                           : 0;
  r->work_bytes = align256(sizeof(DevCounters)) + r->in_bytes + align256(scene_ws_bytes(r->plan));
  r->edges_off = align256(r->plan.ucap * size_t(r->w) * 8);
  r->result_bytes = r->edges_off + align256(r->ecap * 8);
}

// Allocates from the server's pool on stream st (or reports an injected
// failure).
cudaError_t pool_alloc(cg_server* s, void** p, size_t bytes, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->inject_alloc_fail > 0) {
      --s->inject_alloc_fail;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, s->pool, st);
}

// Enqueues an admitted request on its slot's stream. No lock held.
cg_status start_request(cg_server* s, Req* r) {
  cudaStream_t st = s->streams[size_t(r->slot)];
  void* wp = nullptr;
  void* rp = nullptr;
  cudaError_t e = pool_alloc(s, &wp, r->work_bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return srv_fail(CG_ERR_OOM, "request work block: " + std::string(cudaGetErrorString(e)));
  }
  e = pool_alloc(s, &rp, r->result_bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(wp, st);
    return srv_fail(CG_ERR_OOM, "request result block: " + std::string(cudaGetErrorString(e)));
  }
  r->work = static_cast<char*>(wp);
  r->result = static_cast<char*>(rp);
  const cg_scene& sc = r->sc;
  char* base = r->work;
  DevCounters* ctr = reinterpret_cast<DevCounters*>(base);
  size_t off = align256(sizeof(DevCounters));
  const int32_t* pts = sc.pts;
  const int32_t* a = sc.a;
  const int64_t* b = sc.b;
  auto undo = [&](cudaError_t err, const char* what) {
    cudaFreeAsync(r->work, st);
    cudaFreeAsync(r->result, st);
    r->work = r->result = nullptr;
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
  if (cs != CG_OK) {
    cudaFreeAsync(r->work, st);
    cudaFreeAsync(r->result, st);
    r->work = r->result = nullptr;
    return cs;
  }
  if ((e = cudaMemcpyAsync(&s->hctr[r->slot], ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess)
    return undo(e, "reading counters");
  if ((e = cudaEventRecord(s->done_ev[size_t(r->slot)], st)) != cudaSuccess)
    return undo(e, "completion event");
  return CG_OK;
}

// Settles a request whose stream work has finished. No lock held on entry.
void finish_request(cg_server* s, Req* r) {
  cudaStream_t st = s->streams[size_t(r->slot)];
  const DevCounters h = s->hctr[r->slot];
  enum { kOk, kRetry, kFail } what = kOk;
  cg_status fst = CG_OK;
  std::string msg;
  if (h.error & kErrTimeout) {
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
  cudaFreeAsync(r->work, st);
  r->work = nullptr;
  if (what != kOk) {
    cudaFreeAsync(r->result, st);
    r->result = nullptr;
  }
  if (what == kRetry) {
    if (h.overflow) r->cap = std::min(full_cap(r->sc.n), r->cap * 4);
    else r->ecap = size_t(h.n_edges) + 64;
    plan_request(r);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= freed_work + freed_result;
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
  if (s->queue.empty() || s->workers[size_t(k)].free_slots.empty()) return false;
  const Req* r = s->queue.front();
  const size_t need = r->work_bytes + r->result_bytes;
  return need > s->budget || s->in_use + need <= s->budget;
}

// Scheduler thread k: settles the requests of its slots whose completion
// event has fired (polled: a host callback per request would put every
// completion through the driver's single callback thread), then admits queued
// requests while the head fits; sleeps on the condition variable when idle,
// or for about 20 us while requests of its own are in flight.
void scheduler(cg_server* s, int k) {
  cudaSetDevice(s->device);
  cg_server::Worker& me = s->workers[size_t(k)];
  for (;;) {
    std::vector<Req*> fin;
    for (size_t q = 0; q < me.active.size();) {
      Req* r = me.active[q];
      if (cudaEventQuery(s->done_ev[size_t(r->slot)]) == cudaErrorNotReady) {
        ++q;
        continue;
      }
      r->t_done = now_us(s);
      fin.push_back(r);
      me.active[q] = me.active.back();
      me.active.pop_back();
    }
    for (Req* r : fin) finish_request(s, r);
    // Admit in arrival order while the head fits.
    bool admitted = false;
    for (;;) {
      Req* r = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop || !admissible(s, k)) break;
        r = s->queue.front();
        s->queue.pop_front();
        const size_t need = r->work_bytes + r->result_bytes;
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
        ++me.running;
        s->in_use += need;
        if (s->in_use > s->peak) s->peak = s->in_use;
        ++s->running;
        if (s->running > s->max_running) s->max_running = s->running;
        r->state = CG_REQ_RUNNING;
        if (r->t_admit < 0) r->t_admit = now_us(s);
      }
      const cg_status st = start_request(s, r);
      if (st == CG_OK) {
        me.active.push_back(r);
        admitted = true;
        continue;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->work_bytes + r->result_bytes;
      me.free_slots.push_back(r->slot);
      --me.running;
      r->slot = -1;
      --s->running;
      r->state = CG_REQ_FAILED;
      r->status = st;
      r->err = cg_last_error();
      ++s->failed;
      s->cv_done.notify_all();
    }
    if (!fin.empty() || admitted) continue;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return (!s->stop && admissible(s, k)) || (s->stop && me.active.empty()); };
    if (me.active.empty()) s->cv_sched.wait(lk, ready);
    else s->cv_sched.wait_for(lk, std::chrono::microseconds(20), ready);
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
  for (auto& t : s->tune) t = default_tune();
  auto bail = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto ev : s->done_ev) cudaEventDestroy(ev);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->hctr) cudaFreeHost(s->hctr);
    if (s->pool) cudaMemPoolDestroy(s->pool);
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
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return bail(e, "creating a completion event");
    s->done_ev.push_back(ev);
  }
  for (int k = max_inflight - 1; k >= 0; --k)
    s->workers[size_t(k % n_threads)].free_slots.push_back(k);
  if ((e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "creating the copy stream");
  if ((e = cudaMallocHost(&s->hctr, sizeof(DevCounters) * size_t(max_inflight))) != cudaSuccess)
    return bail(e, "pinned counters");
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return bail(e, "memory pool");
  uint64_t keep = hbm_budget_bytes;  // cached between requests, up to the budget
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
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
    if (r->result) srv->in_use -= r->result_bytes;
  }
  if (r->result) {
    DevGuard g(srv->device);
    cudaFreeAsync(r->result, srv->copy_stream);
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
  for (auto& kv : srv->reqs) {
    Req* r = kv.second;
    if (r->result) cudaFreeAsync(r->result, srv->copy_stream);
    delete r;
  }
  srv->reqs.clear();
  cudaStreamSynchronize(srv->copy_stream);
  for (auto st : srv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto ev : srv->done_ev) cudaEventDestroy(ev);
  cudaStreamDestroy(srv->copy_stream);
  cudaMemPoolDestroy(srv->pool);
  cudaFreeHost(srv->hctr);
  delete srv;
  return CG_OK;
}

}  // extern "C"
