// cg_neighbors_h1_noalloc: the Hamming-1 neighbour search for vectors of
// l <= 64 bits with every piece of scratch memory taken from one fixed array
// compiled into this library, so the call allocates nothing.
//
// Who needs it: callers that must not (or cannot) allocate device memory at
// the point of the call -- for example code running under a hard real-time
// or fixed-memory budget, host processes whose allocator is owned by another
// framework, or callers that pre-plan every byte of device memory. They pass
// their own input and output buffers; the table, the look-back words and the
// counters live in `g_scratch` below.
//
// Properties:
//   * Capacity: at most kNoAllocMaxCells cells per call (larger inputs are
//     rejected with CG_ERR_INVALID_ARG before any work is enqueued). The array
//     takes kScratchBytes of device memory on every device that loads the
//     library, until the process exits.
//   * Set-up: the first call on a device, with that device current, looks up
//     the array's device address with cudaGetSymbolAddress (once per device,
//     under a lock). Make that first call before any stream capture.
//   * Like cg_neighbors_h1, the call waits for its work on the stream to
//     finish before it returns E through the host pointer.
//   * Input checks are those of cg_neighbors_h1: rows that are not strictly
//     ascending, or that have bits at or above l, give CG_ERR_INVALID_ARG.
//   * Sharing: every call uses the same array and leaves its contents behind;
//     each call first clears what must start from zero (table, counters,
//     look-back words). Calls whose work overlaps on the GPU (different
//     streams, or different host threads) race on the array and give undefined
//     results: serialise them.
#include <mutex>
#include <string>

#include "../../include/cellgraph.h"
#include "cg_internal.cuh"

namespace {

constexpr size_t kNoAllocMaxCells = CG_NOALLOC_MAX_CELLS;
constexpr size_t kTableCap = 2 * kNoAllocMaxCells;  // power of two, load <= 1/2
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Layout of the array: counters | table keys | table values | cells | look-back.
constexpr size_t kOffCtr = 0;
constexpr size_t kOffKeys = align_up(kOffCtr + sizeof(cg::DevCounters));
constexpr size_t kOffVals = align_up(kOffKeys + kTableCap * sizeof(uint64_t));
constexpr size_t kOffCells = align_up(kOffVals + kTableCap * sizeof(uint32_t));
constexpr size_t kOffStatus = align_up(kOffCells + kNoAllocMaxCells * sizeof(uint64_t));
constexpr size_t kStatusWords = kNoAllocMaxCells / 32 + 2;
constexpr size_t kScratchBytes = align_up(kOffStatus + kStatusWords * sizeof(unsigned long long));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

cg_status noalloc_fail(cg_status st, const char* msg) {
  cg::set_last_error(msg);
  return st;
}

// Device address of g_scratch on the current device (looked up once).
cg_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(CG_ERR_CUDA, "cg_neighbors_h1_noalloc: no usable current device");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(CG_ERR_CUDA, "cg_neighbors_h1_noalloc: cudaGetSymbolAddress failed");
    cg::sm_count();  // cache the SM count now, so later calls do no host-side set-up
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_neighbors_h1_noalloc(const void* cells, int64_t n_cells, int ell, int word_bits,
                                  uint32_t* edges, int64_t edges_cap, int64_t* n_edges,
                                  void* stream) {
  using namespace cg;
  if (n_cells < 0 || size_t(n_cells) > kNoAllocMaxCells)
    return noalloc_fail(CG_ERR_INVALID_ARG,
                        "cg_neighbors_h1_noalloc: n_cells exceeds the fixed capacity of 65536");
  if (ell < 1 || ell > 64)
    return noalloc_fail(CG_ERR_INVALID_ARG, "cg_neighbors_h1_noalloc: needs 1 <= l <= 64");
  if (word_bits != 32 && word_bits != 64)
    return noalloc_fail(CG_ERR_INVALID_ARG, "cg_neighbors_h1_noalloc: word_bits must be 32 or 64");
  if (!n_edges || (n_cells > 0 && !cells) || edges_cap < 0 || (edges_cap > 0 && !edges))
    return noalloc_fail(CG_ERR_INVALID_ARG, "cg_neighbors_h1_noalloc: NULL or bad argument");
  void* base = nullptr;
  cg_status st = scratch_address(&base);
  if (st) return st;
  char* b = static_cast<char*>(base);
  DevCounters* ctr = reinterpret_cast<DevCounters*>(b + kOffCtr);
  uint64_t* tkeys = reinterpret_cast<uint64_t*>(b + kOffKeys);
  uint32_t* tvals = reinterpret_cast<uint32_t*>(b + kOffVals);
  uint64_t* icells = reinterpret_cast<uint64_t*>(b + kOffCells);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(b + kOffStatus);
  SmallTable t{tkeys, tvals, uint32_t(kTableCap - 1), table_shift(kTableCap), nullptr, 0u, ctr};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t un = size_t(n_cells > 0 ? n_cells : 1);
  cudaError_t e = launch_clear_build(tkeys, kTableCap, status, ne_status_words(un), ctr, s);
  if (e == cudaSuccess) e = launch_load_cells(cells, n_cells, word_bits, ell, icells, ctr, s);
  // The same precondition check as cg_neighbors_h1: strictly ascending rows.
  if (e == cudaSuccess) e = launch_check_sorted(icells, 1, ctr, un, s);
  if (e == cudaSuccess) e = launch_index_small(icells, t, un, s);
  if (e == cudaSuccess)
    e = launch_neighbors_emit_small(icells, t, ell, CG_STRATEGY_HASH, status, edges, edges_cap,
                                    un, s);
  DevCounters host{};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cg::set_last_error((std::string("cg_neighbors_h1_noalloc: ") + cudaGetErrorString(e)).c_str());
    return CG_ERR_CUDA;
  }
  // Error bits in the order cg_neighbors_h1 reports them.
  if (host.error & kErrUnsorted)
    return noalloc_fail(CG_ERR_INVALID_ARG,
                        "cg_neighbors_h1_noalloc: cells are not sorted ascending and unique");
  if (host.error & kErrHighBits)
    return noalloc_fail(CG_ERR_INVALID_ARG,
                        "cg_neighbors_h1_noalloc: cells have bits set at or above l");
  if (host.error & kErrTimeout)
    return noalloc_fail(CG_ERR_TIMEOUT, "cg_neighbors_h1_noalloc: a bounded wait ran out");
  if (host.error)
    return noalloc_fail(CG_ERR_INTERNAL,
                        "cg_neighbors_h1_noalloc: a device-side consistency check failed");
  if (host.overflow)
    return noalloc_fail(CG_ERR_INTERNAL, "cg_neighbors_h1_noalloc: lookup table overflow");
  *n_edges = int64_t(host.n_edges);
  if (int64_t(host.n_edges) > edges_cap)
    return noalloc_fail(CG_ERR_CAPACITY, "cg_neighbors_h1_noalloc: edges_cap too small");
  return CG_OK;
}

}  // extern "C"
