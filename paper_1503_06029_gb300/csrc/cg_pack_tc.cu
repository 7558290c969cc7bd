// Step 1 of the cell-graph construction (sign vectors, §2.1) on the 5th-gen
// tensor cores, for l <= 64 and d <= 4.
//
// The l affine forms s_c(p) = a_c . p - b_c of a tile of 128 points are one
// small contraction: S = P~ x A~^T with K = 16. The integers are split so that
// every product and every partial sum is exactly representable, which makes
// the fp16 x fp16 -> fp32 tensor-core result exact:
//
//   p = 2048 ph + pl          (pl in [0, 2048), |ph| <= 2048 for |p| < 2^22)
//   b = 2048 bh + bl          (bl in [0, 2048)),  bh = 1024 c1 + c0 (c0 in [0, 1024))
//   S_hi = sum_k a_k ph_k - 1024 c1 - c0          (integer, |S_hi| < 2^24)
//   S_lo = sum_k a_k pl_k - bl + 1/2              (half-integer, |S_lo| < 2^23)
//   s + 1/2 = 2048 S_hi + S_lo
//
// Row of P~ (one point):  [ph_0..ph_{d-1}, pl_0..pl_{d-1}, 1024, 1, 1, 1/2, 0...]
// Column of A~ (hi, c):   [a_c, 0, -c1, -c0, 0, 0, ...]
// Column of A~ (lo, c):   [0, a_c, 0, 0, -bl, 1, ...]
//
// The hi and lo results of constraint c land in TMEM columns c and NC/2 + c.
// One fma per result gives fl(s + 1/2); since s + 1/2 is never 0, its sign bit
// is exactly [s < 0]. The split needs |a_ck| <= 2048, sum_k |a_ck| < 4096,
// |b_c| < 2^31 (checked once per block) and |p_k| < 2^22 (checked per tile);
// a tile outside these ranges is evaluated in fp32 with the proven error bound
// and exact 128-bit re-evaluation of uncertain bits (same method as the FFMA
// kernel in cg_pack.cu).
//
// Per tile: threads write their row of P~ to shared memory (no-swizzle K-major
// core-matrix layout), one thread issues tcgen05.mma (M = 128, N = NC, K = 16)
// into this block's TMEM columns and commits to an mbarrier; every thread then
// reads its point's row of S with tcgen05.ld, combines hi and lo with one fp32
// FMA per constraint, and collects the sign bits. Up to 512 / NC blocks share
// an SM (TMEM has 512 columns), so one block's MMA overlaps the others'
// epilogues.
#include <cuda_fp16.h>

#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kTThreads = 128;          // one thread per point of a tile
constexpr int kTilePts = 128;
constexpr uint32_t kSpinLimit = 2000;  // tries of ~1 ms each at most

// ----------------------------- PTX wrappers -----------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle (core matrices of 8 rows x 16 B):
// start address, leading-dimension byte offset (between core matrices along
// K), stride-dimension byte offset (between core matrices along M/N), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor, kind::f16: D f32, A/B f16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar_smem) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          mbar_smem));
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar_smem, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_smem), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits for the phase with the given parity, suspending in hardware for up to
// ~1 ms (the time hint, in ns) instead of spinning; false if it timed out.
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar_smem, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar_smem), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t uabs32(int32_t v) {
  return v < 0 ? 0u - uint32_t(v) : uint32_t(v);
}

template <int D>
__device__ __forceinline__ bool exact_ge(const int32_t* __restrict__ a_row, int64_t b,
                                         const int32_t (&p)[D]) {
  __int128 s = -static_cast<__int128>(b);
#pragma unroll
  for (int k = 0; k < D; ++k) s += static_cast<__int128>(int64_t(a_row[k]) * int64_t(p[k]));
  return s >= 0;
}

// Offset of element (row, k) in the no-swizzle K-major layout with K = 16
// halves per row: core matrix (row/8, k/8) at (row/8)*256 + (k/8)*128 bytes.
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = 256;
__device__ __forceinline__ uint32_t kmajor_offset(int row, int kchunk) {
  return uint32_t(row >> 3) * kSBO + uint32_t(kchunk) * kLBO + uint32_t(row & 7) * 16;
}

__device__ __forceinline__ uint32_t h2(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ------------------------------- sinks -------------------------------

struct TcInsert {
  SmallTable t;
  // First half of an insertion: the home slot and its current content (the
  // load is issued here and consumed one tile later).
  __device__ __forceinline__ void probe(uint64_t key, uint32_t& slot, uint64_t& cur) const {
    slot = home_slot(key, t.shift);
    cur = key == kEmpty ? 0ull : t.keys[slot];
  }
  __device__ __forceinline__ void finish(uint64_t key, uint32_t slot, uint64_t cur) const {
    if (key == kEmpty || cur != key) small_insert_from(t, key, slot, cur);
  }
};

// --------------------------------- kernel ---------------------------------

struct TcShared {
  alignas(1024) unsigned char a[kTilePts * 32];  // P~ tile, 128 rows x 16 halves
  alignas(1024) unsigned char b[128 * 32];       // A~, up to 128 rows x 16 halves
  uint32_t wmax[2][4][4];
  unsigned long long mbar;
  uint32_t tmem;
};

// Spill list of tiles the exact split cannot take (evaluated afterwards by the
// fp32 kernel in list mode).
struct TcSpill {
  uint32_t* tiles;
  unsigned int* count;
};

template <int D>
__device__ __forceinline__ void write_row(unsigned char* a, int row, const int32_t (&pi)[D]) {
  float v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int32_t ph = pi[k] >> 11;  // floor
    v[k] = float(ph);
    v[D + k] = float(pi[k] - ph * 2048);
  }
  v[2 * D] = 1024.0f;
  v[2 * D + 1] = 1.0f;
  v[2 * D + 2] = 1.0f;
  v[2 * D + 3] = 0.5f;
  uint4 q0, q1;
  q0.x = h2(v[0], v[1]);
  q0.y = h2(v[2], v[3]);
  q0.z = h2(v[4], v[5]);
  q0.w = h2(v[6], v[7]);
  q1.x = h2(v[8], v[9]);
  q1.y = h2(v[10], v[11]);
  q1.z = h2(v[12], v[13]);
  q1.w = h2(v[14], v[15]);
  *reinterpret_cast<uint4*>(a + kmajor_offset(row, 0)) = q0;
  *reinterpret_cast<uint4*>(a + kmajor_offset(row, 1)) = q1;
}

template <int D>
__device__ __forceinline__ void load_point(const PackArgs& pa, int64_t tile, int64_t ntiles,
                                           int tid, int32_t (&pi)[D]) {
  const int64_t p = tile * kTilePts + tid;
  const bool ok = tile < ntiles && p < pa.n;
#pragma unroll
  for (int k = 0; k < D; ++k) pi[k] = ok ? __ldg(pa.pts + p * D + k) : 0;
}

// Rows of A~ (the constraints' split coefficients, NC rows of 16 halves) in
// the no-swizzle K-major layout, written by threads tid, tid + nthreads, ...;
// returns 0 when a constraint of this thread is outside the exact-split ranges.
template <int D, int NC>
__device__ __forceinline__ int stage_b_rows(const PackArgs& pa, unsigned char* b, int tid,
                                            int nthreads) {
  constexpr int kL = NC / 2;
  int ok = 1;
  for (int row = tid; row < NC; row += nthreads) {
    const bool lo_half = row >= kL;
    const int c = lo_half ? row - kL : row;
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.0f;
    if (c < pa.ell) {
      const int32_t* ar = pa.a + int64_t(c) * D;
      const int64_t bt = pa.b[c];
      uint32_t sum = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const uint32_t m = uabs32(ar[k]);
        if (m > 2048u) ok = 0;
        sum += min(m, 4096u);
        v[lo_half ? D + k : k] = float(m <= 2048u ? ar[k] : 0);
      }
      if (sum >= 4096u) ok = 0;
      if (bt < -(int64_t(1) << 31) || bt >= (int64_t(1) << 31)) ok = 0;
      const int64_t bh = bt >> 11;  // floor
      const int64_t bl = bt - bh * 2048;
      const int64_t c1 = bh >> 10;
      const int64_t c0 = bh - c1 * 1024;
      if (!lo_half) {
        v[2 * D] = float(-c1);
        v[2 * D + 1] = float(-c0);
      } else {
        v[2 * D + 2] = float(-bl);
        v[2 * D + 3] = 1.0f;
      }
    } else if (lo_half) {
      v[2 * D + 3] = -1.0f;  // padding slot: s + 1/2 = -1/2, bit 0
    }
    uint4 q0, q1;
    q0.x = h2(v[0], v[1]);
    q0.y = h2(v[2], v[3]);
    q0.z = h2(v[4], v[5]);
    q0.w = h2(v[6], v[7]);
    q1.x = h2(v[8], v[9]);
    q1.y = h2(v[10], v[11]);
    q1.z = h2(v[12], v[13]);
    q1.w = h2(v[14], v[15]);
    *reinterpret_cast<uint4*>(b + kmajor_offset(row, 0)) = q0;
    *reinterpret_cast<uint4*>(b + kmajor_offset(row, 1)) = q1;
  }
  return ok;
}

template <int D, int NC, class Sink>
__global__ void __launch_bounds__(kTThreads)
    pack_tc_kernel(PackArgs pa, Sink sink, TcSpill spill, unsigned int* error, uint32_t polls) {
  constexpr int kL = NC / 2;  // constraint slots (32 or 64)
  constexpr int kCh = kL / 32;
  static_assert(D >= 1 && D <= 4, "d");
  extern __shared__ __align__(16) unsigned char dyn[];
  const uint32_t base = smem_u32(dyn);
  TcShared& sh = *reinterpret_cast<TcShared*>(dyn + (((base + 1023u) & ~1023u) - base));
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int64_t ntiles = (pa.n + kTilePts - 1) / kTilePts;
  const int64_t stride = gridDim.x;
  const uint32_t mbar = smem_u32(&sh.mbar);

  // ---- set-up: TMEM columns, mbarrier, A~ in shared memory ----
  if (warp == 0) {
    tmem_alloc(smem_u32(&sh.tmem), NC);
    fence_before_sync();
  }
  if (tid == 0) mbar_init(mbar, 1);
  const int ok = stage_b_rows<D, NC>(pa, sh.b, tid, kTThreads);
  fence_proxy_async();
  const bool all_ok = __syncthreads_and(ok) != 0;
  fence_after_sync();
  const uint32_t tmem = sh.tmem;
  const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
  const uint64_t bdesc = smem_desc(smem_u32(sh.b), kLBO, kSBO);
  const uint64_t adesc = smem_desc(smem_u32(sh.a), kLBO, kSBO);
  constexpr uint32_t idesc = instr_desc(NC);
  uint32_t phase = 0;
  bool timed_out = false;
  int it = 0;

  // Stages the tile whose points are in `pts` and starts its MMA when the
  // exact split applies; otherwise the tile goes on the spill list. Every
  // thread of the block calls this (it contains the block's one barrier per
  // tile). Returns whether an MMA was started.
  auto stage = [&](int64_t t, const int32_t (&pts)[D]) -> bool {
    const int buf = it & 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const uint32_t m = __reduce_max_sync(0xffffffffu, uabs32(pts[k]));
      if (lane == 0) sh.wmax[buf][warp][k] = m;
    }
    write_row<D>(sh.a, tid, pts);
    fence_proxy_async();
    fence_before_sync();
    // After a wait of any warp ran out, no warp starts another MMA (the
    // decision is the same in every thread of the block).
    const bool stop = __syncthreads_or(timed_out ? 1 : 0) != 0;
    bool in_range = all_ok && !stop;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const uint32_t M = max(max(sh.wmax[buf][0][k], sh.wmax[buf][1][k]),
                             max(sh.wmax[buf][2][k], sh.wmax[buf][3][k]));
      in_range = in_range && M < (1u << 22);
    }
    if (tid == 0) {
      if (in_range) {
        fence_after_sync();
        mma_f16(tmem, adesc, bdesc, idesc);
        mma_commit(mbar);
      } else {
        const unsigned int at = atomicAdd(spill.count, 1u);
        spill.tiles[at] = uint32_t(t);
      }
    }
    ++it;
    return in_range;
  };

  // Pipeline: while the MMA of tile i runs, the block holds the points of tile
  // i+1; right after reading tile i's results from TMEM it stages tile i+1 and
  // starts its MMA, then extracts tile i's sign bits and inserts them (each
  // insertion's table probe is resolved one tile later).
  // The points of tile i+2 are requested during iteration i (a whole
  // iteration of latency cover).
  int64_t tile = blockIdx.x;
  int32_t nxt[D], nxt2[D];
  load_point<D>(pa, tile, ntiles, tid, nxt);
  load_point<D>(pa, tile + stride, ntiles, tid, nxt2);
  bool cur_mma = false;
  if (tile < ntiles) cur_mma = stage(tile, nxt);
#pragma unroll
  for (int k = 0; k < D; ++k) nxt[k] = nxt2[k];
  bool pend = false;
  uint64_t pend_key = 0, pend_cur = 0;
  uint32_t pend_slot = 0;
  for (; tile < ntiles; tile += stride) {
    const int64_t p = tile * kTilePts + tid;
    const bool valid = p < pa.n;
    const int64_t next = tile + stride;
    load_point<D>(pa, next + stride, ntiles, tid, nxt2);
    uint64_t key = 0;
    bool had = false;
    if (cur_mma) {
      if (lane == 0) {
        bool done = false;  // `polls` tries at most; 0 gives up at once
        for (uint32_t spins = 0; spins < polls && !done; ++spins) done = mbar_try_wait(mbar, phase);
        if (!done) timed_out = true;
      }
      __syncwarp();
      timed_out = __shfl_sync(0xffffffffu, timed_out ? 1 : 0, 0) != 0;
      fence_after_sync();
      if (!timed_out) {
        phase ^= 1u;
        had = true;
        // Per 32 constraints: hi and lo results from TMEM, fl(2048 hi + lo)
        // (one rounding of a value that is never 0, so its sign bit is exact),
        // sign bits gathered in four independent chains of 8, then packed.
#pragma unroll
        for (int ch = 0; ch < kCh; ++ch) {
          uint32_t hi[32], lo[32];
          tmem_ld32(taddr + uint32_t(ch * 32), hi);
          tmem_ld32(taddr + uint32_t(kL + ch * 32), lo);
          tmem_wait_ld();
          uint32_t w[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t acc = 0;
#pragma unroll
            for (int j = 8 * g + 7; j >= 8 * g; --j) {
              const float v = fmaf(__uint_as_float(hi[j]), 2048.0f, __uint_as_float(lo[j]));
              acc = __funnelshift_l(__float_as_uint(v), acc, 1);
            }
            w[g] = ~acc;
          }
          const uint32_t word = __byte_perm(__byte_perm(w[0], w[1], 0x0040),
                                            __byte_perm(w[2], w[3], 0x0040), 0x5410);
          key |= uint64_t(word) << (32 * ch);
        }
      } else if (lane == 0 && error) {
        atomicOr(error, kErrTimeout);
      }
    }
    // TMEM and the A tile are free again: stage the next tile now, so that its
    // MMA overlaps the rest of this iteration.
    if (next < ntiles) cur_mma = stage(next, nxt);
#pragma unroll
    for (int k = 0; k < D; ++k) nxt[k] = nxt2[k];
    if (pend) {
      sink.finish(pend_key, pend_slot, pend_cur);
      pend = false;
    }
    if (had && valid) {
      sink.probe(key, pend_slot, pend_cur);
      pend_key = key;
      pend = true;
    }
  }
  if (pend) sink.finish(pend_key, pend_slot, pend_cur);
  if (timed_out) {
    // An MMA that did not complete in time may still write TMEM: wait for it
    // (bounded, with the full limit whatever the test limit) before giving the
    // columns back. No MMA is started after the one given up on.
    for (uint32_t spins = 0; spins < kSpinLimit && !mbar_try_wait(mbar, phase); ++spins) {
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, NC);
  }
}

template <int D, int NC, class Sink>
cudaError_t launch_tc_dn(const PackArgs& pa, const Sink& sink, TcSpill spill, unsigned int* error,
                         cudaStream_t s) {
  // Shared memory is padded so that at most 512 / NC blocks share an SM: their
  // TMEM allocations then always fit.
  constexpr int kPerSm = 512 / NC;
  const size_t smem = std::max(sizeof(TcShared) + 1024, size_t(216 * 1024) / kPerSm);
  auto kern = pack_tc_kernel<D, NC, Sink>;
  cudaError_t err = ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
  if (err != cudaSuccess) return err;
  const int64_t ntiles = (pa.n + kTilePts - 1) / kTilePts;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, int64_t(sm_count()) * kPerSm));
  kern<<<unsigned(grid), kTThreads, smem, s>>>(pa, sink, spill, error, wait_limit(kSpinLimit));
  count_launch();
  return cudaGetLastError();
}

template <class Sink>
cudaError_t launch_tc_any(const PackArgs& pa, const Sink& sink, TcSpill sp, unsigned int* error,
                          cudaStream_t s) {
  const bool two = pa.ell > 32;
  switch (pa.d) {
    case 1: return two ? launch_tc_dn<1, 128>(pa, sink, sp, error, s) : launch_tc_dn<1, 64>(pa, sink, sp, error, s);
    case 2: return two ? launch_tc_dn<2, 128>(pa, sink, sp, error, s) : launch_tc_dn<2, 64>(pa, sink, sp, error, s);
    case 3: return two ? launch_tc_dn<3, 128>(pa, sink, sp, error, s) : launch_tc_dn<3, 64>(pa, sink, sp, error, s);
    case 4: return two ? launch_tc_dn<4, 128>(pa, sink, sp, error, s) : launch_tc_dn<4, 64>(pa, sink, sp, error, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_pack_tc_insert(const PackArgs& pa, const SmallTable& t, uint32_t* spill_tiles,
                                  cudaStream_t s) {
  if (pa.n == 0) return cudaSuccess;
  if (pa.ell > 64) return cudaErrorInvalidValue;
  cudaError_t e =
      launch_tc_any(pa, TcInsert{t}, TcSpill{spill_tiles, &t.ctr->tc_spill}, &t.ctr->error, s);
  if (e != cudaSuccess) return e;
  // Tiles the tensor path could not take, in fp32 with exact re-evaluation.
  PackArgs listed = pa;
  listed.tiles = spill_tiles;
  listed.n_tiles = &t.ctr->tc_spill;
  return launch_pack_insert(listed, t, s);
}

}  // namespace cg
