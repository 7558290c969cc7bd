// Step 1 of the cell-graph construction: sign vectors (§2.1, Figure 1).
//
// Bit i of point p's vector is [a_i . p >= b_i]. The test is exact for every
// int32 point/normal and int64 offset. The kernel decides almost every bit with
// d scalar fp32 FMAs per (point, constraint) -- one 16-byte shared-memory row
// [a_0 .. a_{d-1}, -b] feeds the FMAs of four points -- and falls back to
// 128-bit integer arithmetic only where the fp32 value is too close to zero for
// its rounding error bound to fix the sign. (A packed fma.rn.f32x2 form, two
// points per instruction, is kept as a template option: on GB300 it issues no
// faster, measured at 0.244 against 0.239 ms on the 2^24-point scene.)
//
//   With u = 2^-24, rounded inputs a^ = fl(a_k), p^ = fl(p_k), c^ = fl(-b) and
//   the chain t = fma(a^_{d-1}, p^_{d-1}, ... fma(a^_0, p^_0, c^)), the error
//   |t - (a.p - b)| is at most (gamma_d (1+u)^2 + 2u + u^2) T with
//   T = sum_k |a_k||p_k| + |b| and gamma_d = d u / (1 - d u) (standard
//   floating-point error analysis of an FMA dot product, e.g. Higham,
//   "Accuracy and Stability of Numerical Algorithms", ch. 3). For d <= 4 this is
//   below E = (d + 4) u T.
//
// T is bounded per tile of points from the tile's largest |p_k| (rounded
// upwards). Each constraint row is then scaled by 2^-e, the power of two with
// E 2^-e < 1; the scaling is exact, so |t'| >= 2 proves the sign. |t'| >= 2 is
// exactly "bit 30 of the float is set", which lets one LOP3 accumulate the
// certainty test of two results; a thread whose accumulated bit 30 is clear
// has the uncertain bits of that 32-constraint chunk re-evaluated exactly, by
// the whole warp together (lanes over constraints).
//
// Bits are collected with a funnel shift of the float sign bit (constraints are
// visited from the highest to the lowest index of the chunk), which yields the
// complement of the vector; padding constraints (i >= l) evaluate to -4 and so
// produce 0 bits.
#include <type_traits>

#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;
constexpr int kPts = 4;  // points per thread: two f32x2 pairs
constexpr int kTilePts = kThreads * kPts;

__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  return uint64_t(__float_as_uint(lo)) | (uint64_t(__float_as_uint(hi)) << 32);
}

__device__ __forceinline__ uint32_t uabs32(int32_t v) {
  return v < 0 ? 0u - uint32_t(v) : uint32_t(v);
}
__device__ __forceinline__ uint64_t uabs64(int64_t v) {
  return v < 0 ? 0ull - uint64_t(v) : uint64_t(v);
}

// Exact [a_row . p >= b] with 128-bit accumulation.
template <int D>
__device__ __forceinline__ bool exact_ge(const int32_t* __restrict__ a_row, int64_t b,
                                         const int32_t (&p)[D]) {
  __int128 s = -static_cast<__int128>(b);
#pragma unroll
  for (int k = 0; k < D; ++k) s += static_cast<__int128>(int64_t(a_row[k]) * int64_t(p[k]));
  return s >= 0;
}

// Settles the uncertain bits of one 32-constraint chunk exactly, for every
// lane of the warp whose chunk test failed (some |t'| < 2). The warp works on
// one such lane at a time, lane j taking constraint 32 chunk + j of each of
// that lane's P points (points p_lane0 + L P + q for lane L): it recomputes
// the fp32 value, and where |t'| < 2 decides the bit with 128-bit integer
// arithmetic. w[q] holds, as gathered by the main loop, bit j = 1 when point q
// does not satisfy constraint j. Must be called by the whole warp.
template <int D, int P, int kQ, int R = 2>
__device__ __forceinline__ void settle_uncertain(const PackArgs& pa, const float4* cc, int chunk,
                                                 int64_t p_lane0, bool uncertain,
                                                 uint32_t (&w)[P]) {
  const int lane = threadIdx.x & 31;
  uint32_t todo = __ballot_sync(0xffffffffu, uncertain);
  const int t = chunk * 32 + lane;
  const float* f = reinterpret_cast<const float*>(cc + lane * kQ);
  while (todo) {
    const int L = __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t pL = p_lane0 + int64_t(L) * P;
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      if (pL + q >= pa.n) break;
      int32_t pq[D];
#pragma unroll
      for (int k = 0; k < D; ++k) pq[k] = __ldg(pa.pts + (pL + q) * D + k);
      float acc = f[R * D];
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(f[R * k], __int2float_rn(pq[k]), acc);
      const bool unc = t < pa.ell && fabsf(acc) < 2.0f;
      bool ge = false;
      if (unc) ge = exact_ge<D>(pa.a + int64_t(t) * D, pa.b[t], pq);
      const uint32_t um = __ballot_sync(0xffffffffu, unc);
      const uint32_t gm = __ballot_sync(0xffffffffu, ge);
      if (lane == L) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq)
          if (qq == q) w[qq] = (w[qq] & ~um) | (~gm & um);
      }
    }
  }
}

// Per-constraint scaled coefficients, each repeated R times (R = 2 for the
// f32x2 kernels, 1 for the scalar ones): [a0 .. a0 a1 .. a_{D-1} c .. c]
// padded to whole float4s.
template <int D, int R = 2>
struct Coef {
  static constexpr int kFloats = R * (D + 1);
  static constexpr int kQuads = (kFloats + 3) / 4;
};

// Writes constraint t's coefficients for a tile whose |p_k| <= M[k]. When
// scale is given it receives the factor 2^-e the row was scaled by (0 for a
// padding row or one whose values are all exactly zero).
template <int D, int R = 2>
__device__ void build_coef(const PackArgs& pa, int t, const uint32_t (&M)[D], float4* dst,
                           float* scale = nullptr) {
  if (scale) *scale = 0.0f;
  float v[Coef<D, R>::kQuads * 4];
#pragma unroll
  for (int q = 0; q < Coef<D, R>::kQuads * 4; ++q) v[q] = 0.0f;
  float c;
  if (t >= pa.ell) {
    c = -4.0f;  // padding: certain, negative, bit 0
  } else {
    const int32_t* ar = pa.a + int64_t(t) * D;
    const int64_t bt = pa.b[t];
    float T = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k)
      T = __fmaf_ru(__uint2float_ru(uabs32(ar[k])), __uint2float_ru(M[k]), T);
    T = __fadd_ru(T, __ull2float_ru(uabs64(bt)));
    if (T == 0.0f) {
      c = 4.0f;  // every point of the tile gives a . p - b == 0 exactly: bit 1
    } else {
      const float E = __fmul_ru(T, float(D + 4) * 0x1p-24f);
      int e;
      frexpf(E, &e);  // E = m 2^e, 0.5 <= m < 1, so E 2^-e < 1
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float ak = ldexpf(__int2float_rn(ar[k]), -e);
#pragma unroll
        for (int r = 0; r < R; ++r) v[R * k + r] = ak;
      }
      c = ldexpf(-__ll2float_rn(bt), -e);
      if (scale) *scale = ldexpf(1.0f, -e);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) v[R * D + r] = c;
#pragma unroll
  for (int q = 0; q < Coef<D, R>::kQuads; ++q)
    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Writes the words of each point to keys[n][W] (word_bits 32 or 64).
struct StoreSink {
  void* keys;
  int word_bits;
  int w;  // words per vector in word_bits units
  __device__ void word(int64_t p, int chunk, uint32_t bits, uint32_t& lo_stash, bool last) const {
    if (word_bits == 32) {
      static_cast<uint32_t*>(keys)[p * w + chunk] = bits;
    } else if ((chunk & 1) == 0 && !last) {
      lo_stash = bits;
    } else {
      const uint64_t v = (chunk & 1) ? (uint64_t(lo_stash) | (uint64_t(bits) << 32)) : bits;
      static_cast<uint64_t*>(keys)[p * w + (chunk >> 1)] = v;
    }
  }
  __device__ void done(int64_t, uint64_t) const {}
  static constexpr bool kKeepKey = false;
};

}  // namespace

namespace {

template <int D, class Sink>
__global__ void __launch_bounds__(kThreads)
    pack_kernel(PackArgs pa, Sink sink, int n_chunks, int vec_ok) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kQ = Coef<D>::kQuads;
  float4* coef = reinterpret_cast<float4*>(smem_raw);
  uint32_t* wmax = reinterpret_cast<uint32_t*>(coef + size_t(n_chunks) * 32 * kQ);  // [8][D]
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n = pa.n;
  const int64_t n_tiles = (n + kTilePts - 1) / kTilePts;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTilePts + int64_t(threadIdx.x) * kPts;
    int32_t pi[kPts][D];
    if (vec_ok && p0 + kPts <= n) {
      // kPts * D int32 = D int4, 16-byte aligned (p0 * D * 4 is a multiple of 16).
      const int4* src = reinterpret_cast<const int4*>(pa.pts + p0 * D);
      int32_t tmp[kPts * D];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const int4 v = __ldg(src + q);
        tmp[4 * q] = v.x;
        tmp[4 * q + 1] = v.y;
        tmp[4 * q + 2] = v.z;
        tmp[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < kPts; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) pi[q][k] = tmp[q * D + k];
    } else {
#pragma unroll
      for (int q = 0; q < kPts; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) pi[q][k] = (p0 + q < n) ? __ldg(pa.pts + (p0 + q) * D + k) : 0;
    }

    // Largest |p_k| of the tile, per coordinate.
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < kPts; ++q) m = max(m, uabs32(pi[q][k]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) wmax[warp * D + k] = m;
    }
    __syncthreads();  // also: every thread is done with the previous tile's coef
    {
      uint32_t M[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        uint32_t m = 0;
        for (int w = 0; w < kThreads / 32; ++w) m = max(m, wmax[w * D + k]);
        M[k] = m;
      }
      for (int t = threadIdx.x; t < n_chunks * 32; t += kThreads)
        build_coef<D>(pa, t, M, coef + size_t(t) * kQ);
    }
    __syncthreads();

    uint64_t X[kPts / 2][D];
#pragma unroll
    for (int h = 0; h < kPts / 2; ++h)
#pragma unroll
      for (int k = 0; k < D; ++k)
        X[h][k] = pack2(__int2float_rn(pi[2 * h][k]), __int2float_rn(pi[2 * h + 1][k]));

    uint32_t stash[kPts] = {0, 0, 0, 0};
    uint64_t key[kPts] = {0, 0, 0, 0};
    for (int chunk = 0; chunk < n_chunks; ++chunk) {
      uint32_t w[kPts] = {0, 0, 0, 0};
      uint32_t cert = 0xffffffffu;
      const float4* cc = coef + size_t(chunk) * 32 * kQ;
#pragma unroll 8
      for (int j = 31; j >= 0; --j) {
        float4 q4[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) q4[q] = cc[j * kQ + q];
        const float* f = reinterpret_cast<const float*>(q4);
        uint64_t A[D];
#pragma unroll
        for (int k = 0; k < D; ++k) A[k] = pack2(f[2 * k], f[2 * k + 1]);
        const uint64_t C = pack2(f[2 * D], f[2 * D + 1]);
#pragma unroll
        for (int h = 0; h < kPts / 2; ++h) {
          uint64_t acc = C;
#pragma unroll
          for (int k = 0; k < D; ++k) acc = ffma2(A[k], X[h][k], acc);
          const uint32_t lo = uint32_t(acc);
          const uint32_t hi = uint32_t(acc >> 32);
          w[2 * h] = __funnelshift_l(lo, w[2 * h], 1);
          w[2 * h + 1] = __funnelshift_l(hi, w[2 * h + 1], 1);
          cert &= lo & hi;
        }
      }
      settle_uncertain<D, kPts, kQ>(pa, cc, chunk, p0 - int64_t(lane) * kPts,
                                     !(cert & 0x40000000u), w);
      const bool last = chunk == n_chunks - 1;
#pragma unroll
      for (int q = 0; q < kPts; ++q) {
        const uint32_t bits = ~w[q];
        if (Sink::kKeepKey) {
          if (chunk == 0) key[q] = bits;
          else key[q] |= uint64_t(bits) << 32;
        } else if (p0 + q < n) {
          sink.word(p0 + q, chunk, bits, stash[q], last);
        }
      }
    }
    if (Sink::kKeepKey) {
#pragma unroll
      for (int q = 0; q < kPts; ++q)
        if (p0 + q < n) sink.done(p0 + q, key[q]);
    }
  }
}

// ---------------------------------------------------------------------------
// Fast path for l <= 64 (NCH = 1 or 2 chunks of 32 constraints): 8 points per
// thread (four f32x2 pairs), every loop fully unrolled, no block barrier after
// the set-up. The coefficient rows are built once per block for a bound taken
// from the block's first points (rounded up to a power of two); a warp whose
// points exceed that bound builds its own rows in a private slice of shared
// memory, so the error bound always covers the points it is applied to.
// ---------------------------------------------------------------------------
constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;

__device__ __forceinline__ uint32_t pow2_ceil(uint32_t m) {
  return m <= 1 ? m : (1u << (32 - __clz(m - 1)));
}

template <int D, int P>
__device__ __forceinline__ void load_points(const PackArgs& pa, int64_t p0, int vec_ok,
                                            int32_t (&pi)[P][D]) {
  if (vec_ok && p0 + P <= pa.n) {
    const int4* src = reinterpret_cast<const int4*>(pa.pts + p0 * D);
    int32_t tmp[P * D];
#pragma unroll
    for (int q = 0; q < P * D / 4; ++q) {
      const int4 v = __ldg(src + q);
      tmp[4 * q] = v.x;
      tmp[4 * q + 1] = v.y;
      tmp[4 * q + 2] = v.z;
      tmp[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
      for (int k = 0; k < D; ++k) pi[q][k] = tmp[q * D + k];
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
      for (int k = 0; k < D; ++k)
        pi[q][k] = (p0 + q < pa.n) ? __ldg(pa.pts + (p0 + q) * D + k) : 0;
  }
}

// A warp's whole tile of 32 P points read coalesced (lane l takes 16-byte
// words l, l + 32, ... of the tile) and handed to the lanes through shared
// memory (lane l gets points l P .. l P + P - 1). Reading each lane's P points
// itself puts 16 P D bytes between consecutive lanes' requests; over the host
// link (points read in place from pinned host memory) that pattern measured
// 189 GB/s against 211 GB/s coalesced, and on device memory both are alike.
// A tile that is not whole or not 16-byte aligned takes load_points.
template <int D, int P>
__device__ __forceinline__ void load_points_warp(const PackArgs& pa, int64_t warp_p0, int vec_ok,
                                                 int4* __restrict__ stage,
                                                 int32_t (&pi)[P][D]) {
  constexpr int K = P * D / 4;  // 16-byte words per lane
  static_assert((P * D) % 4 == 0, "whole 16-byte words per lane");
  const int lane = threadIdx.x & 31;
  if (!vec_ok || warp_p0 + 32 * P > pa.n) {
    load_points<D, P>(pa, warp_p0 + lane * P, vec_ok, pi);
    return;
  }
  const int4* src = reinterpret_cast<const int4*>(pa.pts + warp_p0 * D);
#pragma unroll
  for (int k = 0; k < K; ++k) stage[k * 32 + lane] = __ldg(src + k * 32 + lane);
  __syncwarp();
  int32_t tmp[P * D];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int4 v = stage[lane * K + k];
    tmp[4 * k] = v.x;
    tmp[4 * k + 1] = v.y;
    tmp[4 * k + 2] = v.z;
    tmp[4 * k + 3] = v.w;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < P; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) pi[q][k] = tmp[q * D + k];
}

// Words of l <= 64 vectors written to keys (64-bit: one word per point;
// 32-bit: NCH words per point).
template <int NCH>
struct FastStore {
  void* keys;
  int word_bits;
  template <int P>
  __device__ __forceinline__ void finish(int64_t p0, int64_t n, const uint64_t (&key)[P]) const {
    if (word_bits == 64) {
      uint64_t* out = static_cast<uint64_t*>(keys) + p0;
      if (p0 + P <= n && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < P; q += 2)
          *reinterpret_cast<ulonglong2*>(out + q) = make_ulonglong2(key[q], key[q + 1]);
      } else {
#pragma unroll
        for (int q = 0; q < P; ++q)
          if (p0 + q < n) out[q] = key[q];
      }
    } else {
      uint32_t* out = static_cast<uint32_t*>(keys) + p0 * NCH;
#pragma unroll
      for (int q = 0; q < P; ++q)
        if (p0 + q < n) {
#pragma unroll
          for (int c = 0; c < NCH; ++c) out[q * NCH + c] = uint32_t(key[q] >> (32 * c));
        }
    }
  }
};

// Inserts the vectors into the dedup table: the home slots of all of a
// thread's vectors are read first (all loads in flight); only vectors not
// found there take the probing/CAS path.
struct FastInsert {
  SmallTable t;
  template <int P>
  __device__ __forceinline__ void finish(int64_t p0, int64_t n, const uint64_t (&key)[P]) const {
    uint32_t slot[P];
    uint64_t cur[P];
#pragma unroll
    for (int q = 0; q < P; ++q) slot[q] = home_slot(key[q], t.shift);
#pragma unroll
    for (int q = 0; q < P; ++q)
      cur[q] = (p0 + q < n && key[q] != kEmpty) ? t.keys[slot[q]] : 0ull;
#pragma unroll
    for (int q = 0; q < P; ++q)
      if (p0 + q < n && (key[q] == kEmpty || cur[q] != key[q]))
        small_insert_from(t, key[q], slot[q], cur[q]);
  }
};

// One warp tile: the P points of this lane (pi, the first at p0) tested
// against the NCH * 32 constraint rows cf; key[q] receives point q's vector.
// Uncertain chunks are settled exactly by the whole warp (call from all lanes).
template <int D, int NCH, int P, bool F2, int UJ>
__device__ __forceinline__ void eval_tile(const PackArgs& pa, const float4* cf, int64_t p0,
                                          const int32_t (&pi)[P][D], uint64_t (&key)[P],
                                          int c0 = 0) {
  constexpr int R = F2 ? 2 : 1;
  constexpr int kQ = Coef<D, R>::kQuads;
  const int lane = threadIdx.x & 31;
  uint64_t X[P / 2][D];
  float Xs[P][D];
#pragma unroll
  for (int q = 0; q < P; ++q)
#pragma unroll
    for (int k = 0; k < D; ++k) Xs[q][k] = __int2float_rn(pi[q][k]);
#pragma unroll
  for (int h = 0; h < P / 2; ++h)
#pragma unroll
    for (int k = 0; k < D; ++k) X[h][k] = pack2(Xs[2 * h][k], Xs[2 * h + 1][k]);

#pragma unroll 1
  for (int c = 0; c < NCH; ++c) {
    uint32_t w[P];
#pragma unroll
    for (int q = 0; q < P; ++q) w[q] = 0;
    uint32_t cert = 0xffffffffu;
    const float4* cc = cf + (c0 + c) * 32 * kQ;
#pragma unroll UJ
    for (int j = 31; j >= 0; --j) {
      float4 q4[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) q4[q] = cc[j * kQ + q];
      const float* f = reinterpret_cast<const float*>(q4);
      if (F2) {
        uint64_t A[D];
#pragma unroll
        for (int k = 0; k < D; ++k) A[k] = pack2(f[2 * k], f[2 * k + 1]);
        const uint64_t C = pack2(f[2 * D], f[2 * D + 1]);
#pragma unroll
        for (int h = 0; h < P / 2; ++h) {
          uint64_t acc = C;
#pragma unroll
          for (int k = 0; k < D; ++k) acc = ffma2(A[k], X[h][k], acc);
          const uint32_t lo = uint32_t(acc);
          const uint32_t hi = uint32_t(acc >> 32);
          w[2 * h] = __funnelshift_l(lo, w[2 * h], 1);
          w[2 * h + 1] = __funnelshift_l(hi, w[2 * h + 1], 1);
          cert &= lo & hi;
        }
      } else {
#pragma unroll
        for (int h = 0; h < P / 2; ++h) {
          float a0 = f[R * D], a1 = f[R * D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            a0 = fmaf(f[R * k], Xs[2 * h][k], a0);
            a1 = fmaf(f[R * k], Xs[2 * h + 1][k], a1);
          }
          const uint32_t lo = __float_as_uint(a0);
          const uint32_t hi = __float_as_uint(a1);
          w[2 * h] = __funnelshift_l(lo, w[2 * h], 1);
          w[2 * h + 1] = __funnelshift_l(hi, w[2 * h + 1], 1);
          cert &= lo & hi;
        }
      }
    }
    settle_uncertain<D, P, kQ, R>(pa, cc, c0 + c, p0 - int64_t(lane) * P,
                                  !(cert & 0x40000000u), w);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      if (c == 0) key[q] = ~w[q];
      else key[q] |= uint64_t(~w[q]) << 32;
    }
  }
}

// P points per thread (P/2 f32x2 pairs when F2, else scalar FFMA); the
// 32-constraint loop is unrolled UJ times (fully by default: the row offsets
// become immediates, which measured about 4% faster than 8 on l = 64, d = 3).
template <int D, int NCH, class Sink, int P = 4, bool F2 = false, int UJ = 32>
__global__ void __launch_bounds__(kFThreads)
    pack_fast_kernel(PackArgs pa, Sink sink, int vec_ok) {
  constexpr int R = F2 ? 2 : 1;  // scalar FMAs read each coefficient once
  constexpr int kQ = Coef<D, R>::kQuads;
  constexpr int kRows = NCH * 32;
  constexpr int kWarpPts = 32 * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* blk = reinterpret_cast<float4*>(smem_raw);
  float4* priv = blk + (1 + (threadIdx.x >> 5)) * (kRows * kQ);
  __shared__ uint32_t mblk[D];
  __shared__ int4 stage_all[kFWarps][32 * (P * D / 4)];
  griddep_wait();  // the table was cleared by the previous kernel
  griddep_release();
  int4* stage = stage_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t n = pa.n;
  // Work items: all warp tiles, or (when a tile list is given, P == 4) the
  // listed 128-point tiles.
  const bool listed = pa.tiles != nullptr && P == 4;
  if (pa.tiles != nullptr && P != 4) return;
  const int64_t n_all = (n + kWarpPts - 1) / kWarpPts;
  const int64_t n_wt = listed ? (int64_t(*pa.n_tiles) < n_all ? int64_t(*pa.n_tiles) : n_all) : n_all;
  const int64_t stride = int64_t(gridDim.x) * kFWarps;
  int64_t it = int64_t(blockIdx.x) * kFWarps + (threadIdx.x >> 5);

  // Block set-up: bound from every warp's first tile, rows for that bound.
  if (threadIdx.x < D) mblk[threadIdx.x] = 0;
  __syncthreads();
  {
    int32_t pi[P][D];
    const int64_t wt0 = it < n_wt ? (listed ? int64_t(pa.tiles[it]) : it) : n_all;
    load_points_warp<D, P>(pa, wt0 * kWarpPts, vec_ok, stage, pi);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) m = max(m, uabs32(pi[q][k]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) atomicMax(&mblk[k], m);
    }
  }
  __syncthreads();
  uint32_t Mb[D], Mp[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    Mb[k] = pow2_ceil(mblk[k]);
    Mp[k] = 0;
  }
  for (int t = threadIdx.x; t < kRows; t += kFThreads) build_coef<D, R>(pa, t, Mb, blk + t * kQ);
  __syncthreads();
  bool priv_ok = false;

  for (; it < n_wt; it += stride) {
    const int64_t wt = listed ? int64_t(pa.tiles[it]) : it;
    const int64_t p0 = wt * kWarpPts + int64_t(lane) * P;
    int32_t pi[P][D];
    load_points_warp<D, P>(pa, wt * kWarpPts, vec_ok, stage, pi);
    uint32_t mw[D];
    bool fits_blk = true, fits_priv = priv_ok;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) m = max(m, uabs32(pi[q][k]));
      mw[k] = __reduce_max_sync(0xffffffffu, m);
      fits_blk = fits_blk && mw[k] <= Mb[k];
      fits_priv = fits_priv && mw[k] <= Mp[k];
    }
    const float4* cf = blk;
    if (!fits_blk) {
      if (!fits_priv) {
#pragma unroll
        for (int k = 0; k < D; ++k) Mp[k] = pow2_ceil(mw[k]);
        for (int t = lane; t < kRows; t += 32) build_coef<D, R>(pa, t, Mp, priv + t * kQ);
        __syncwarp();
        priv_ok = true;
      }
      cf = priv;
    }
    uint64_t X[P / 2][D];
    float Xs[P][D];
  #pragma unroll
    for (int q = 0; q < P; ++q)
  #pragma unroll
      for (int k = 0; k < D; ++k) Xs[q][k] = __int2float_rn(pi[q][k]);
  #pragma unroll
    for (int h = 0; h < P / 2; ++h)
  #pragma unroll
      for (int k = 0; k < D; ++k) X[h][k] = pack2(Xs[2 * h][k], Xs[2 * h + 1][k]);

      uint64_t key[P];
#pragma unroll 1
    for (int c = 0; c < NCH; ++c) {
      uint32_t w[P];
  #pragma unroll
      for (int q = 0; q < P; ++q) w[q] = 0;
      uint32_t cert = 0xffffffffu;
      const float4* cc = cf + c * 32 * kQ;
  #pragma unroll UJ
      for (int j = 31; j >= 0; --j) {
        float4 q4[kQ];
  #pragma unroll
        for (int q = 0; q < kQ; ++q) q4[q] = cc[j * kQ + q];
        const float* f = reinterpret_cast<const float*>(q4);
        if (F2) {
          uint64_t A[D];
  #pragma unroll
          for (int k = 0; k < D; ++k) A[k] = pack2(f[2 * k], f[2 * k + 1]);
          const uint64_t C = pack2(f[2 * D], f[2 * D + 1]);
  #pragma unroll
          for (int h = 0; h < P / 2; ++h) {
            uint64_t acc = C;
  #pragma unroll
            for (int k = 0; k < D; ++k) acc = ffma2(A[k], X[h][k], acc);
            const uint32_t lo = uint32_t(acc);
            const uint32_t hi = uint32_t(acc >> 32);
            w[2 * h] = __funnelshift_l(lo, w[2 * h], 1);
            w[2 * h + 1] = __funnelshift_l(hi, w[2 * h + 1], 1);
            cert &= lo & hi;
          }
        } else {
  #pragma unroll
          for (int h = 0; h < P / 2; ++h) {
            float a0 = f[R * D], a1 = f[R * D];
  #pragma unroll
            for (int k = 0; k < D; ++k) {
              a0 = fmaf(f[R * k], Xs[2 * h][k], a0);
              a1 = fmaf(f[R * k], Xs[2 * h + 1][k], a1);
            }
            const uint32_t lo = __float_as_uint(a0);
            const uint32_t hi = __float_as_uint(a1);
            w[2 * h] = __funnelshift_l(lo, w[2 * h], 1);
            w[2 * h + 1] = __funnelshift_l(hi, w[2 * h + 1], 1);
            cert &= lo & hi;
          }
        }
      }
      settle_uncertain<D, P, kQ, R>(pa, cc, c, p0 - int64_t(lane) * P, !(cert & 0x40000000u), w);
  #pragma unroll
      for (int q = 0; q < P; ++q) {
        if (c == 0) key[q] = ~w[q];
        else key[q] |= uint64_t(~w[q]) << 32;
      }
    }
    sink.template finish<P>(p0, n, key);
  }
}

template <int D, int NCH, class Sink, int P = 4, bool F2 = false, int UJ = 32>
cudaError_t launch_fast(const PackArgs& pa, const Sink& sink, cudaStream_t s) {
  const size_t smem = size_t(1 + kFWarps) * NCH * 32 * Coef<D, F2 ? 2 : 1>::kQuads * sizeof(float4);
  auto kern = pack_fast_kernel<D, NCH, Sink, P, F2, UJ>;
  int per_sm = 0;
  cudaError_t err =
      blocks_per_sm(reinterpret_cast<const void*>(kern), kFThreads, smem, &per_sm);
  if (err != cudaSuccess) return err;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int64_t n_wt = (pa.n + 32 * P - 1) / (32 * P);
  const int64_t want = (n_wt + kFWarps - 1) / kFWarps;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sm_count()) * per_sm));
  const int vec_ok = (reinterpret_cast<uintptr_t>(pa.pts) % 16) == 0;
  err = launch_dep(kern, dim3(unsigned(grid)), dim3(kFThreads), smem, s, pa, sink, vec_ok);
  count_launch();
  return err;
}

// ---------------------------------------------------------------------------
// Box grid (l <= 64). A placement kernel lays a grid of integer boxes over
// the points, a classification kernel marks, per cell, each constraint as
// holding on the whole cell (`base`), failing on the whole cell, or crossing
// it (listed in `list`, up to kGridList of them); the sign kernel then tests
// each point against its cell's listed constraints only and takes the other
// bits from the cell.
//
// Placement: per axis, G slabs of 2^s integers covering the range of 1,024
// evenly spaced sample points and 1/256 of it on each side; s is raised on
// the axis with the most slabs (the last of equal ones) while axis 0 has more
// than kMaxSweep slabs, the others more than kMaxOther together, or all more
// cells than the workspace holds. The grid's box stays inside the int32 range,
// so a point's slab (p - lo) >> s computed modulo 2^32 is below G exactly
// when the point lies in the box; a point outside it tests every constraint
// in exact integer arithmetic.
//
// Soundness of a cell's classification. The rows are built as for a tile
// with |p_k| <= M_k, M_k the largest |coordinate| of the grid's box, so for
// any real point x of the box the FMA chain at fl(x) is within 1 of
// s (a . x - b) (s = 2^-e the row's scale; the error bound in the header
// covers rounded inputs, in any order of the chain). At the centre c of a
// cell of half-widths h_k every point p of the cell has
// |s (a . p - b) - s (a . c - b)| <= s sum_k |a_k| h_k <= R (R rounded
// upwards), so with v the chain at fl(c): v >= 2 + R proves bit 1 on the
// whole cell and v <= -(2 + R) proves bit 0.
//
// The cells of one column (fixed slabs on axes 1..d-1, every slab g of axis
// 0) are classified together. Along axis 0 the exact value a . p - b moves
// monotonically with g (in the direction of the sign of a_0), so a cell
// proven "bit 1" proves every cell beyond it in that direction, and likewise
// for "bit 0". Per (column, constraint) a thread estimates both boundaries
// from the chain, walks each to the last cell the test still proves, and
// marks the runs in per-column difference words (XOR at each end of a run); a
// prefix XOR along the column then gives every cell's words.
// ---------------------------------------------------------------------------
constexpr int kGridSample = 1024;  // points whose box places the grid
constexpr int kGridThreads = 256;
constexpr int kGridWarps = kGridThreads / 32;
constexpr int kMaxSweep = 256;   // slabs along axis 0 (one warp sweeps a column)
constexpr int kMaxOther = 2048;  // slabs of the other axes together

enum : int { kCellCross = 0, kCellOne = 1, kCellZero = 2 };
constexpr int kGridList = 7;            // crossing constraints listed per cell
constexpr uint32_t kGridOverflow = 255;  // count byte of a cell with more

// Centre of slab g (2^s integers from lo + g 2^s), rounded once to fp32:
// twice the centre is an integer, rounded to fp32 and halved exactly.
__device__ __forceinline__ float slab_centre(int32_t lo, int s, int g) {
  const int64_t c2 = 2 * (int64_t(lo) + (int64_t(g) << s)) + ((int64_t(1) << s) - 1);
  return 0.5f * __ll2float_rn(c2);
}

// The test at a cell centre whose axis-0 coordinate is x0, c1 the chain over
// the other axes (started from the row's constant).
__device__ __forceinline__ int cell_test(float f0, float x0, float c1, float q) {
  const float v = fmaf(f0, x0, c1);
  return v >= q ? kCellOne : (v <= -q ? kCellZero : kCellCross);
}

__device__ __forceinline__ int clamp_slab(float g, int lo, int hi) {
  g = fminf(fmaxf(g, float(lo)), float(hi));  // also maps NaN to lo
  return int(g);
}

__device__ __forceinline__ int64_t slabs_for(int64_t want, int s) {
  return (want + (int64_t(1) << s) - 1) >> s;
}

// Runs of the cells of one column (axis-0 slabs [0, G0)) on which the test
// proves bit 1 ([*one_lo, *one_hi)) and the run on which the constraint may
// cross ([*cr_lo, *cr_hi)); the rest is proven bit 0. cen0: the axis-0 slab
// centres; c1: the chain over the other axes.
__device__ __forceinline__ void column_runs(const float* cen0, int G0, float f0, float rf0,
                                            float c1, float q, float x00, float rw0,
                                            int* one_lo, int* one_hi, int* cr_lo, int* cr_hi) {
  auto test = [&](int gg) { return cell_test(f0, cen0[gg], c1, q); };
  *one_lo = *one_hi = *cr_lo = *cr_hi = 0;
  if (f0 == 0.0f) {
    const int t = test(0);  // the same value on every cell of the column
    if (t == kCellOne) *one_hi = G0;
    else if (t == kCellCross) *cr_hi = G0;
    return;
  }
  // estimates only: the walks below decide
  const float g_one = ((q - c1) * rf0 - x00) * rw0;    // where v = q
  const float g_zero = ((-q - c1) * rf0 - x00) * rw0;  // where v = -q
  if (f0 > 0.0f) {
    // bit 1 on [a, G0): the first proven cell at or after the estimate, then
    // back while the cell before is proven too
    int a = clamp_slab(ceilf(g_one), 0, G0);
    while (a < G0 && test(a) != kCellOne) ++a;
    while (a > 0 && a < G0 && test(a - 1) == kCellOne) --a;
    // bit 0 on [0, z + 1)
    int z = clamp_slab(floorf(g_zero), -1, G0 - 1);
    while (z >= 0 && test(z) != kCellZero) --z;
    while (z >= 0 && z < G0 - 1 && test(z + 1) == kCellZero) ++z;
    *one_lo = a, *one_hi = G0;
    *cr_lo = z + 1, *cr_hi = max(a, z + 1);
  } else {
    // bit 1 on [0, a + 1)
    int a = clamp_slab(floorf(g_one), -1, G0 - 1);
    while (a >= 0 && test(a) != kCellOne) --a;
    while (a >= 0 && a < G0 - 1 && test(a + 1) == kCellOne) ++a;
    // bit 0 on [z, G0)
    int z = clamp_slab(ceilf(g_zero), 0, G0);
    while (z < G0 && test(z) != kCellZero) ++z;
    while (z > 0 && z < G0 && test(z - 1) == kCellZero) --z;
    *one_lo = 0, *one_hi = a + 1;
    *cr_lo = a + 1, *cr_hi = max(z, a + 1);
  }
}

// A cell's crossing constraints: indices in bytes 0 .. kGridList - 1, their
// count in byte 7 (kGridOverflow when there are more: the point then tests
// every constraint).
__device__ __forceinline__ uint64_t grid_list(uint64_t cross) {
  if (__popcll(cross) > kGridList) return uint64_t(kGridOverflow) << 56;
  uint64_t list = 0;
  uint32_t t = 0;
  while (cross) {
    const int j = __ffsll(cross) - 1;
    cross &= cross - 1;
    list |= uint64_t(j) << (8 * t);
    ++t;
  }
  return list | (uint64_t(t) << 56);
}

constexpr int kPlaceThreads = 1024;
static_assert(kMaxSweep + kMaxOther <= kGridMaxCentres, "centre table");

// Placement (one block): the box of the sample, the slabs per axis, the slab
// centres, the rows for the grid's box and each row's threshold q = 2 + R,
// all written to g.geom for the classification and the sign kernel.
template <int D, int NCH>
__global__ void __launch_bounds__(kPlaceThreads) grid_place_kernel(PackArgs pa, PackGrid g) {
  constexpr int kQ = Coef<D, 1>::kQuads;
  constexpr int kRows = NCH * 32;
  static_assert(kQ <= kGridMaxQuads && kRows <= kGridMaxRows, "grid rows");
  __shared__ int32_t red[2][kPlaceThreads / 32][D];
  __shared__ int32_t geo_lo[D], geo_sh[D], geo_n[D], cen_off[D];
  // Launched plainly after the stream's earlier kernels (the previous build's
  // reads of the grid are over); with a programmatic launch this wait would
  // order it.
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n = pa.n;
  GridGeom* geo = g.geom;

  int32_t mn[D], mx[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    mn[k] = INT32_MAX;
    mx[k] = INT32_MIN;
  }
  for (int j = threadIdx.x; j < kGridSample; j += kPlaceThreads) {
    const int64_t i = n <= kGridSample ? int64_t(j) : int64_t(j) * (n - 1) / (kGridSample - 1);
    if (i < n) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int32_t v = __ldg(pa.pts + i * D + k);
        mn[k] = min(mn[k], v);
        mx[k] = max(mx[k], v);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    mn[k] = __reduce_min_sync(0xffffffffu, mn[k]);
    mx[k] = __reduce_max_sync(0xffffffffu, mx[k]);
    if (lane == 0) {
      red[0][warp][k] = mn[k];
      red[1][warp][k] = mx[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Slabs: raise s on the axis with the most slabs (of equal counts, the
    // last: axis 0, the one a warp sweeps, stays finest) while axis 0 has more
    // than kMaxSweep, the others more than kMaxOther together, or all more
    // than the budget. Axes over their own limit are brought under it
    // directly: the rule raises them first, one after the other, whatever
    // the order.
    int64_t first[D], ext[D], want[D], cnt[D];
    int s[D];
    for (int k = 0; k < D; ++k) {
      int32_t a = INT32_MAX, b = INT32_MIN;
      for (int w = 0; w < kPlaceThreads / 32; ++w) {
        a = min(a, red[0][w][k]);
        b = max(b, red[1][w][k]);
      }
      if (a > b) a = b = 0;
      first[k] = a;
      ext[k] = int64_t(b) - int64_t(a) + 1;
      want[k] = min(ext[k] + ext[k] / 128 + 2, int64_t(1) << 32);
      s[k] = 0;
      const int64_t lim = k == 0 ? kMaxSweep : kMaxOther;
      while (slabs_for(want[k], s[k]) > lim) ++s[k];
      cnt[k] = slabs_for(want[k], s[k]);
    }
    const uint64_t budget = uint64_t(1) << g.total_bits;
    for (int guard = 0; guard < 32 * D; ++guard) {
      int64_t other = 0;
      uint64_t prod = 1;
      bool over = false;
      for (int k = 0; k < D; ++k) {
        if (k > 0) other += cnt[k];
        prod *= uint64_t(cnt[k]);  // counts <= 2^32, prod <= budget before: no overflow
        if (prod > budget) over = true, prod = budget + 1;
      }
      int kk = -1;
      const int k0 = other > kMaxOther ? 1 : 0;
      if (cnt[0] > kMaxSweep) kk = 0;
      else if (other > kMaxOther || over)
        for (int k = k0; k < D; ++k)
          if (s[k] < 31 && (kk < 0 || cnt[k] >= cnt[kk])) kk = k;  // ties: the last axis
      if (kk < 0) break;
      ++s[kk];
      cnt[kk] = slabs_for(want[kk], s[kk]);
    }
    int off = 0;
    for (int k = 0; k < D; ++k) {
      int64_t span = cnt[k] << s[k];
      if (span > (int64_t(1) << 32)) {
        cnt[k] = (int64_t(1) << 32) >> s[k];
        span = cnt[k] << s[k];
      }
      int64_t lo = first[k] - (span - ext[k]) / 2;
      if (lo < int64_t(INT32_MIN)) lo = INT32_MIN;
      if (lo + span > (int64_t(1) << 31)) lo = (int64_t(1) << 31) - span;
      geo_lo[k] = int32_t(lo);
      geo_sh[k] = s[k];
      geo_n[k] = int32_t(cnt[k]);
      cen_off[k] = off;
      off += int(cnt[k]);
      geo->lo[k] = int32_t(lo);
      geo->shift[k] = s[k];
      geo->count[k] = int32_t(cnt[k]);
      geo->cen_off[k] = cen_off[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < D; ++k)
    for (int t = threadIdx.x; t < geo_n[k]; t += kPlaceThreads)
      geo->cen[cen_off[k] + t] = slab_centre(geo_lo[k], geo_sh[k], t);
  uint32_t M[D];
  float hh[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int64_t lo = geo_lo[k];
    const int64_t hi = lo + (int64_t(geo_n[k]) << geo_sh[k]) - 1;
    M[k] = max(uabs32(int32_t(lo)), uabs32(int32_t(hi)));
    hh[k] = 0.5f * __ull2float_ru((1ull << geo_sh[k]) - 1ull);
  }
  for (int t = threadIdx.x; t < kRows; t += kPlaceThreads) {
    float sc;
    build_coef<D, 1>(pa, t, M, geo->rows + t * kQ, &sc);
    float R = 0.0f;
    if (sc != 0.0f) {
      const int32_t* ar = pa.a + int64_t(t) * D;
#pragma unroll
      for (int k = 0; k < D; ++k) R = __fmaf_ru(__uint2float_ru(uabs32(ar[k])), hh[k], R);
      R = __fmul_ru(R, sc);
    }
    geo->qlim[t] = __fadd_ru(2.0f, R);
  }
}

// Classification: each warp takes whole columns: lane j takes constraints j
// and j + 32, marks its runs in the warp's difference words, and the warp
// turns them into the column's cell words (prefix XOR) and writes them.
template <int D, int NCH>
__global__ void __launch_bounds__(kGridThreads) grid_setup_kernel(PackArgs pa, PackGrid g) {
  constexpr int kQ = Coef<D, 1>::kQuads;
  constexpr int kRows = NCH * 32;
  constexpr int kWords = 2 * NCH;  // base words, then cross words
  __shared__ float4 rows[kRows * kQ];
  __shared__ float qlim[kRows];
  __shared__ int32_t geo_lo[D], geo_sh[D], geo_n[D], cen_off[D];
  __shared__ float cen[kMaxSweep + kMaxOther];  // slab centres, axis 0 first
  __shared__ uint32_t diff_all[kGridWarps][kWords][kMaxSweep + 1];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const GridGeom* geo = g.geom;
  if (threadIdx.x < D) {
    geo_lo[threadIdx.x] = geo->lo[threadIdx.x];
    geo_sh[threadIdx.x] = geo->shift[threadIdx.x];
    geo_n[threadIdx.x] = geo->count[threadIdx.x];
    cen_off[threadIdx.x] = geo->cen_off[threadIdx.x];
  }
  for (int t = threadIdx.x; t < kRows * kQ; t += kGridThreads) rows[t] = geo->rows[t];
  for (int t = threadIdx.x; t < kRows; t += kGridThreads) qlim[t] = geo->qlim[t];
  __syncthreads();
  int n_cen = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) n_cen += geo_n[k];
  for (int t = threadIdx.x; t < n_cen; t += kGridThreads) cen[t] = geo->cen[t];
  __syncthreads();

  // 3. Columns, one warp each.
  const int G0 = geo_n[0];
  uint32_t n_cols = 1;
#pragma unroll
  for (int k = 1; k < D; ++k) n_cols *= uint32_t(geo_n[k]);
  const float x00 = cen[0];
  const float rw0 = ldexpf(1.0f, -geo_sh[0]);  // 1 / slab width (exact)
  float f0[NCH], rf0[NCH], q[NCH];
#pragma unroll
  for (int h = 0; h < NCH; ++h) {
    const float* f = reinterpret_cast<const float*>(rows + (32 * h + lane) * kQ);
    f0[h] = f[0];
    rf0[h] = f0[h] != 0.0f ? 1.0f / f0[h] : 0.0f;
    q[h] = qlim[32 * h + lane];
  }
  uint32_t(*diff)[kMaxSweep + 1] = diff_all[warp];
  const int per = (G0 + 31) / 32;
  for (uint32_t col = blockIdx.x * kGridWarps + warp; col < n_cols;
       col += gridDim.x * kGridWarps) {
#pragma unroll
    for (int w = 0; w < kWords; ++w)
      for (int x = lane; x <= G0; x += 32) diff[w][x] = 0;
    __syncwarp();
    int gk[D];
    {
      uint32_t rest = col;
#pragma unroll
      for (int k = 1; k < D; ++k) {
        const uint32_t nxt = k + 1 < D ? rest / uint32_t(geo_n[k]) : 0u;
        gk[k] = int(rest - nxt * uint32_t(geo_n[k]));
        rest = nxt;
      }
    }
#pragma unroll
    for (int h = 0; h < NCH; ++h) {
      const int i = 32 * h + lane;
      if (i >= pa.ell) continue;
      const float* f = reinterpret_cast<const float*>(rows + i * kQ);
      float c1 = f[D];
#pragma unroll
      for (int k = 1; k < D; ++k) c1 = fmaf(f[k], cen[cen_off[k] + gk[k]], c1);
      int one_lo, one_hi, cr_lo, cr_hi;
      column_runs(cen, G0, f0[h], rf0[h], c1, q[h], x00, rw0, &one_lo, &one_hi, &cr_lo, &cr_hi);
      const uint32_t bit = 1u << lane;
      if (one_lo < one_hi) {
        atomicXor(&diff[h][one_lo], bit);
        atomicXor(&diff[h][one_hi], bit);
      }
      if (cr_lo < cr_hi) {
        atomicXor(&diff[NCH + h][cr_lo], bit);
        atomicXor(&diff[NCH + h][cr_hi], bit);
      }
    }
    __syncwarp();
    // prefix XOR along the column, word array by word array
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
      uint32_t* a = diff[w];
      const int b0 = lane * per;
      uint32_t acc = 0;
      for (int t = 0; t < per; ++t)
        if (b0 + t < G0) {
          acc ^= a[b0 + t];
          a[b0 + t] = acc;
        }
      uint32_t x = acc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x ^= y;
      }
      const uint32_t before = x ^ acc;
      for (int t = 0; t < per; ++t)
        if (b0 + t < G0) a[b0 + t] ^= before;
    }
    __syncwarp();
    // the column's cells (axis 0 fastest: cell g0 + G0 * column), the
    // crossing constraints as a list of up to kGridList indices
    for (int x = lane; x < G0; x += 32) {
      uint64_t base = diff[0][x];
      uint64_t cross = diff[NCH][x];
      if (NCH == 2) {
        base |= uint64_t(diff[1][x]) << 32;
        cross |= uint64_t(diff[3][x]) << 32;
      }
      g.cells[size_t(x) + size_t(G0) * col] = GridCell{base, grid_list(cross)};
    }
    __syncwarp();
  }
  griddep_release();
}

// Exact decision of the listed crossing constraints of one point whose fp32
// value was too close to zero (|t'| < 2): the values recomputed, the
// uncertain ones settled in 128-bit integers.
template <int D, int kQ>
__device__ __noinline__ uint64_t grid_settle(const PackArgs& pa, const float4* rows, uint64_t list,
                                             float x0, float x1, float x2, float x3, int32_t p0,
                                             int32_t p1, int32_t p2, int32_t p3, uint64_t kw) {
  const float xa[4] = {x0, x1, x2, x3};
  const int32_t pa4[4] = {p0, p1, p2, p3};
  int32_t p[D];
#pragma unroll
  for (int k = 0; k < D; ++k) p[k] = pa4[k];
  const uint32_t c = uint32_t(list >> 56);
  for (uint32_t t = 0; t < c; ++t) {
    const int j = int((list >> (8 * t)) & 63u);
    const float* f = reinterpret_cast<const float*>(rows + j * kQ);
    float v = f[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v = fmaf(f[k], xa[k], v);
    if (!(__float_as_uint(v) & 0x40000000u)) {
      const bool ge = exact_ge<D>(pa.a + int64_t(j) * D, pa.b[j], p);
      kw = ge ? (kw | (1ull << j)) : (kw & ~(1ull << j));
    }
  }
  return kw;
}

// [a_t . p >= b_t] for every constraint t < l: in 128-bit integers for a
// point outside the grid (`exact`), else with the rows and the exact decision
// of uncertain values (a cell with more than kGridList crossing constraints).
template <int D, int kQ>
__device__ __noinline__ uint64_t grid_all(const PackArgs& pa, const float4* rows, bool exact,
                                          int32_t p0, int32_t p1, int32_t p2, int32_t p3) {
  const int32_t pa4[4] = {p0, p1, p2, p3};
  int32_t p[D];
  float x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    p[k] = pa4[k];
    x[k] = __int2float_rn(p[k]);
  }
  uint64_t kw = 0;
  for (int t = 0; t < pa.ell; ++t) {
    bool ge;
    if (exact) {
      ge = exact_ge<D>(pa.a + int64_t(t) * D, pa.b[t], p);
    } else {
      const float* f = reinterpret_cast<const float*>(rows + t * kQ);
      float v = f[D];
#pragma unroll
      for (int k = 0; k < D; ++k) v = fmaf(f[k], x[k], v);
      ge = (__float_as_uint(v) & 0x40000000u) ? v >= 0.0f
                                               : exact_ge<D>(pa.a + int64_t(t) * D, pa.b[t], p);
    }
    if (ge) kw |= 1ull << t;
  }
  return kw;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Point tiles in flight per warp (two at d = 4, whose tiles are larger).
template <int D>
struct GridStages {
  static constexpr int value = D == 4 ? 2 : 3;
};

// Sign + insert with the grid. Per warp, 128-point tiles stream through a
// ring of GridStages shared-memory slots filled by cp.async (whole tiles of
// 16-byte aligned points; others are read directly), so the points of the
// next tiles are on their way while one is evaluated. Per point: its cell's
// entry (one 16-byte load from the L2-resident grid) and a loop over the
// cell's listed crossing constraints, with one set of rows built for the
// grid's box;
// the previous tile's vectors are inserted while this tile's entries load.
template <int D, int NCH, class Sink>
__global__ void __launch_bounds__(kFThreads, 4)
    pack_grid_kernel(PackArgs pa, Sink sink, PackGrid g, int vec_ok) {
  constexpr int P = 4;
  constexpr int kQ = Coef<D, 1>::kQuads;
  constexpr int kRows = NCH * 32;
  constexpr int kWarpPts = 32 * P;
  constexpr int K = P * D / 4;  // 16-byte words per lane per tile
  constexpr int kStages = GridStages<D>::value;
  __shared__ float4 rows[kRows * kQ];
  __shared__ int4 ring_all[kFWarps][kStages][32 * K];
  griddep_wait();  // the table cleared and the grid classified
  griddep_release();
  int4(*ring)[32 * K] = ring_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t n = pa.n;
  uint32_t glo[D], gsh[D], gcnt[D], gmul[D];
  {
    uint32_t mul = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      glo[k] = uint32_t(g.geom->lo[k]);
      gsh[k] = uint32_t(g.geom->shift[k]);
      gcnt[k] = uint32_t(g.geom->count[k]);
      gmul[k] = mul;
      mul *= gcnt[k];
    }
  }
  // the rows the placement built for the grid's box
  for (int t = threadIdx.x; t < kRows * kQ; t += kFThreads) rows[t] = g.geom->rows[t];
  __syncthreads();

  const int64_t n_wt = (n + kWarpPts - 1) / kWarpPts;
  const int64_t stride = int64_t(gridDim.x) * kFWarps;
  const int64_t it0 = int64_t(blockIdx.x) * kFWarps + (threadIdx.x >> 5);
  auto whole = [&](int64_t t) { return vec_ok && (t + 1) * kWarpPts <= n; };
  // Every call commits one group (empty past the end), so that waiting for
  // all but the newest kStages - 1 groups always means "this tile".
  auto issue = [&](int64_t t, int slot) {
    if (t < n_wt && whole(t)) {
      const int4* src = reinterpret_cast<const int4*>(pa.pts + t * kWarpPts * D);
#pragma unroll
      for (int k = 0; k < K; ++k) cp_async16(&ring[slot][k * 32 + lane], src + k * 32 + lane);
    }
    cp_async_commit();
  };
  int64_t t_issue = it0;
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    issue(t_issue, st);
    t_issue += stride;
  }
  int slot = 0;
  bool have_prev = false;
  int64_t p0_prev = 0;
  uint64_t key_prev[P];
  for (int64_t it = it0; it < n_wt; it += stride) {
    issue(t_issue, (slot + kStages - 1) % kStages);
    t_issue += stride;
    cp_async_wait<kStages - 1>();
    __syncwarp();
    const int64_t p0 = it * kWarpPts + int64_t(lane) * P;
    int32_t pi[P][D];
    if (whole(it)) {
      int32_t tmp[P * D];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int4 v = ring[slot][lane * K + k];
        tmp[4 * k] = v.x;
        tmp[4 * k + 1] = v.y;
        tmp[4 * k + 2] = v.z;
        tmp[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < P; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) pi[q][k] = tmp[q * D + k];
    } else {
      load_points<D, P>(pa, p0, vec_ok, pi);
    }
    __syncwarp();  // the slot is refilled by the next iteration's issue
    GridCell e[P];
    bool outside[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      bool in = p0 + q < n;
      uint32_t idx = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const uint32_t gk = (uint32_t(pi[q][k]) - glo[k]) >> gsh[k];
        in = in && gk < gcnt[k];
        idx += gk * gmul[k];
      }
      outside[q] = !in && p0 + q < n;
      e[q] = in ? g.cells[idx] : GridCell{0ull, 0ull};  // count 0: nothing listed
    }
    if (have_prev) sink.template finish<P>(p0_prev, n, key_prev);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      float x[D];
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = __int2float_rn(pi[q][k]);
      const uint64_t list = e[q].list;
      const uint32_t c = uint32_t(list >> 56);
      uint32_t klo = uint32_t(e[q].base), khi = uint32_t(e[q].base >> 32);
      uint32_t cert = 0xffffffffu;
      uint32_t w0 = uint32_t(list), w1 = uint32_t(list >> 32);
      for (uint32_t t = 0; t < c && c != kGridOverflow; ++t) {
        const uint32_t j = w0 & 63u;
        w0 = __funnelshift_r(w0, w1, 8);
        w1 >>= 8;
        float4 q4[kQ];
#pragma unroll
        for (int r = 0; r < kQ; ++r) q4[r] = rows[j * kQ + r];
        const float* f = reinterpret_cast<const float*>(q4);
        float v = f[D];
#pragma unroll
        for (int k = 0; k < D; ++k) v = fmaf(f[k], x[k], v);
        const uint32_t u = __float_as_uint(v);
        const uint32_t r = (1u << (j & 31u)) & ~uint32_t(int32_t(u) >> 31);
        if (NCH == 1 || j < 32) klo |= r;
        else khi |= r;
        cert &= u;
      }
      uint64_t kw = klo | (uint64_t(khi) << 32);
      if (!(cert & 0x40000000u))
        kw = grid_settle<D, kQ>(pa, rows, list, x[0], x[D > 1 ? 1 : 0], x[D > 2 ? 2 : 0],
                                x[D > 3 ? 3 : 0], pi[q][0], pi[q][D > 1 ? 1 : 0],
                                pi[q][D > 2 ? 2 : 0], pi[q][D > 3 ? 3 : 0], kw);
      if (outside[q] || c == kGridOverflow)
        kw = grid_all<D, kQ>(pa, rows, outside[q], pi[q][0], pi[q][D > 1 ? 1 : 0],
                             pi[q][D > 2 ? 2 : 0], pi[q][D > 3 ? 3 : 0]);
      key_prev[q] = kw;
    }
    p0_prev = p0;
    have_prev = true;
    slot = slot + 1 == kStages ? 0 : slot + 1;
  }
  if (have_prev) sink.template finish<P>(p0_prev, n, key_prev);
  cp_async_wait<0>();
}

template <int D, int NCH>
cudaError_t launch_grid_setup_dn(const PackArgs& pa, const PackGrid& g, cudaStream_t s) {
  // One warp per column; at most 2^total_bits columns (the placement is made
  // on the device).
  const int64_t want = ((int64_t(1) << g.total_bits) + kGridWarps - 1) / kGridWarps;
  const int64_t sg = std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sm_count()) * 2));
  // Plain launches (the kernels' griddepcontrol calls are then no-ops): with
  // programmatic dependent launch the persistent sign kernel after it measured
  // 0.1 ms slower per build (0.39 against 0.27 ms per planes_3d step).
  grid_place_kernel<D, NCH><<<1, kPlaceThreads, 0, s>>>(pa, g);
  grid_setup_kernel<D, NCH><<<unsigned(sg), kGridThreads, 0, s>>>(pa, g);
  count_launch(2);
  return cudaGetLastError();
}

template <int D, int NCH>
cudaError_t launch_grid_dn(const PackArgs& pa, const SmallTable& t, const PackGrid& g,
                           cudaStream_t s) {
  auto kern = pack_grid_kernel<D, NCH, FastInsert>;
  int per_sm = 0;
  cudaError_t err = blocks_per_sm(reinterpret_cast<const void*>(kern), kFThreads, 0, &per_sm);
  if (err != cudaSuccess) return err;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int64_t n_wt = (pa.n + 127) / 128;
  const int64_t want = (n_wt + kFWarps - 1) / kFWarps;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sm_count()) * per_sm));
  const int vec_ok = (reinterpret_cast<uintptr_t>(pa.pts) % 16) == 0;
  kern<<<unsigned(grid), kFThreads, 0, s>>>(pa, FastInsert{t}, g, vec_ok);
  count_launch();
  return cudaGetLastError();
}

// Many scenes of l <= 64 in one launch (batches): warp w takes the contiguous
// tile range [w per, (w + 1) per) of the batch's tile numbering; per tile it
// finds the scene (tiles are visited in increasing order, so the scene index
// only moves forward), reads the 128 points coalesced, and rebuilds its
// private constraint rows when the scene changes or the tile's coordinates
// exceed the bound the rows were built for. Evaluation and insertion are the
// single-scene kernel's (eval_tile, FastInsert). With W > 0 (scenes of
// 64 < l <= 64 W) the W words of each vector are evaluated two chunks at a
// time and written to the scene's keys64 instead of inserted.
template <int D, int NCH, int W = 0>
__global__ void __launch_bounds__(kFThreads)
    pack_seg_kernel(const SegPackScene* __restrict__ sc, int n_scenes, uint64_t total_tiles) {
  constexpr int P = 4;
  constexpr int kQ = Coef<D, 1>::kQuads;
  constexpr int kRows = (W > 0 ? 2 * W : NCH) * 32;
  constexpr int kWarpPts = 32 * P;
  __shared__ float4 rows_all[kFWarps][kRows * kQ];
  __shared__ int4 stage_all[kFWarps][32 * (P * D / 4)];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4* rows = rows_all[warp];
  int4* stage = stage_all[warp];
  const uint64_t nw = uint64_t(gridDim.x) * kFWarps;
  const uint64_t per = (total_tiles + nw - 1) / nw;
  const uint64_t g0 = (uint64_t(blockIdx.x) * kFWarps + warp) * per;
  const uint64_t g1 = min(total_tiles, g0 + per);
  if (g0 >= g1) return;
  int s = 0;  // last scene whose first tile is <= g0
  {
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sc[mid].tile0 <= g0) lo = mid;
      else hi = mid - 1;
    }
    s = lo;
  }
  int built = -1;  // scene of the rows in shared memory
  uint32_t Mb[D];
#pragma unroll
  for (int k = 0; k < D; ++k) Mb[k] = 0;
  for (uint64_t g = g0; g < g1; ++g) {
    while (s + 1 < n_scenes && sc[s + 1].tile0 <= g) ++s;
    const SegPackScene& S = sc[s];
    const PackArgs pa{S.pts, S.n, D, S.a, S.b, S.ell};
    const int64_t wp0 = int64_t(g - S.tile0) * kWarpPts;
    const int vec_ok = (reinterpret_cast<uintptr_t>(S.pts) % 16) == 0;
    int32_t pi[P][D];
    load_points_warp<D, P>(pa, wp0, vec_ok, stage, pi);
    bool fits = built == s;
    uint32_t mw[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) m = max(m, uabs32(pi[q][k]));
      mw[k] = __reduce_max_sync(0xffffffffu, m);
      fits = fits && mw[k] <= Mb[k];
    }
    if (!fits) {
#pragma unroll
      for (int k = 0; k < D; ++k) Mb[k] = pow2_ceil(mw[k]);
      __syncwarp();  // every lane is done with the previous rows
      for (int t = lane; t < kRows; t += 32) build_coef<D, 1>(pa, t, Mb, rows + t * kQ);
      __syncwarp();
      built = s;
    }
    const int64_t p0 = wp0 + int64_t(lane) * P;
    uint64_t key[P];
    if (W == 0) {
      eval_tile<D, NCH, P, false, 32>(pa, rows, p0, pi, key);
      FastInsert{S.t}.template finish<P>(p0, S.n, key);
    } else {
#pragma unroll 1
      for (int q = 0; q < W; ++q) {
        eval_tile<D, 2, P, false, 32>(pa, rows, p0, pi, key, 2 * q);
#pragma unroll
        for (int k = 0; k < P; ++k)
          if (p0 + k < S.n) S.keys64[uint64_t(p0 + k) * W + q] = key[k];
      }
    }
  }
}

template <int D, int NCH, int W = 0>
cudaError_t launch_seg_dn(const SegPackScene* scenes, int n_scenes, uint64_t total_tiles,
                          cudaStream_t s) {
  auto kern = pack_seg_kernel<D, NCH, W>;
  int per_sm = 0;
  cudaError_t err = blocks_per_sm(reinterpret_cast<const void*>(kern), kFThreads, 0, &per_sm);
  if (err != cudaSuccess) return err;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const uint64_t want = (total_tiles + kFWarps - 1) / kFWarps;
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(sm_count()) * per_sm));
  kern<<<unsigned(grid), kFThreads, 0, s>>>(scenes, n_scenes, total_tiles);
  count_launch();
  return cudaGetLastError();
}

template <class SinkFor>
cudaError_t launch_fast_any(const PackArgs& pa, SinkFor make, cudaStream_t s) {
  const bool two = pa.ell > 32;
  switch (pa.d) {
    case 1: return two ? launch_fast<1, 2>(pa, make.template get<2>(), s)
                       : launch_fast<1, 1>(pa, make.template get<1>(), s);
    case 2: return two ? launch_fast<2, 2>(pa, make.template get<2>(), s)
                       : launch_fast<2, 1>(pa, make.template get<1>(), s);
    case 3: return two ? launch_fast<3, 2>(pa, make.template get<2>(), s)
                       : launch_fast<3, 1>(pa, make.template get<1>(), s);
    case 4: return two ? launch_fast<4, 2>(pa, make.template get<2>(), s)
                       : launch_fast<4, 1>(pa, make.template get<1>(), s);
    default: return cudaErrorInvalidValue;
  }
}

struct MakeStore {
  void* keys;
  int word_bits;
  template <int NCH>
  FastStore<NCH> get() const { return FastStore<NCH>{keys, word_bits}; }
};

struct MakeInsert {
  SmallTable t;
  template <int NCH>
  FastInsert get() const { return FastInsert{t}; }
};

template <int D, class Sink>
cudaError_t launch_d(const PackArgs& pa, const Sink& sink, cudaStream_t s) {
  if (pa.n == 0) return cudaSuccess;
  const int n_chunks = (pa.ell + 31) / 32;
  const size_t smem = size_t(n_chunks) * 32 * Coef<D>::kQuads * sizeof(float4) +
                      sizeof(uint32_t) * (kThreads / 32) * D;
  auto kern = pack_kernel<D, Sink>;
  int per_sm = 0;
  cudaError_t err = blocks_per_sm(reinterpret_cast<const void*>(kern), kThreads, smem, &per_sm);
  if (err != cudaSuccess) return err;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int64_t n_tiles = (pa.n + kTilePts - 1) / kTilePts;
  const int64_t grid = std::min<int64_t>(n_tiles, int64_t(sm_count()) * per_sm);
  const int vec_ok = (reinterpret_cast<uintptr_t>(pa.pts) % 16) == 0;
  kern<<<unsigned(grid), kThreads, smem, s>>>(pa, sink, n_chunks, vec_ok);
  count_launch();
  return cudaGetLastError();
}

template <class Sink>
cudaError_t launch_any(const PackArgs& pa, const Sink& sink, cudaStream_t s) {
  switch (pa.d) {
    case 1: return launch_d<1>(pa, sink, s);
    case 2: return launch_d<2>(pa, sink, s);
    case 3: return launch_d<3>(pa, sink, s);
    case 4: return launch_d<4>(pa, sink, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_pack_store(const PackArgs& pa, int word_bits, void* keys, cudaStream_t s) {
  if (pa.n == 0) return cudaSuccess;
  if (pa.ell <= 64) return launch_fast_any(pa, MakeStore{keys, word_bits}, s);
  StoreSink sink{keys, word_bits, (pa.ell + word_bits - 1) / word_bits};
  return launch_any(pa, sink, s);
}

cudaError_t launch_pack_insert_seg(const SegPackScene* scenes, int n_scenes, uint64_t total_tiles,
                                   int d, int nch, cudaStream_t s) {
  if (n_scenes <= 0 || total_tiles == 0) return cudaSuccess;
  if (nch != 1 && nch != 2) return cudaErrorInvalidValue;
  switch (d) {
    case 1: return nch == 2 ? launch_seg_dn<1, 2>(scenes, n_scenes, total_tiles, s)
                            : launch_seg_dn<1, 1>(scenes, n_scenes, total_tiles, s);
    case 2: return nch == 2 ? launch_seg_dn<2, 2>(scenes, n_scenes, total_tiles, s)
                            : launch_seg_dn<2, 1>(scenes, n_scenes, total_tiles, s);
    case 3: return nch == 2 ? launch_seg_dn<3, 2>(scenes, n_scenes, total_tiles, s)
                            : launch_seg_dn<3, 1>(scenes, n_scenes, total_tiles, s);
    case 4: return nch == 2 ? launch_seg_dn<4, 2>(scenes, n_scenes, total_tiles, s)
                            : launch_seg_dn<4, 1>(scenes, n_scenes, total_tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_store_seg(const SegPackScene* scenes, int n_scenes, uint64_t total_tiles,
                                  int d, int w64, cudaStream_t s) {
  if (n_scenes <= 0 || total_tiles == 0) return cudaSuccess;
  auto by_w = [&](auto dtag) -> cudaError_t {
    constexpr int D = decltype(dtag)::value;
    switch (w64) {
      case 2: return launch_seg_dn<D, 2, 2>(scenes, n_scenes, total_tiles, s);
      case 3: return launch_seg_dn<D, 2, 3>(scenes, n_scenes, total_tiles, s);
      case 4: return launch_seg_dn<D, 2, 4>(scenes, n_scenes, total_tiles, s);
      default: return cudaErrorInvalidValue;
    }
  };
  switch (d) {
    case 1: return by_w(std::integral_constant<int, 1>{});
    case 2: return by_w(std::integral_constant<int, 2>{});
    case 3: return by_w(std::integral_constant<int, 3>{});
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_insert(const PackArgs& pa, const SmallTable& t, cudaStream_t s) {
  if (pa.ell > 64) return cudaErrorInvalidValue;
  if (pa.n == 0) return cudaSuccess;
  return launch_fast_any(pa, MakeInsert{t}, s);
}

cudaError_t launch_pack_grid_setup(const PackArgs& pa, const PackGrid& g, cudaStream_t s) {
  if (pa.ell > 64) return cudaErrorInvalidValue;
  if (pa.n == 0) return cudaSuccess;
  const bool two = pa.ell > 32;
  switch (pa.d) {
    case 1: return two ? launch_grid_setup_dn<1, 2>(pa, g, s) : launch_grid_setup_dn<1, 1>(pa, g, s);
    case 2: return two ? launch_grid_setup_dn<2, 2>(pa, g, s) : launch_grid_setup_dn<2, 1>(pa, g, s);
    case 3: return two ? launch_grid_setup_dn<3, 2>(pa, g, s) : launch_grid_setup_dn<3, 1>(pa, g, s);
    case 4: return two ? launch_grid_setup_dn<4, 2>(pa, g, s) : launch_grid_setup_dn<4, 1>(pa, g, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_insert_grid(const PackArgs& pa, const SmallTable& t, const PackGrid& g,
                                    cudaStream_t s) {
  if (pa.ell > 64) return cudaErrorInvalidValue;
  if (pa.n == 0) return cudaSuccess;
  const bool two = pa.ell > 32;
  switch (pa.d) {
    case 1: return two ? launch_grid_dn<1, 2>(pa, t, g, s) : launch_grid_dn<1, 1>(pa, t, g, s);
    case 2: return two ? launch_grid_dn<2, 2>(pa, t, g, s) : launch_grid_dn<2, 1>(pa, t, g, s);
    case 3: return two ? launch_grid_dn<3, 2>(pa, t, g, s) : launch_grid_dn<3, 1>(pa, t, g, s);
    case 4: return two ? launch_grid_dn<4, 2>(pa, t, g, s) : launch_grid_dn<4, 1>(pa, t, g, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cg
