// Step 1 for curved boundaries: sign vectors of quadric constraints (§2.1: the
// constraints c_i are inequalities whose boundaries partition the space into
// cells; §2 notes that the construction carries over to settings more
// complicated than lines).
//
// Bit i of point p is [ sum_{j<=k} q_i,jk p_j p_k + sum_k a_ik p_k >= b_i ],
// exact for every int32 point and coefficient and int64 offset. A quadric is a
// linear form over the point's feature vector
//   phi(p) = (p_j p_k for j <= k, p_0 .. p_{d-1}),  F = d(d+1)/2 + d features,
// so the kernel computes phi once per point and evaluates every constraint as
// an fp32 FMA chain over phi, exactly as the half-space kernel does over p:
//
//   With u = 2^-24, every feature is computed as fl(fl(p_j) fl(p_k)) or
//   fl(p_k) (relative error <= (1+u)^3 - 1), every coefficient and the offset
//   are rounded once (relative error <= u), and the chain
//   t = fma(c_{F-1}, x_{F-1}, ... fma(c_0, x_0, fl(-b))) adds F rounding steps
//   (error <= gamma_F sum |c^ x^|, standard FMA dot-product analysis, Higham
//   ch. 3). Together |t - s| <= (gamma_F (1+u)^4 + (1+u)^4 - 1) T
//   < (F + 8) u T, with T = sum |q_jk| M_j M_k + sum |a_k| M_k + |b| for the
//   tile's bounds M_k >= |p_k| (T rounded upwards).
//
// Each constraint row is scaled by the power of two 2^-e with E 2^-e < 1,
// E = (F + 8) u T; the scaling is exact, so |t'| >= 2 (bit 30 of the float)
// proves the sign. Chunks of 32 constraints whose test fails for some point are
// settled by the whole warp in exact 128-bit integer arithmetic (lanes over
// constraints). Padding constraints (i >= l) evaluate to -4 (bit 0).
#include <string>

#include "../../include/cellgraph.h"
#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
constexpr int kQGroupChunks = 16;  // rows of at most 16 chunks (512 constraints) in shared memory

template <int D>
struct Quad {
  static constexpr int M = D * (D + 1) / 2;  // monomials
  static constexpr int F = M + D;            // features
  static constexpr int kQuads = (F + 1 + 3) / 4;
  static constexpr int P = D <= 3 ? 4 : 2;   // points per thread
};

__device__ __forceinline__ uint32_t uabs32q(int32_t v) {
  return v < 0 ? 0u - uint32_t(v) : uint32_t(v);
}
__device__ __forceinline__ uint64_t uabs64q(int64_t v) {
  return v < 0 ? 0ull - uint64_t(v) : uint64_t(v);
}

struct QuadArgs {
  const int32_t* pts;
  int64_t n;
  const int32_t* q;  // [l][M]
  const int32_t* a;  // [l][D]
  const int64_t* b;  // [l]
  int ell;
  int word_bits;
  int w;  // words per vector in word_bits units
  void* keys;
};

// Exact [q_t . mono(p) + a_t . p >= b_t] in 128-bit integers.
template <int D>
__device__ __forceinline__ bool quad_exact_ge(const QuadArgs& qa, int t, const int32_t (&p)[D]) {
  constexpr int M = Quad<D>::M;
  const int32_t* qr = qa.q + int64_t(t) * M;
  const int32_t* ar = qa.a + int64_t(t) * D;
  __int128 s = -static_cast<__int128>(qa.b[t]);
  int m = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
#pragma unroll
    for (int k = j; k < D; ++k, ++m)
      s += static_cast<__int128>(qr[m]) * static_cast<__int128>(int64_t(p[j]) * int64_t(p[k]));
  }
#pragma unroll
  for (int k = 0; k < D; ++k) s += static_cast<__int128>(int64_t(ar[k]) * int64_t(p[k]));
  return s >= 0;
}

// Scaled row of constraint t for a tile with |p_k| <= Mk[k]:
// [q (M floats), a (D floats), c] padded to whole float4s.
template <int D>
__device__ void quad_build_row(const QuadArgs& qa, int t, const float (&Mk)[D], float4* dst) {
  constexpr int M = Quad<D>::M;
  constexpr int F = Quad<D>::F;
  float v[Quad<D>::kQuads * 4];
#pragma unroll
  for (int i = 0; i < Quad<D>::kQuads * 4; ++i) v[i] = 0.0f;
  float c;
  if (t >= qa.ell) {
    c = -4.0f;  // padding: certain, negative, bit 0
  } else {
    const int32_t* qr = qa.q + int64_t(t) * M;
    const int32_t* ar = qa.a + int64_t(t) * D;
    const int64_t bt = qa.b[t];
    float T = __ull2float_ru(uabs64q(bt));
    int m = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int k = j; k < D; ++k, ++m)
        T = __fmaf_ru(__uint2float_ru(uabs32q(qr[m])), __fmul_ru(Mk[j], Mk[k]), T);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) T = __fmaf_ru(__uint2float_ru(uabs32q(ar[k])), Mk[k], T);
    if (T == 0.0f) {
      c = 4.0f;  // every coefficient and the offset are 0: s == 0, bit 1
    } else {
      const float E = __fmul_ru(T, float(F + 8) * 0x1p-24f);
      int e;
      frexpf(E, &e);  // E = m 2^e with 0.5 <= m < 1: E 2^-e < 1
#pragma unroll
      for (int i = 0; i < M; ++i) v[i] = ldexpf(__int2float_rn(qr[i]), -e);
#pragma unroll
      for (int k = 0; k < D; ++k) v[M + k] = ldexpf(__int2float_rn(ar[k]), -e);
      c = ldexpf(-__ll2float_rn(bt), -e);
    }
  }
  v[F] = c;
#pragma unroll
  for (int i = 0; i < Quad<D>::kQuads; ++i)
    dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// Uncertain chunks: for every lane whose chunk test failed, the warp evaluates
// the lane's P points against the chunk's 32 constraints exactly (lane j takes
// constraint 32 chunk + j) and overwrites the lane's sign bits. Whole warp.
template <int D, int P>
__device__ __forceinline__ void quad_settle(const QuadArgs& qa, int chunk, int64_t p_lane0,
                                            bool uncertain, uint32_t (&w)[P]) {
  const int lane = threadIdx.x & 31;
  uint32_t todo = __ballot_sync(0xffffffffu, uncertain);
  const int t = chunk * 32 + lane;
  while (todo) {
    const int L = __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t pL = p_lane0 + int64_t(L) * P;
#pragma unroll 1
    for (int q = 0; q < P; ++q) {
      if (pL + q >= qa.n) break;
      int32_t pq[D];
#pragma unroll
      for (int k = 0; k < D; ++k) pq[k] = __ldg(qa.pts + (pL + q) * D + k);
      const bool ge = t < qa.ell && quad_exact_ge<D>(qa, t, pq);
      const uint32_t neg = ~__ballot_sync(0xffffffffu, ge);  // sign bit 1: not satisfied
      if (lane == L) {
#pragma unroll
        for (int qq = 0; qq < P; ++qq)
          if (qq == q) w[qq] = neg;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kQThreads)
    quadric_kernel(QuadArgs qa, int n_chunks, int vec_ok) {
  constexpr int M = Quad<D>::M;
  constexpr int F = Quad<D>::F;
  constexpr int kQ = Quad<D>::kQuads;
  constexpr int P = Quad<D>::P;
  constexpr int kTile = kQThreads * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* rows = reinterpret_cast<float4*>(smem_raw);
  __shared__ uint32_t wmax[kQWarps][D];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n = qa.n;
  const int64_t n_tiles = (n + kTile - 1) / kTile;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTile + int64_t(threadIdx.x) * P;
    int32_t pi[P][D];
    if (vec_ok && (P * D) % 4 == 0 && p0 + P <= n) {
      const int4* src = reinterpret_cast<const int4*>(qa.pts + p0 * D);
      int32_t tmp[P * D];
#pragma unroll
      for (int i = 0; i < P * D / 4; ++i) {
        const int4 v = __ldg(src + i);
        tmp[4 * i] = v.x;
        tmp[4 * i + 1] = v.y;
        tmp[4 * i + 2] = v.z;
        tmp[4 * i + 3] = v.w;
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
          pi[q][k] = (p0 + q < n) ? __ldg(qa.pts + (p0 + q) * D + k) : 0;
    }
    // Largest |p_k| of the tile.
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) m = max(m, uabs32q(pi[q][k]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) wmax[warp][k] = m;
    }
    // Features: monomials, then the coordinates.
    float x[P][F];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      float pf[D];
#pragma unroll
      for (int k = 0; k < D; ++k) pf[k] = __int2float_rn(pi[q][k]);
      int m = 0;
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int k = j; k < D; ++k, ++m) x[q][m] = __fmul_rn(pf[j], pf[k]);
#pragma unroll
      for (int k = 0; k < D; ++k) x[q][M + k] = pf[k];
    }
    __syncthreads();  // wmax complete; every thread is done with the previous rows
    float Mk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      uint32_t m = 0;
      for (int w2 = 0; w2 < kQWarps; ++w2) m = max(m, wmax[w2][k]);
      Mk[k] = __uint2float_ru(m);
    }
    uint32_t stash[P];
#pragma unroll
    for (int q = 0; q < P; ++q) stash[q] = 0;
    for (int g0 = 0; g0 < n_chunks; g0 += kQGroupChunks) {
      const int g1 = min(n_chunks, g0 + kQGroupChunks);
      if (g0 > 0) __syncthreads();  // the previous group's rows are no longer read
      for (int t = g0 * 32 + threadIdx.x; t < g1 * 32; t += kQThreads)
        quad_build_row<D>(qa, t, Mk, rows + size_t(t - g0 * 32) * kQ);
      __syncthreads();
      for (int c = g0; c < g1; ++c) {
        uint32_t w[P];
#pragma unroll
        for (int q = 0; q < P; ++q) w[q] = 0;
        uint32_t cert = 0xffffffffu;
        const float4* cc = rows + size_t(c - g0) * 32 * kQ;
#pragma unroll 4
        for (int j = 31; j >= 0; --j) {
          float4 r4[kQ];
#pragma unroll
          for (int i = 0; i < kQ; ++i) r4[i] = cc[j * kQ + i];
          const float* f = reinterpret_cast<const float*>(r4);
#pragma unroll
          for (int q = 0; q < P; ++q) {
            float acc = f[F];
#pragma unroll
            for (int i = 0; i < F; ++i) acc = fmaf(f[i], x[q][i], acc);
            const uint32_t bits = __float_as_uint(acc);
            w[q] = __funnelshift_l(bits, w[q], 1);
            cert &= bits;
          }
        }
        quad_settle<D, P>(qa, c, p0 - int64_t(lane) * P, !(cert & 0x40000000u), w);
        const bool last = c == n_chunks - 1;
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int64_t p = p0 + q;
          if (p >= n) continue;
          const uint32_t bits = ~w[q];
          if (qa.word_bits == 32) {
            static_cast<uint32_t*>(qa.keys)[p * qa.w + c] = bits;
          } else if ((c & 1) == 0 && !last) {
            stash[q] = bits;
          } else {
            const uint64_t v = (c & 1) ? (uint64_t(stash[q]) | (uint64_t(bits) << 32)) : bits;
            static_cast<uint64_t*>(qa.keys)[p * qa.w + (c >> 1)] = v;
          }
        }
      }
    }
  }
}

template <int D>
cudaError_t launch_quadric_d(const QuadArgs& qa, cudaStream_t s) {
  constexpr int P = Quad<D>::P;
  const int n_chunks = (qa.ell + 31) / 32;
  const int group = n_chunks < kQGroupChunks ? n_chunks : kQGroupChunks;
  const size_t smem = size_t(group) * 32 * Quad<D>::kQuads * sizeof(float4);
  auto kern = quadric_kernel<D>;
  cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = blocks_per_sm(reinterpret_cast<const void*>(kern), kQThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int64_t n_tiles = (qa.n + kQThreads * P - 1) / (kQThreads * P);
  const int64_t grid = std::min<int64_t>(n_tiles, int64_t(sm_count()) * per_sm);
  const int vec_ok = (reinterpret_cast<uintptr_t>(qa.pts) % 16) == 0;
  kern<<<unsigned(grid), kQThreads, smem, s>>>(qa, n_chunks, vec_ok);
  count_launch();
  return cudaGetLastError();
}

cg_status quad_fail(cg_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace
}  // namespace cg

extern "C" {

cg_status cg_pack_signs_quadric(const int32_t* pts, int64_t n, int d, const int32_t* q,
                                const int32_t* a, const int64_t* b, int ell, int word_bits,
                                void* keys, void* stream) {
  using namespace cg;
  if (n < 0) return quad_fail(CG_ERR_INVALID_ARG, "cg_pack_signs_quadric: n < 0");
  if (ell < 1 || ell > 4096)
    return quad_fail(CG_ERR_INVALID_ARG, "cg_pack_signs_quadric: l must satisfy 1 <= l <= 4096");
  if (word_bits != 32 && word_bits != 64)
    return quad_fail(CG_ERR_INVALID_ARG, "cg_pack_signs_quadric: word_bits must be 32 or 64");
  if (d < 1 || d > 4)
    return quad_fail(CG_ERR_INVALID_ARG, "cg_pack_signs_quadric: d must satisfy 1 <= d <= 4");
  if (n > 0 && (!pts || !q || !a || !b || !keys))
    return quad_fail(CG_ERR_INVALID_ARG, "cg_pack_signs_quadric: NULL array");
  if (n == 0) return CG_OK;
  QuadArgs qa{pts, n, q, a, b, ell, word_bits, (ell + word_bits - 1) / word_bits, keys};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (d) {
    case 1: e = launch_quadric_d<1>(qa, s); break;
    case 2: e = launch_quadric_d<2>(qa, s); break;
    case 3: e = launch_quadric_d<3>(qa, s); break;
    default: e = launch_quadric_d<4>(qa, s); break;
  }
  if (e != cudaSuccess) {
    set_last_error((std::string("cg_pack_signs_quadric: ") + cudaGetErrorString(e)).c_str());
    return CG_ERR_CUDA;
  }
  return CG_OK;
}

}  // extern "C"
