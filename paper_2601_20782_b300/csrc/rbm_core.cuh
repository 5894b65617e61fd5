// Device-side building blocks of the RBM sampler and local energy, shared by the
// per-dtype translation units (rbm.cu: FP32 sampling copy; rbm_f16.cu, rbm_bf16.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace nqs {
namespace rbmk {


constexpr uint32_t BULK_CHUNK = 32768;

// Threads per CTA bound for E cached units per lane (register budget per thread).
constexpr int threads_for_regs(int regs) {
  int w = 65536 / (32 * regs);
  w = w < 2 ? 2 : (w > 32 ? 32 : w);
  return 32 * w;
}
// sweep: the cache pairs stay live, the row and the factors are streamed
constexpr int sweep_threads(int E) { return threads_for_regs(2 * E + 46); }
// local energy: the cache plus two sites' rows and factors in flight
constexpr int eloc_threads(int E) { return threads_for_regs(2 * E + 46); }
constexpr uint32_t WAIT_POLLS = 1u << 22;


// ------------------------------------------------------------------------------------
// Paired FP32 arithmetic (fma.rn.f32x2 / mul.rn.f32x2, sm_100 family): two FP32
// operations per issued instruction, each rounded as its scalar counterpart.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// ------------------------------------------------------------------------------------
// Per-chain cache layout.  L lanes per chain, E hidden units per lane held as H = ceil(E/2)
// float2 pairs.  Lane gl owns units j = 4 (v L + gl) + c for v < E / 4, c < 4 (one 16-byte
// vector), and j = 4 (E / 4) L + t L + gl for the E % 4 tail units.  For odd E the last
// pair's second slot is a dummy unit with lam = mu = 1/2 and R = 1, which contributes
// exactly nothing (g = 1) and stays unchanged by updates.
template <int L, int E>
struct Lay {
  static constexpr int V = E / 4, T = E % 4, H = (E + 1) / 2;
  // row[j] for the lane's units into pairs; `pad` fills the dummy slot
  template <bool LDG>
  __device__ static __forceinline__ void load(const float *row, int gl, float2 (&r)[H], float pad) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float4 *p4 = reinterpret_cast<const float4 *>(row + 4 * (v * L + gl));
      const float4 q = LDG ? __ldg(p4) : *p4;
      r[2 * v] = make_float2(q.x, q.y);
      r[2 * v + 1] = make_float2(q.z, q.w);
    }
    const float *tail = row + 4 * V * L + gl;
    auto ld = [&](int t) { return LDG ? __ldg(tail + t * L) : tail[t * L]; };
    if constexpr (T == 1) r[2 * V] = make_float2(ld(0), pad);
    if constexpr (T == 2) r[2 * V] = make_float2(ld(0), ld(1));
    if constexpr (T == 3) {
      r[2 * V] = make_float2(ld(0), ld(1));
      r[2 * V + 1] = make_float2(ld(2), pad);
    }
  }
};

// Sampling-copy arithmetic of the 16-bit tables: pairs of BF16 / F16 values and their
// packed FMA (Table tab:precision; the sampling copy of Sec. 4.2).
template <typename TT>
struct Prec;
template <>
struct Prec<float> {  // the FP32 sampling copy has no 16-bit shadows
  using T2 = float2;
};
template <>
struct Prec<__half> {
  using T2 = __half2;
  __device__ static __forceinline__ T2 from_f2(float2 v) { return __float22half2_rn(v); }
  __device__ static __forceinline__ float2 to_f2(T2 v) { return __half22float2(v); }
  __device__ static __forceinline__ T2 fma(T2 a, T2 b, T2 c) { return __hfma2(a, b, c); }
  __device__ static __forceinline__ T2 mul(T2 a, T2 b) { return __hmul2(a, b); }
  __device__ static __forceinline__ T2 make(__half x, __half y) { return __halves2half2(x, y); }
  __device__ static __forceinline__ __half one() { return __float2half(1.f); }
};
template <>
struct Prec<__nv_bfloat16> {
  using T2 = __nv_bfloat162;
  __device__ static __forceinline__ T2 from_f2(float2 v) { return __float22bfloat162_rn(v); }
  __device__ static __forceinline__ float2 to_f2(T2 v) { return __bfloat1622float2(v); }
  __device__ static __forceinline__ T2 fma(T2 a, T2 b, T2 c) { return __hfma2(a, b, c); }
  __device__ static __forceinline__ T2 mul(T2 a, T2 b) { return __hmul2(a, b); }
  __device__ static __forceinline__ T2 make(__nv_bfloat16 x, __nv_bfloat16 y) { return __halves2bfloat162(x, y); }
  __device__ static __forceinline__ __nv_bfloat16 one() { return __float2bfloat16(1.f); }
};

// row[j] of a 16-bit table for the lane's units, as pairs (same unit layout as Lay)
template <int L, int E, typename TT>
__device__ __forceinline__ void load_pairs_tt(const TT *row, int gl, typename Prec<TT>::T2 (&r)[Lay<L, E>::H]) {
  using LY = Lay<L, E>;
  using P = Prec<TT>;
#pragma unroll
  for (int v = 0; v < LY::V; ++v) {
    const uint2 q = *reinterpret_cast<const uint2 *>(row + 4 * (v * L + gl));
    r[2 * v] = *reinterpret_cast<const typename P::T2 *>(&q.x);
    r[2 * v + 1] = *reinterpret_cast<const typename P::T2 *>(&q.y);
  }
  const TT *tail = row + 4 * LY::V * L + gl;
  if constexpr (LY::T == 1) r[2 * LY::V] = P::make(tail[0], P::one());
  if constexpr (LY::T == 2) r[2 * LY::V] = P::make(tail[0], tail[L]);
  if constexpr (LY::T == 3) {
    r[2 * LY::V] = P::make(tail[0], tail[L]);
    r[2 * LY::V + 1] = P::make(tail[2 * L], P::one());
  }
}

// 16-bit shadows of the FP32 cache, used by the low-precision factor arithmetic
template <int H, typename TT>
__device__ __forceinline__ void make_shadows(const float2 (&lam)[H], const float2 (&mu)[H],
                                             typename Prec<TT>::T2 (&lh)[H], typename Prec<TT>::T2 (&mh)[H]) {
#pragma unroll
  for (int k = 0; k < H; ++k) {
    lh[k] = Prec<TT>::from_f2(lam[k]);
    mh[k] = Prec<TT>::from_f2(mu[k]);
  }
}

__device__ __forceinline__ void sigmoid_pair(float th, float &lam, float &mu) {
  const float e = expf(-2.f * fabsf(th));
  const float p = 1.f / (1.f + e);
  const float q = e * p;
  lam = th >= 0.f ? p : q;
  mu = th >= 0.f ? q : p;
}

// The same pair from the MUFU forms: e^{-2|th|} as 2^{-2|th| log2 e} and the reciprocal by
// rcp.approx.  The rounding of the exponent's argument puts a relative error of at most
// 2|th| 2^-24 (plus a few ulp) on the smaller entry, e^{-2|th|} / (1 + e^{-2|th|}); the
// larger is within a few ulp.  Used where the pairs are rebuilt for every sample (chain-ordered local energy).
__device__ __forceinline__ void sigmoid_pair_fast(float th, float &lam, float &mu) {
  const float e = ex2_approx(-2.8853900817779268f * fabsf(th));
  const float p = rcp_approx(1.f + e);
  const float q = e * p;
  lam = th >= 0.f ? p : q;
  mu = th >= 0.f ? q : p;
}

template <int L, int E>
__device__ __forceinline__ void compute_theta(float2 (&th)[Lay<L, E>::H], uint32_t sw, const float *__restrict__ Wt,
                                              const float *__restrict__ b, int N, int W, int M_pad, int gl) {
  using LY = Lay<L, E>;
  LY::template load<true>(b, gl, th, 0.f);
  for (int wi = 0; wi < W; ++wi) {
    const uint32_t word = __shfl_sync(FULL_MASK, sw, wi, L);
    const int nb = min(32, N - 32 * wi);
    for (int bit = 0; bit < nb; ++bit) {
      const float s = ((word >> bit) & 1u) ? 1.f : -1.f;
      float2 w[LY::H];
      LY::template load<true>(Wt + (size_t)(32 * wi + bit) * M_pad, gl, w, 0.f);
      const float2 s2 = make_float2(s, s);
#pragma unroll
      for (int k = 0; k < LY::H; ++k) th[k] = fma2(s2, w[k], th[k]);
    }
  }
}

template <int L, int E>
__device__ __forceinline__ void build_cache(float2 (&lam)[Lay<L, E>::H], float2 (&mu)[Lay<L, E>::H], uint32_t sw,
                                            const float *Wt, const float *b, int N, int W, int M_pad, int gl) {
  float2 th[Lay<L, E>::H];
  compute_theta<L, E>(th, sw, Wt, b, N, W, M_pad, gl);
#pragma unroll
  for (int k = 0; k < Lay<L, E>::H; ++k) {
    sigmoid_pair(th[k].x, lam[k].x, mu[k].x);
    sigmoid_pair(th[k].y, lam[k].y, mu[k].y);
  }
}

// sum_i a_i s_i over the group (every lane gets the same value)
template <int L>
__device__ __forceinline__ float visible_term(uint32_t sw, const float2 *aK, int N, int gl) {
  float v = 0.f;
  for (int i0 = 0; i0 < N; i0 += L) {
    const int i = i0 + gl;
    const uint32_t word = __shfl_sync(FULL_MASK, sw, (min(i, N - 1)) >> 5, L);
    if (i < N) v += ((word >> (i & 31)) & 1u) ? aK[i].x : -aK[i].x;
  }
  return group_allsum<L>(v);
}

// log psi from the cache: sum_i a_i s_i - 1/2 sum_j log(4 lam_j mu_j)
template <int L, int E>
__device__ __forceinline__ float cache_logpsi(const float2 (&lam)[Lay<L, E>::H], const float2 (&mu)[Lay<L, E>::H],
                                              uint32_t sw, const float2 *aK, int N, int gl) {
  float part = 0.f;
#pragma unroll
  for (int k = 0; k < Lay<L, E>::H; ++k)
    part += (2.f + log2f(lam[k].x) + log2f(mu[k].x)) + (2.f + log2f(lam[k].y) + log2f(mu[k].y));
  return visible_term<L>(sw, aK, N, gl) - 0.5f * LN2F * group_allsum<L>(part);
}

// Factor pairs multiplied together before one MUFU lg2: 16 factors of size e^{+-4|W|} (times
// the cache's scale drift) stay well inside the FP32 range for the weights the sampler is
// used with; a product that leaves it sends the group to the exact path (flip_logsum).
constexpr int PAIRS_PER_LG2 = 8;

// sum over groups of PAIRS_PER_LG2 pairs of log2 of the product of the factors g_k = a_k r_k + b_k
template <int H>
__device__ __forceinline__ float product_log2(const float2 (&a)[H], const float2 (&b)[H], const float2 (&r)[H]) {
  float part = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < H; k0 += PAIRS_PER_LG2) {
    float2 pr = fma2(a[k0], r[k0], b[k0]);
#pragma unroll
    for (int k = k0 + 1; k < (k0 + PAIRS_PER_LG2 < H ? k0 + PAIRS_PER_LG2 : H); ++k)
      pr = mul2(pr, fma2(a[k], r[k], b[k]));
    part += lg2_approx(pr.x * pr.y);
  }
  return part;
}

// Streams the lane's row in 4-pair groups: loads a group, forms its factors g and
// their product, and returns the lane's partial sum of log2 products; *g_out keeps the
// factors only when requested (exact fallback path).
template <int L, int E>
__device__ __forceinline__ float flip_partial(bool up, const float2 (&lam)[Lay<L, E>::H],
                                             const float2 (&mu)[Lay<L, E>::H], const float *row, int gl) {
  using LY = Lay<L, E>;
  float2 rv[LY::H];
  LY::template load<false>(row, gl, rv, 1.f);
  // g = mu + lam R (up) or lam + mu R (down): one uniform branch, no per-unit selects
  return up ? product_log2<LY::H>(lam, mu, rv) : product_log2<LY::H>(mu, lam, rv);
}

// Exact sum of log2 g over the lane's units (fallback when a product left the FP32 range).
template <int L, int E>
__device__ __forceinline__ float flip_partial_exact(bool up, const float2 (&lam)[Lay<L, E>::H],
                                                 const float2 (&mu)[Lay<L, E>::H], const float *row, int gl) {
  using LY = Lay<L, E>;
  float2 rv[LY::H];
  LY::template load<false>(row, gl, rv, 1.f);
  float p = 0.f;
#pragma unroll
  for (int k = 0; k < LY::H; ++k) {
    const float2 g = up ? fma2(lam[k], rv[k], mu[k]) : fma2(mu[k], rv[k], lam[k]);
    p += log2f(g.x) + log2f(g.y);
  }
  return p;
}

// Group sum of the lane partials.  With one chain per warp the partials are added exactly
// as 2^-20 fixed-point integers by one redux.sync (a 32-lane sum in one instruction, and the
// same bits in every lane, so the accept decision is warp-uniform); each partial is rounded
// to 2^-21, so the sum carries at most 32 * 2^-21 absolute error in log2 units.  A product
// that left the normal FP32 range, or a partial beyond +-2^10, sends the group to the exact
// path: one accurate log per factor and a floating-point butterfly.
template <int L, int E>
__device__ __forceinline__ float flip_logsum(bool up, const float2 (&lam)[Lay<L, E>::H],
                                            const float2 (&mu)[Lay<L, E>::H], const float *row, int gl) {
  const float part = flip_partial<L, E>(up, lam, mu, row, gl);
  if constexpr (L == 32) {
    const bool bad = !(fabsf(part) < 1024.f);
    if (!__any_sync(FULL_MASK, bad)) {
      const int q = __float2int_rn(part * 1048576.f);
      return (float)__reduce_add_sync(FULL_MASK, q) * 9.5367431640625e-7f;
    }
  } else {
    const float tot = group_allsum<L>(part);
    if (!__any_sync(FULL_MASK, !isfinite(tot))) return tot;
  }
  return group_allsum<L>(flip_partial_exact<L, E>(up, lam, mu, row, gl));
}

// Low-precision counterpart of flip_partial: the factors g are formed in 16-bit pair
// arithmetic from the 16-bit shadows and table (the network's elementwise math in the
// sampling dtype); their product over hidden units is the reduction of the log-amplitude
// and is taken in FP32 (App. I: reductions in higher precision), PAIRS_PER_LG2 pairs of units per MUFU lg2.
template <int L, int E, typename TT>
__device__ __forceinline__ float flip_partial_lp(bool up, const typename Prec<TT>::T2 (&lh)[Lay<L, E>::H],
                                                const typename Prec<TT>::T2 (&mh)[Lay<L, E>::H], const TT *row,
                                                int gl) {
  using LY = Lay<L, E>;
  using P = Prec<TT>;
  typename P::T2 rv[LY::H];
  load_pairs_tt<L, E, TT>(row, gl, rv);
  auto prod = [&](const typename P::T2(&a)[LY::H], const typename P::T2(&b)[LY::H]) {
    float part = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < LY::H; k0 += PAIRS_PER_LG2) {
      float2 pr = P::to_f2(P::fma(a[k0], rv[k0], b[k0]));
#pragma unroll
      for (int k = k0 + 1; k < (k0 + PAIRS_PER_LG2 < LY::H ? k0 + PAIRS_PER_LG2 : LY::H); ++k)
        pr = mul2(pr, P::to_f2(P::fma(a[k], rv[k], b[k])));
      part += lg2_approx(pr.x * pr.y);
    }
    return part;
  };
  return up ? prod(lh, mh) : prod(mh, lh);  // one uniform branch, no per-unit selects
}

// exact path of the low-precision sum: each 16-bit factor converted and logged separately
template <int L, int E, typename TT>
__device__ __forceinline__ float flip_partial_lp_exact(bool up, const typename Prec<TT>::T2 (&lh)[Lay<L, E>::H],
                                                      const typename Prec<TT>::T2 (&mh)[Lay<L, E>::H], const TT *row,
                                                      int gl) {
  using LY = Lay<L, E>;
  using P = Prec<TT>;
  typename P::T2 rv[LY::H];
  load_pairs_tt<L, E, TT>(row, gl, rv);
  float p = 0.f;
#pragma unroll
  for (int k = 0; k < LY::H; ++k) {
    const float2 g = P::to_f2(up ? P::fma(lh[k], rv[k], mh[k]) : P::fma(mh[k], rv[k], lh[k]));
    p += log2f(g.x) + log2f(g.y);
  }
  return p;
}

template <int L, int E, typename TT>
__device__ __forceinline__ float flip_logsum_lp(bool up, const typename Prec<TT>::T2 (&lh)[Lay<L, E>::H],
                                               const typename Prec<TT>::T2 (&mh)[Lay<L, E>::H], const TT *row, int gl) {
  const float part = flip_partial_lp<L, E, TT>(up, lh, mh, row, gl);
  if constexpr (L == 32) {
    const bool bad = !(fabsf(part) < 1024.f);
    if (!__any_sync(FULL_MASK, bad)) {
      const int q = __float2int_rn(part * 1048576.f);
      return (float)__reduce_add_sync(FULL_MASK, q) * 9.5367431640625e-7f;
    }
  } else {
    const float tot = group_allsum<L>(part);
    if (!__any_sync(FULL_MASK, !isfinite(tot))) return tot;
  }
  return group_allsum<L>(flip_partial_lp_exact<L, E, TT>(up, lh, mh, row, gl));
}

// Loads the [N][M_pad] table into shared memory with 1D bulk copies.  Returns false
// (after recording STATUS_TIMEOUT) if the copies did not land within the poll limit.
template <typename TT>
__device__ bool load_table(TT *sR, const TT *R, uint32_t bytes, uint64_t *bar, int *status) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, bytes);
    for (uint32_t off = 0; off < bytes; off += BULK_CHUNK)
      bulk_g2s(reinterpret_cast<char *>(sR) + off, reinterpret_cast<const char *>(R) + off,
               min(BULK_CHUNK, bytes - off), bar);
  }
  bool ok = mbar_wait_bounded(bar, 0, WAIT_POLLS);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
    mbar_wait_bounded(bar, 0, WAIT_POLLS);  // let copies in flight land before the CTA exits
  }
  return __syncthreads_and(ok);
}

// Accepted flip: lam/mu = e^{2 theta} is multiplied by R (spin up) or 1/R (spin down):
//   up:   lam' = lam R / g, mu' = mu / g,  g = mu + lam R
//   down: mu' = mu R / g,  lam' = lam / g, g = lam + mu R
// The row is re-read pair by pair and g recomputed, so neither has to stay live in
// registers from the proposal to the decision.
struct SweepParams {
  const void *R;  // [N][M_pad] table in the sampling dtype
  const float2 *aK;
  const float *Wt;
  const float *b;
  uint32_t *state;
  uint32_t *samples;
  float *logpsi;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
  int *status;
  int64_t C;
  int N, W, M_pad, n_sweeps, burn_in, refresh;
  int renorm;  // accepted flips between normalisations of the cache (ChainCache)
  uint32_t sweep_offset, k0, k1;
  float noise_sigma;  // noisy-RBM kernels only: standard deviation of zeta
  uint32_t noise_k0, noise_k1;
};

// Noisy RBM (Sec. 4.1): log psi~(x) = log psi(x) + zeta(x)/2, zeta(x) ~ N(0, sigma) fixed per
// configuration.  zeta is computed from the configuration: Philox4x32-10 chained over its
// words (h = (TAG_NOISE, W, 0, 0); per block of four words h = Philox(h ^ words; key)), then
// Box-Muller on u1 = ((h.x >> 8) + 1) 2^-24, u2 = (h.y >> 8) 2^-24.  Word j is held by lane j
// of the group (lanes >= W hold 0).  Returns zeta(x) / 2.
constexpr uint32_t TAG_NOISE = 0x4E4F4953u;  // "NOIS"
template <int L>
__device__ __forceinline__ float noise_half(uint32_t sw, int W, float sigma, uint32_t k0, uint32_t k1) {
  uint4 h = make_uint4(TAG_NOISE, (uint32_t)W, 0u, 0u);
  for (int b = 0; b < W; b += 4) {
    const uint32_t w0 = __shfl_sync(FULL_MASK, sw, b, L), w1 = __shfl_sync(FULL_MASK, sw, b + 1, L);
    const uint32_t w2 = __shfl_sync(FULL_MASK, sw, b + 2, L), w3 = __shfl_sync(FULL_MASK, sw, b + 3, L);
    h = philox4x32_10(make_uint4(h.x ^ w0, h.y ^ w1, h.z ^ w2, h.w ^ w3), k0, k1);
  }
  const float u1 = (float)((h.x >> 8) + 1u) * 5.9604644775390625e-8f;
  const float u2 = (float)(h.y >> 8) * 5.9604644775390625e-8f;
  return 0.5f * sigma * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// log u for u = k 2^-24 (k = 0 gives -inf: always accept).  Accepting iff
// 2 dlogpsi > log u is the rule u < exp(2 dlogpsi).
__device__ __forceinline__ float log_uniform(uint32_t w) {
  const uint32_t k = w >> 8;
  return k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
}

// Per-chain state of the sampler: the FP32 cache (lam, mu) and, for a 16-bit sampling
// copy, its 16-bit shadows used by the factor arithmetic.
//
// Between normalisations the pairs are kept unnormalised: (lam~_j, mu~_j) = s_j (lam_j, mu_j)
// with lam~/mu~ = e^{2 theta_j} exact and the chain's running log-scale ls = sum_j log2 s_j.
// A proposal's factors become g~_j = s_j g_j, so sum_j log2 g_j = sum_j log2 g~_j - ls.  An
// accepted flip multiplies lam~ (spin up) or mu~ (spin down) by R and nothing else: then
// s_j' = s_j g_j, so for the FP32 copy the new ls is the sum of log2 g~ the accepted proposal
// just computed; a 16-bit copy recomputes it from the FP32 pairs (see accept).
// Every `renorm` accepted flips (a bound on the drift chosen from the weights at
// nqs_set_params) the pairs are normalised again and ls returns to 0.
template <int L, int E, typename TT>
struct ChainCache {
  using LY = Lay<L, E>;
  static constexpr bool LP = !std::is_same<TT, float>::value;
  using T2 = typename Prec<TT>::T2;
  float2 lam[LY::H], mu[LY::H];
  T2 lh[LP ? LY::H : 1], mh[LP ? LY::H : 1];
  float ls = 0.f;  // sum_j log2 (lam~_j + mu~_j)
  int since = 0;   // accepted flips since the last normalisation

  __device__ __forceinline__ void build(uint32_t sw, const float *Wt, const float *b, int N, int W, int M_pad,
                                        int gl) {
    build_cache<L, E>(lam, mu, sw, Wt, b, N, W, M_pad, gl);
    if constexpr (LP) make_shadows<LY::H, TT>(lam, mu, lh, mh);
    ls = 0.f;
    since = 0;
  }
  // the cache of pre-activations th (sigmoid pairs), e.g. after an incremental update of th
  __device__ __forceinline__ void from_theta(const float2 (&th)[LY::H]) {
#pragma unroll
    for (int k = 0; k < LY::H; ++k) {
      sigmoid_pair_fast(th[k].x, lam[k].x, mu[k].x);
      sigmoid_pair_fast(th[k].y, lam[k].y, mu[k].y);
    }
    if constexpr (LP) make_shadows<LY::H, TT>(lam, mu, lh, mh);
    ls = 0.f;
    since = 0;
  }
  // this lane's share of sum_j log2 g~_j (grouped products; may be non-finite for a product
  // that leaves the FP32 range) and its exact counterpart
  __device__ __forceinline__ float partial(bool up, const TT *row, int gl) const {
    if constexpr (LP) return flip_partial_lp<L, E, TT>(up, lh, mh, row, gl);
    else return flip_partial<L, E>(up, lam, mu, row, gl);
  }
  __device__ __forceinline__ float partial_exact(bool up, const TT *row, int gl) const {
    if constexpr (LP) return flip_partial_lp_exact<L, E, TT>(up, lh, mh, row, gl);
    else return flip_partial_exact<L, E>(up, lam, mu, row, gl);
  }
  // sum_j log2 g~_j of flipping the site whose table row is `row` (subtract ls for sum log2 g)
  __device__ __forceinline__ float logsum(bool up, const TT *row, int gl) const {
    if constexpr (LP) return flip_logsum_lp<L, E, TT>(up, lh, mh, row, gl);
    else return flip_logsum<L, E>(up, lam, mu, row, gl);
  }
  // ls recomputed from the FP32 pairs: sum_j log2 (lam~_j + mu~_j) over the group, with the
  // grouped products and fixed-point reduction of the proposals (exact logs as fallback)
  __device__ __forceinline__ float scale_log2() const {
    const float2 one = make_float2(1.f, 1.f);
    float part = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < LY::H; k0 += PAIRS_PER_LG2) {
      float2 pr = fma2(lam[k0], one, mu[k0]);
#pragma unroll
      for (int k = k0 + 1; k < (k0 + PAIRS_PER_LG2 < LY::H ? k0 + PAIRS_PER_LG2 : LY::H); ++k)
        pr = mul2(pr, fma2(lam[k], one, mu[k]));
      part += lg2_approx(pr.x * pr.y);
    }
    if constexpr (L == 32) {
      if (!__any_sync(FULL_MASK, !(fabsf(part) < 1024.f)))
        return (float)__reduce_add_sync(FULL_MASK, __float2int_rn(part * 1048576.f)) * 9.5367431640625e-7f;
    } else {
      const float tot = group_allsum<L>(part);
      if (!__any_sync(FULL_MASK, !isfinite(tot))) return tot;
    }
    float p2 = 0.f;
#pragma unroll
    for (int k = 0; k < LY::H; ++k) p2 += log2f(lam[k].x + mu[k].x) + log2f(lam[k].y + mu[k].y);
    return group_allsum<L>(p2);
  }
  __device__ __forceinline__ void normalize() {
#pragma unroll
    for (int k = 0; k < LY::H; ++k) {
      const float2 s = make_float2(lam[k].x + mu[k].x, lam[k].y + mu[k].y);
      const float2 inv = make_float2(rcp_approx(s.x), rcp_approx(s.y));
      lam[k] = mul2(lam[k], inv);
      mu[k] = mul2(mu[k], inv);
    }
    if constexpr (LP) make_shadows<LY::H, TT>(lam, mu, lh, mh);
    ls = 0.f;
    since = 0;
  }
  // accepted flip of the site whose table row is `row`; tot = its logsum(up, row, gl)
  template <bool SMEM>
  __device__ __forceinline__ void accept(bool up, const TT *row, int gl, float tot, int renorm) {
    if constexpr (LP) {
      typename Prec<TT>::T2 rv[LY::H];
      load_pairs_tt<L, E, TT>(row, gl, rv);
      if (up) {
#pragma unroll
        for (int k = 0; k < LY::H; ++k) {
          lam[k] = mul2(lam[k], Prec<TT>::to_f2(rv[k]));
          lh[k] = Prec<TT>::from_f2(lam[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < LY::H; ++k) {
          mu[k] = mul2(mu[k], Prec<TT>::to_f2(rv[k]));
          mh[k] = Prec<TT>::from_f2(mu[k]);
        }
      }
    } else {
      float2 rv[LY::H];
      LY::template load<false>(row, gl, rv, 1.f);
      if (up) {
#pragma unroll
        for (int k = 0; k < LY::H; ++k) lam[k] = mul2(lam[k], rv[k]);
      } else {
#pragma unroll
        for (int k = 0; k < LY::H; ++k) mu[k] = mul2(mu[k], rv[k]);
      }
    }
    if (++since >= renorm) {
      normalize();
    } else if constexpr (LP) {
      // a 16-bit copy's tot carries its factor rounding; taking it as the scale would carry that
      // error into every later proposal until the next normalisation, so the scale is recomputed
      ls = scale_log2();
    } else {
      ls = tot;  // FP32: the accepted proposal's sum is the new scale (to ~1e-7)
    }
  }
  __device__ __forceinline__ float logpsi(uint32_t sw, const float2 *aK, int N, int gl) const {
    return cache_logpsi<L, E>(lam, mu, sw, aK, N, gl) + ls * LN2F;  // log cosh theta_j gains log s_j
  }
};

// Copies the table (and aK) into shared memory when SMEM; returns the table pointer to
// use, or nullptr if the bulk copy timed out (STATUS_TIMEOUT recorded).
template <typename TT, bool SMEM>
__device__ __forceinline__ const TT *stage_table(unsigned char *smem_raw, const void *Rg, const float2 *aK, int N,
                                                 int M_pad, uint64_t *bar, int *status, float2 **saK_out) {
  const uint32_t table_bytes = SMEM ? (uint32_t)N * M_pad * (uint32_t)sizeof(TT) : 0u;
  const TT *R = static_cast<const TT *>(Rg);
  if constexpr (SMEM) {
    if (!load_table(reinterpret_cast<TT *>(smem_raw), R, table_bytes, bar, status)) return nullptr;
    R = reinterpret_cast<const TT *>(smem_raw);
  }
  float2 *saK = reinterpret_cast<float2 *>(smem_raw + ((table_bytes + 15u) & ~15u));
  for (int i = threadIdx.x; i < N; i += blockDim.x) saK[i] = aK[i];
  __syncthreads();
  *saK_out = saK;
  return R;
}

// The N proposals of sweep t of one chain (state sw, cache, accept count nacc, noise zx).
// TRACE: record accept bits and increments (p.acc_bits / p.delta); the untraced loop
// carries no bookkeeping.
template <int L, int E, bool SMEM, typename TT, bool NOISE, bool TRACE>
__device__ __forceinline__ void sweep_once(const SweepParams &p, const TT *R, const float2 *saK, int t, int64_t cc,
                                           bool valid, int gl, uint32_t &sw, ChainCache<L, E, TT> &cache,
                                           int64_t &nacc, float &zx) {
  const int N = p.N, W = p.W, M_pad = p.M_pad;
  const uint32_t sweep_id = p.sweep_offset + (uint32_t)t;
  uint32_t abits = 0u;
  for (int p0 = 0; p0 < N; p0 += 2 * L) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(p0 / 2 + gl), sweep_id, (uint32_t)cc, TAG_SWEEP), p.k0, p.k1);
    const uint32_t site0 = index_from_word(w.x, (uint32_t)N), site1 = index_from_word(w.z, (uint32_t)N);
    const float thr0 = log_uniform(w.y), thr1 = log_uniform(w.w);
    const int np = min(2 * L, N - p0);
    // proposal q = 2k + h of this block: site and log u from lane k's pair h
    auto step = [&](int q, uint32_t site_src, float thr_src) {
      const uint32_t site = __shfl_sync(FULL_MASK, site_src, q >> 1, L);
      const float thr = __shfl_sync(FULL_MASK, thr_src, q >> 1, L);
      const uint32_t word = __shfl_sync(FULL_MASK, sw, site >> 5, L);
      const bool up = (word >> (site & 31)) & 1u;
      const TT *row = R + (size_t)site * M_pad;
      const float tot = cache.logsum(up, row, gl);
      const float2 ak = saK[site];
      float dlt = 2.f * (ak.y - (up ? ak.x : -ak.x)) + (tot - cache.ls) * LN2F;
      float zy = 0.f;
      if constexpr (NOISE) {  // log psi~(y) - log psi~(x) = dlt + zeta(y)/2 - zeta(x)/2
        zy = noise_half<L>(sw ^ (gl == (int)(site >> 5) ? 1u << (site & 31) : 0u), W, p.noise_sigma, p.noise_k0,
                           p.noise_k1);
        dlt += zy - zx;
      }
      const bool acc = 2.f * dlt > thr;
      if (acc) {
        cache.template accept<SMEM>(up, row, gl, tot, p.renorm);
        if (gl == (int)(site >> 5)) sw ^= 1u << (site & 31);
        ++nacc;
        if constexpr (NOISE) zx = zy;
      }
      if constexpr (TRACE) {
        const int pq = p0 + q;
        if (p.acc_bits) {
          abits |= (acc ? 1u : 0u) << (pq & 31);
          if ((pq & 31) == 31 || pq == N - 1) {
            if (valid && gl == 0) p.acc_bits[((int64_t)cc * p.n_sweeps + t) * W + (pq >> 5)] = abits;
            abits = 0u;
          }
        }
        if (p.delta && valid && gl == 0) p.delta[((int64_t)cc * p.n_sweeps + t) * N + pq] = dlt;
      }
    };
    for (int q = 0; q < np; q += 2) {
      step(q, site0, thr0);
      if (q + 1 < np) step(q + 1, site1, thr1);
    }
  }
}

// All sweeps of the chain base + (lane / L) for a group of L lanes; chains at or beyond
// `limit` are idle (they shadow chain limit - 1 and write nothing).  R is the table (shared
// or global memory), saK the (a_i, K_i) pairs in shared memory.
template <int L, int E, bool SMEM, typename TT, bool NOISE = false>
__device__ __forceinline__ void sweep_chain(const SweepParams &p, const TT *R, const float2 *saK, int64_t base,
                                            int64_t limit) {
  const int lane = threadIdx.x & 31;
  const int grp = lane / L, gl = lane % L;
  const int N = p.N, W = p.W, M_pad = p.M_pad;
  const int64_t c = base + grp;
  const bool valid = c < limit;
  const int64_t cc = valid ? c : limit - 1;
  uint32_t sw = gl < W ? p.state[cc * W + gl] : 0u;
  ChainCache<L, E, TT> cache;
  cache.build(sw, p.Wt, p.b, N, W, M_pad, gl);
  int64_t nacc = 0;
  float zx = 0.f;  // noisy RBM: zeta(x) / 2 of the chain's configuration
  if constexpr (NOISE) zx = noise_half<L>(sw, W, p.noise_sigma, p.noise_k0, p.noise_k1);
  const bool trace = p.acc_bits != nullptr || p.delta != nullptr;

  for (int t = 0; t < p.n_sweeps; ++t) {
    if (trace)
      sweep_once<L, E, SMEM, TT, NOISE, true>(p, R, saK, t, cc, valid, gl, sw, cache, nacc, zx);
    else
      sweep_once<L, E, SMEM, TT, NOISE, false>(p, R, saK, t, cc, valid, gl, sw, cache, nacc, zx);
    if (t >= p.burn_in) {
      const int64_t row = (int64_t)(t - p.burn_in) * p.C + cc;
      if (p.samples && valid && gl < W) p.samples[row * W + gl] = sw;
      if (p.logpsi) {
        const float lp = cache.logpsi(sw, saK, N, gl);
        if (valid && gl == 0) p.logpsi[row] = lp;
      }
    }
    if ((t + 1) % p.refresh == 0 && t + 1 < p.n_sweeps) cache.build(sw, p.Wt, p.b, N, W, M_pad, gl);
  }
  if (valid && gl < W) p.state[cc * W + gl] = sw;
  if (valid && gl == 0 && p.n_acc) p.n_acc[cc] = nacc;
}

// One group of L lanes runs one chain for all sweeps; the block shares one copy of
// the table in shared memory (or reads it through L2 when it does not fit).
template <int L, int E, bool SMEM, typename TT, bool NOISE = false>
__global__ void __launch_bounds__(sweep_threads(E), 1) rbm_sweep_kernel(const SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  float2 *saK;
  const TT *R = stage_table<TT, SMEM>(smem_raw, p.R, p.aK, p.N, p.M_pad, &bar, p.status, &saK);
  if (!R) return;
  constexpr int G = 32 / L;
  const int warp = threadIdx.x >> 5;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * G;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * G; base < p.C; base += stride)
    sweep_chain<L, E, SMEM, TT, NOISE>(p, R, saK, base, p.C);
}

struct ElocParams {
  const uint32_t *cfg;
  const int32_t *sites;  // flip-delta mode: the site flipped for each row
  const void *R;
  const float2 *aK;
  const float *Wt;
  const float *b;
  const int2 *bonds;
  float *out;
  int *status;
  int64_t n;
  int n_bonds, N, W, M_pad;
  float J, h;
  int64_t n_chains;  // chain-ordered kernel: rows are k * n_chains + c
  int refresh;       // chain-ordered kernel: theta rebuilt from scratch every this many samples
};

// eps(x) of the TFIM from the configuration's cache (Eq. TFIM, App. I Eq. local_energies):
// J sum_<ij> s_i s_j + h sum_i exp(log psi(flip_i x) - log psi(x)).
//
// With 32 lanes per configuration the N flips go in blocks of 8: each lane forms its partial
// sum of log2 g for the 8 flips, a recursive-halving exchange (lane bits 4, 3, 2, then 1 and
// 0) leaves lane l with the full sum of flip 4 b4 + 2 b3 + b2 of the block, and lanes with
// b1 = b0 = 0 add that flip's exp.  A block whose sums are not all finite is recomputed flip by
// flip on the exact path.  Narrower groups evaluate two flips per iteration with a group sum.
template <int L, int E, typename TT>
__device__ __forceinline__ float tfim_eloc_value(const ChainCache<L, E, TT> &cache, uint32_t sw, const ElocParams &p,
                                                 const TT *R, const float2 *saK, int gl) {
  const int N = p.N, M_pad = p.M_pad;
  float d = 0.f;
  for (int b0 = 0; b0 < p.n_bonds; b0 += L) {
    const int bi = min(b0 + gl, p.n_bonds - 1);
    const int2 bd = p.bonds[bi];
    const uint32_t wa = __shfl_sync(FULL_MASK, sw, bd.x >> 5, L);
    const uint32_t wb = __shfl_sync(FULL_MASK, sw, bd.y >> 5, L);
    const uint32_t sa = (wa >> (bd.x & 31)) & 1u, sb = (wb >> (bd.y & 31)) & 1u;
    if (b0 + gl < p.n_bonds) d += sa == sb ? 1.f : -1.f;
  }
  d = p.J * group_allsum<L>(d);
  float off = 0.f;
  if constexpr (L == 32) {
    constexpr int FB = 8;  // flips per block (8 sites of one word: blocks start at multiples of 8)
    for (int i0 = 0; i0 < N; i0 += FB) {
      const uint32_t word = __shfl_sync(FULL_MASK, sw, i0 >> 5, L);
      float v[FB];
#pragma unroll
      for (int u = 0; u < FB; ++u) {
        const int i = min(i0 + u, N - 1);  // a clamped tail site stays in this word; its term is dropped
        v[u] = cache.partial((word >> (i & 31)) & 1u, R + (size_t)i * M_pad, gl);
      }
      // recursive halving: after the steps on lane bits 4, 3, 2 lane l holds the sum over the 8
      // lanes sharing its low two bits for flip u = 4 b4 + 2 b3 + b2; bits 1 and 0 finish it
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        const int half = FB >> (h + 1);            // 4, 2, 1 values kept
        const bool hi = (gl >> (4 - h)) & 1;       // lane bits 4, 3, 2
#pragma unroll
        for (int q = 0; q < half; ++q) {
          const float keep = hi ? v[q + half] : v[q];
          const float send = hi ? v[q] : v[q + half];
          v[q] = keep + __shfl_xor_sync(FULL_MASK, send, 16 >> h);
        }
      }
      float t = v[0];
      t += __shfl_xor_sync(FULL_MASK, t, 2);
      t += __shfl_xor_sync(FULL_MASK, t, 1);
      const int u = ((gl >> 4) & 1) * 4 + ((gl >> 3) & 1) * 2 + ((gl >> 2) & 1);
      const int i = i0 + u;
      if (__any_sync(FULL_MASK, !isfinite(t))) {  // exact path for the block
        for (int w = 0; w < FB && i0 + w < N; ++w) {
          const int ii = i0 + w;
          const bool up = (word >> (ii & 31)) & 1u;
          const float tot = group_allsum<L>(cache.partial_exact(up, R + (size_t)ii * M_pad, gl));
          const float2 ak = saK[ii];
          if (gl == 0) off += expf(2.f * (ak.y - (up ? ak.x : -ak.x)) + (tot - cache.ls) * LN2F);
        }
      } else if ((gl & 3) == 0 && i < N) {
        const bool up = (word >> (i & 31)) & 1u;
        const float2 ak = saK[i];
        // e^{Delta} as 2^{Delta / ln 2} (ex2.approx: the argument's rounding adds at most
        // |Delta| 2^-24 relative, a few ulp beyond)
        off += ex2_approx(2.f * LOG2EF * (ak.y - (up ? ak.x : -ak.x)) + (t - cache.ls));
      }
    }
    off = group_allsum<L>(off);
  } else {
    for (int i = 0; i < N; i += 2) {
      const int i1 = min(i + 1, N - 1);
      const uint32_t word0 = __shfl_sync(FULL_MASK, sw, i >> 5, L);
      const uint32_t word1 = __shfl_sync(FULL_MASK, sw, i1 >> 5, L);
      const bool up0 = (word0 >> (i & 31)) & 1u, up1 = (word1 >> (i1 & 31)) & 1u;
      const float tot0 = cache.logsum(up0, R + (size_t)i * M_pad, gl);
      const float tot1 = cache.logsum(up1, R + (size_t)i1 * M_pad, gl);
      const float2 ak0 = saK[i], ak1 = saK[i1];
      off += expf(2.f * (ak0.y - (up0 ? ak0.x : -ak0.x)) + tot0 * LN2F);
      if (i + 1 < N) off += expf(2.f * (ak1.y - (up1 ? ak1.x : -ak1.x)) + tot1 * LN2F);
    }
  }
  return d + p.h * off;
}

// TFIM local energy (Eq. TFIM, App. I Eq. local_energies), FLIP = false:
//   eps(x) = J sum_<ij> s_i s_j + h sum_i exp(log psi(flip_i x) - log psi(x)),
// two independent sites per iteration.  FLIP = true: out[x] = log psi(flip_{sites[x]} x)
// - log psi(x), the increment the sampler uses for that proposal (Sec. 3.1).
template <int L, int E, bool SMEM, typename TT, bool FLIP>
__global__ void __launch_bounds__(eloc_threads(E), 1) rbm_tfim_eloc_kernel(const ElocParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  float2 *saK;
  const TT *R = stage_table<TT, SMEM>(smem_raw, p.R, p.aK, p.N, p.M_pad, &bar, p.status, &saK);
  if (!R) return;
  const int N = p.N, W = p.W, M_pad = p.M_pad;

  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / L, gl = lane % L;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * G;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * G; base < p.n; base += stride) {
    const int64_t x = min(base + grp, p.n - 1);
    const uint32_t sw = gl < W ? p.cfg[x * W + gl] : 0u;
    ChainCache<L, E, TT> cache;
    cache.build(sw, p.Wt, p.b, N, W, M_pad, gl);
    if constexpr (FLIP) {
      const int i = p.sites[x];
      const uint32_t word = __shfl_sync(FULL_MASK, sw, i >> 5, L);
      const bool up = (word >> (i & 31)) & 1u;
      const float tot = cache.logsum(up, R + (size_t)i * M_pad, gl);
      const float2 ak = saK[i];
      if (base + grp < p.n && gl == 0) p.out[x] = 2.f * (ak.y - (up ? ak.x : -ak.x)) + tot * LN2F;
    } else {
      const float e = tfim_eloc_value<L, E, TT>(cache, sw, p, R, saK, gl);
      if (base + grp < p.n && gl == 0) p.out[x] = e;
    }
  }
}

// Local energies of sweep-major samples of n_chains chains (row k * n_chains + c), one group
// per chain walking its samples in order: theta = W s + b is updated only for the spins that
// changed since the chain's previous sample (theta += 2 s'_i W_i), rebuilt from scratch every
// `refresh` samples, and each sample's eps is evaluated as in rbm_tfim_eloc_kernel.
template <int L, int E, bool SMEM>
__global__ void __launch_bounds__(eloc_threads(E), 1) rbm_tfim_eloc_chains_kernel(const ElocParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  float2 *saK;
  const float *R = stage_table<float, SMEM>(smem_raw, p.R, p.aK, p.N, p.M_pad, &bar, p.status, &saK);
  if (!R) return;
  using LY = Lay<L, E>;
  const int N = p.N, W = p.W, M_pad = p.M_pad;
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / L, gl = lane % L;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * G;
  const int64_t C = p.n_chains, K = p.n / p.n_chains;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * G; base < C; base += stride) {
    const int64_t c = base + grp;
    const bool valid = c < C;
    const int64_t cc = valid ? c : C - 1;
    float2 th[LY::H];
    ChainCache<L, E, float> cache;
    uint32_t prev = 0u;
    for (int64_t k = 0; k < K; ++k) {
      const int64_t x = k * C + cc;
      const uint32_t sw = gl < W ? p.cfg[x * W + gl] : 0u;
      if (k % p.refresh == 0) {
        compute_theta<L, E>(th, sw, p.Wt, p.b, N, W, M_pad, gl);
      } else {
        for (int wi = 0; wi < W; ++wi) {
          uint32_t m = __shfl_sync(FULL_MASK, sw ^ prev, wi, L);
          const uint32_t now = __shfl_sync(FULL_MASK, sw, wi, L);
          while (m) {  // uniform within the group
            const int bit = __ffs(m) - 1;
            m &= m - 1u;
            const float s2 = ((now >> bit) & 1u) ? 2.f : -2.f;
            float2 w[LY::H];
            LY::template load<true>(p.Wt + (size_t)(32 * wi + bit) * M_pad, gl, w, 0.f);
            const float2 s22 = make_float2(s2, s2);
#pragma unroll
            for (int q = 0; q < LY::H; ++q) th[q] = fma2(s22, w[q], th[q]);
          }
        }
      }
      cache.from_theta(th);
      const float e = tfim_eloc_value<L, E, float>(cache, sw, p, R, saK, gl);
      if (valid && gl == 0) p.out[x] = e;
      prev = sw;
    }
  }
}

// ------------------------------------------------------------------------------------
// Launch configuration: one CTA per SM shares one table copy; warps per CTA from the
// kernel's register use, then trimmed so that every CTA runs the same number of rounds.
template <typename K>
cudaError_t launch_persistent(K kern, const nqs_ctx *c, int64_t groups, int G, size_t shm, cudaStream_t s,
                              const void *arg) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  const int regs_alloc = (std::max(fa.numRegs, 16) + 7) / 8 * 8;
  int warps = std::max(1, std::min(fa.maxThreadsPerBlock / 32, 65536 / (regs_alloc * 32)));
  const int64_t warps_needed = (groups + G - 1) / G;
  int64_t blocks = std::min<int64_t>(c->num_sms, (warps_needed + warps - 1) / warps);
  if (blocks < c->num_sms) {  // spread small jobs over more SMs with fewer warps each
    blocks = std::min<int64_t>(c->num_sms, warps_needed);
    warps = (int)std::max<int64_t>(1, (warps_needed + blocks - 1) / blocks);
  } else {  // equal rounds: the fewest warps per CTA that keep the round count
    const int64_t rounds = (warps_needed + blocks * warps - 1) / (blocks * warps);
    warps = (int)((warps_needed + blocks * rounds - 1) / (blocks * rounds));
  }
  void *args[] = {const_cast<void *>(arg)};
  return cudaLaunchKernel((const void *)kern, dim3((unsigned)blocks), dim3(warps * 32), args, shm, s);
}

template <typename TT>
size_t table_smem(const nqs_ctx *c, bool *fits) {
  const size_t table = ((size_t)c->N * c->M_pad * sizeof(TT) + 15) & ~size_t(15);
  const size_t extra = (size_t)c->N * sizeof(float2) + 16;
  *fits = table + extra + 256 <= (size_t)c->smem_optin;  // + static mbarrier
  return (*fits ? table : 0) + extra;
}

template <typename TT>
struct Runners {
  template <int L, int E>
  struct Sweep {
    static cudaError_t run(const nqs_ctx *c, const SweepParams &p, cudaStream_t s) {
      bool fits;
      const size_t shm = table_smem<TT>(c, &fits);
      return fits ? launch_persistent(rbm_sweep_kernel<L, E, true, TT>, c, p.C, 32 / L, shm, s, &p)
                  : launch_persistent(rbm_sweep_kernel<L, E, false, TT>, c, p.C, 32 / L, shm, s, &p);
    }
  };
  template <int L, int E>
  struct NoisySweep {  // noisy RBM (Sec. 4.1)
    static cudaError_t run(const nqs_ctx *c, const SweepParams &p, cudaStream_t s) {
      bool fits;
      const size_t shm = table_smem<TT>(c, &fits);
      return fits ? launch_persistent(rbm_sweep_kernel<L, E, true, TT, true>, c, p.C, 32 / L, shm, s, &p)
                  : launch_persistent(rbm_sweep_kernel<L, E, false, TT, true>, c, p.C, 32 / L, shm, s, &p);
    }
  };
  template <int L, int E>
  struct ElocChains {  // chain-ordered local energy (FP32 tables)
    static cudaError_t run(const nqs_ctx *c, const ElocParams &p, cudaStream_t s) {
      bool fits;
      const size_t shm = table_smem<float>(c, &fits);
      return fits ? launch_persistent(rbm_tfim_eloc_chains_kernel<L, E, true>, c, p.n_chains, 32 / L, shm, s, &p)
                  : launch_persistent(rbm_tfim_eloc_chains_kernel<L, E, false>, c, p.n_chains, 32 / L, shm, s, &p);
    }
  };
  template <int L, int E>
  struct Eloc {
    static cudaError_t run(const nqs_ctx *c, const ElocParams &p, cudaStream_t s) {
      bool fits;
      const size_t shm = table_smem<TT>(c, &fits);
      if (p.sites)
        return fits ? launch_persistent(rbm_tfim_eloc_kernel<L, E, true, TT, true>, c, p.n, 32 / L, shm, s, &p)
                    : launch_persistent(rbm_tfim_eloc_kernel<L, E, false, TT, true>, c, p.n, 32 / L, shm, s, &p);
      return fits ? launch_persistent(rbm_tfim_eloc_kernel<L, E, true, TT, false>, c, p.n, 32 / L, shm, s, &p)
                  : launch_persistent(rbm_tfim_eloc_kernel<L, E, false, TT, false>, c, p.n, 32 / L, shm, s, &p);
    }
  };
};

// dispatch over the instantiated hidden-unit widths per lane (L = 32)
template <template <int, int> class F, typename... A>
cudaError_t dispatch_l32(int E, A &&...args) {
#define NQS_CASE(EE) \
  if (E == EE) return F<32, EE>::run(args...);
  NQS_CASE(1) NQS_CASE(2) NQS_CASE(3) NQS_CASE(4) NQS_CASE(5) NQS_CASE(6) NQS_CASE(7) NQS_CASE(8) NQS_CASE(9)
  NQS_CASE(10) NQS_CASE(11) NQS_CASE(12) NQS_CASE(13) NQS_CASE(14) NQS_CASE(16) NQS_CASE(18) NQS_CASE(20)
  NQS_CASE(24) NQS_CASE(28) NQS_CASE(32)
#undef NQS_CASE
  return cudaErrorInvalidConfiguration;
}

// dispatch over (L, E): L = 32 for every instantiated width; L = 16 and L = 8 variants
// (two or four chains per warp) for the widths the tuner may pick.
template <template <int, int> class F, typename... A>
cudaError_t dispatch_le(int L, int E, A &&...args) {
#define NQS_CASE(LL, EE) \
  if (L == LL && E == EE) return F<LL, EE>::run(args...);
  NQS_CASE(8, 4) NQS_CASE(16, 2) NQS_CASE(16, 4) NQS_CASE(16, 8) NQS_CASE(16, 16) NQS_CASE(16, 26)
  NQS_CASE(16, 28) NQS_CASE(16, 32)
#undef NQS_CASE
  if (L == 32) return dispatch_l32<F>(E, args...);
  return cudaErrorInvalidConfiguration;
}

}  // namespace rbmk
}  // namespace nqs
