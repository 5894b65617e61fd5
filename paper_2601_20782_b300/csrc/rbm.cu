// RBM path of the hot loop: sampling-copy preparation, chain initialisation,
// Metropolis-Hastings sweeps with an incremental per-chain cache, log psi,
// TFIM local energies, per-sample log-derivatives O_k and the force.
//
// RBM (App. G), with spins s in {-1,+1}:
//     log psi(s) = sum_i a_i s_i + sum_j log cosh(theta_j),  theta = W s + b.
//
// Per-chain cache.  Instead of theta_j the sweep keeps the pair
//     lam_j = e^{theta_j} / (e^{theta_j} + e^{-theta_j}),  mu_j = 1 - lam_j,
// each stored as its own FP32 number (so neither loses relative precision).
// Flipping site i (d_j = 2 W_ji s_i) multiplies cosh(theta_j) by
//     cosh(theta_j - d_j) / cosh(theta_j) = lam_j e^{-d_j} + mu_j e^{d_j}
//                                        = e^{2 W_ji} g_j,
//     g_j = mu_j + lam_j R_ji (s_i = +1),   g_j = lam_j + mu_j R_ji (s_i = -1),
// with the table R_ji = exp(-4 W_ji).  Hence
//     log psi(y) - log psi(x) = 2 (K_i - a_i s_i) + sum_j log g_j,  K_i = sum_j W_ji,
// one FMA and one multiply per hidden unit and no cancellation.  An accepted
// flip updates the cache multiplicatively (lam/mu = e^{2 theta}):
//     s_i = +1: lam' = lam R / g, mu' = mu / g;   s_i = -1: lam' = lam / g, mu' = mu R / g,
// and log cosh(theta_j) = -1/2 log(4 lam_j mu_j).  The cache is rebuilt from
// theta = W s + b every `refresh` sweeps so rounding cannot accumulate.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nqs {
namespace {

constexpr uint32_t BULK_CHUNK = 32768;

// Threads per CTA bound for E cached units per lane (register budget per thread).
constexpr int threads_for_regs(int regs) {
  int w = 65536 / (32 * regs);
  w = w < 2 ? 2 : (w > 32 ? 32 : w);
  return 32 * w;
}
// sweep: the cache pairs stay live, the row and the factors are streamed
constexpr int sweep_threads(int E) { return threads_for_regs(2 * E + 56); }
// local energy: the cache plus two sites' rows and factors in flight
constexpr int eloc_threads(int E) { return threads_for_regs(3 * E + 48); }
constexpr uint32_t WAIT_POLLS = 1u << 22;

// ------------------------------------------------------------------------------------
// sampling-copy preparation (Sec. 4.2: FP64 master -> rounded sampling copy)
template <typename TT>
__device__ __forceinline__ TT round_to(double x);
template <>
__device__ __forceinline__ float round_to<float>(double x) { return static_cast<float>(x); }
template <>
__device__ __forceinline__ __half round_to<__half>(double x) { return __double2half(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 round_to<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename TT>
__global__ void rbm_prepare_kernel(const double *__restrict__ p, int N, int M, int M_pad, float *a, float *b,
                                   float *Wt, TT *R, float *Wm, float *bm, int *status, double wmax) {
  const int64_t total = (int64_t)N * M_pad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / M_pad), j = (int)(idx % M_pad);
    const double w = j < M ? p[N + M + (int64_t)j * N + i] : 0.0;
    const float wr = to_f(round_to<TT>(w));
    Wt[idx] = wr;
    R[idx] = round_to<TT>(exp(-4.0 * (double)wr));
    if (j < M) Wm[(int64_t)i * M + j] = (float)w;
    if (!(fabs(w) <= wmax)) atomicOr(status, STATUS_RANGE);
    if (idx < N) a[idx] = to_f(round_to<TT>(p[idx]));
    if (idx < M_pad) {
      b[idx] = idx < M ? to_f(round_to<TT>(p[N + idx])) : 0.f;
      if (idx < M) bm[idx] = (float)p[N + idx];
    }
  }
}

// aK[i] = (a_i, K_i = sum_j W_ji) from the rounded copy; one warp per site, FP64 sum.
__global__ void rbm_colsum_kernel(const float *Wt, const float *a, int N, int M_pad, float2 *aK) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  double s = 0.0;
  for (int j = lane; j < M_pad; j += 32) s += Wt[(int64_t)warp * M_pad + j];
  s = group_allsum<32>(s);
  if (lane == 0) aK[warp] = make_float2(a[warp], (float)s);
}

// ------------------------------------------------------------------------------------
// chain initialisation (same draws as the oracle's init_spins_random / _balanced)
__global__ void init_random_kernel(uint32_t *state, int64_t C, int N, int W, uint32_t k0, uint32_t k1) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
    for (int b = 0; b < (N + 127) / 128; ++b) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)b, 0u, (uint32_t)c, TAG_INIT), k0, k1);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
      for (int q = 0; q < 4; ++q) {
        const int wi = 4 * b + q;
        if (wi >= W) break;
        const int nb = N - 32 * wi;
        state[c * W + wi] = nb >= 32 ? ws[q] : (ws[q] & ((1u << nb) - 1u));
      }
    }
  }
}

// Fisher-Yates shuffle of (+1 x N/2, -1 x N/2), from the top; N <= 1024.
__global__ void init_balanced_kernel(uint32_t *state, int64_t C, int N, int W, uint32_t k0, uint32_t k1) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits[32];
    for (int q = 0; q < 32; ++q) bits[q] = 0u;
    for (int i = 0; i < N / 2; ++i) bits[i >> 5] |= 1u << (i & 31);
    uint4 w = make_uint4(0, 0, 0, 0);
    int cur_blk = -1;
    for (int i = N - 1; i >= 1; --i) {
      if ((i >> 2) != cur_blk) {
        cur_blk = i >> 2;
        w = philox4x32_10(make_uint4((uint32_t)cur_blk, 1u, (uint32_t)c, TAG_INIT), k0, k1);
      }
      const uint32_t ws = (i & 3) == 0 ? w.x : (i & 3) == 1 ? w.y : (i & 3) == 2 ? w.z : w.w;
      const int j = (int)index_from_word(ws, (uint32_t)(i + 1));
      const uint32_t bi = (bits[i >> 5] >> (i & 31)) & 1u, bj = (bits[j >> 5] >> (j & 31)) & 1u;
      if (bi != bj) {
        bits[i >> 5] ^= 1u << (i & 31);
        bits[j >> 5] ^= 1u << (j & 31);
      }
    }
    for (int q = 0; q < W; ++q) state[c * W + q] = bits[q];
  }
}

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

__device__ __forceinline__ void sigmoid_pair(float th, float &lam, float &mu) {
  const float e = expf(-2.f * fabsf(th));
  const float p = 1.f / (1.f + e);
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
    part += log2f(4.f * lam[k].x * mu[k].x) + log2f(4.f * lam[k].y * mu[k].y);
  return visible_term<L>(sw, aK, N, gl) - 0.5f * LN2F * group_allsum<L>(part);
}

// g for a flip of a site with spin `up`: mu + lam R (up) or lam + mu R (down)
template <int H>
__device__ __forceinline__ void flip_factors(bool up, const float2 (&lam)[H], const float2 (&mu)[H],
                                             const float2 (&rv)[H], float2 (&g)[H]) {
  if (up) {
#pragma unroll
    for (int k = 0; k < H; ++k) g[k] = fma2(lam[k], rv[k], mu[k]);
  } else {
#pragma unroll
    for (int k = 0; k < H; ++k) g[k] = fma2(mu[k], rv[k], lam[k]);
  }
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
  float part = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < LY::H; k0 += 4) {
    float2 pr = up ? fma2(lam[k0], rv[k0], mu[k0]) : fma2(mu[k0], rv[k0], lam[k0]);
#pragma unroll
    for (int k = k0 + 1; k < (k0 + 4 < LY::H ? k0 + 4 : LY::H); ++k)
      pr = mul2(pr, up ? fma2(lam[k], rv[k], mu[k]) : fma2(mu[k], rv[k], lam[k]));
    part += lg2_approx(pr.x * pr.y);
  }
  return part;
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

// Group sum of the lane partials; see sum_log2 for the reduction and its exact fallback.
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

// sum_j log2 g_j over the group: products of up to 8 factors (4 pairs) per MUFU lg2.
// With one chain per warp the lane partials are added exactly as 2^-20 fixed-point
// integers by one redux.sync (a 32-lane sum in one instruction instead of a 5-stage
// shuffle tree); each partial is rounded to 2^-21, so the sum carries at most
// 32 * 2^-21 absolute error in log2 units.  A product that leaves the normal FP32
// range, or a partial beyond +-2^10, sends the group to the exact path: one accurate
// log per factor and a floating-point butterfly.
template <int L, int H>
__device__ __forceinline__ float sum_log2(const float2 (&g)[H]) {
  float part = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < H; k0 += 4) {
    float2 pr = g[k0];
#pragma unroll
    for (int k = k0 + 1; k < (k0 + 4 < H ? k0 + 4 : H); ++k) pr = mul2(pr, g[k]);
    part += lg2_approx(pr.x * pr.y);
  }
  if constexpr (L == 32) {
    const bool bad = !(fabsf(part) < 1024.f);  // also catches inf / nan
    if (!__any_sync(FULL_MASK, bad)) {
      const int q = __float2int_rn(part * 1048576.f);
      return (float)__reduce_add_sync(FULL_MASK, q) * 9.5367431640625e-7f;
    }
  } else {
    const float tot = group_allsum<L>(part);
    if (!__any_sync(FULL_MASK, !isfinite(tot))) return tot;
  }
  float p2 = 0.f;
#pragma unroll
  for (int k = 0; k < H; ++k) p2 += log2f(g[k].x) + log2f(g[k].y);
  return group_allsum<L>(p2);
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
template <int L, int E, bool SMEM>
__device__ __forceinline__ void accept_update(bool up, float2 (&lam)[Lay<L, E>::H], float2 (&mu)[Lay<L, E>::H],
                                              const float *row, int gl) {
  using LY = Lay<L, E>;
  auto upd = [&](int k, float2 r) {
    if (up) {
      const float2 g = fma2(lam[k], r, mu[k]);
      const float2 inv = make_float2(rcp_approx(g.x), rcp_approx(g.y));
      lam[k] = mul2(mul2(lam[k], r), inv);
      mu[k] = mul2(mu[k], inv);
    } else {
      const float2 g = fma2(mu[k], r, lam[k]);
      const float2 inv = make_float2(rcp_approx(g.x), rcp_approx(g.y));
      mu[k] = mul2(mul2(mu[k], r), inv);
      lam[k] = mul2(lam[k], inv);
    }
  };
#pragma unroll
  for (int v = 0; v < LY::V; ++v) {
    float4 q;
    q = *reinterpret_cast<const float4 *>(row + 4 * (v * L + gl));
    upd(2 * v, make_float2(q.x, q.y));
    upd(2 * v + 1, make_float2(q.z, q.w));
  }
  float t[3] = {1.f, 1.f, 1.f};
#pragma unroll
  for (int k = 0; k < LY::T; ++k) {
    t[k] = row[4 * LY::V * L + k * L + gl];
  }
  if constexpr (LY::T == 1) upd(2 * LY::V, make_float2(t[0], 1.f));
  if constexpr (LY::T == 2) upd(2 * LY::V, make_float2(t[0], t[1]));
  if constexpr (LY::T == 3) {
    upd(2 * LY::V, make_float2(t[0], t[1]));
    upd(2 * LY::V + 1, make_float2(t[2], 1.f));
  }
}

struct SweepParams {
  const float *R;
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
  uint32_t sweep_offset, k0, k1;
};

// log u for u = k 2^-24 (k = 0 gives -inf: always accept).  Accepting iff
// 2 dlogpsi > log u is the rule u < exp(2 dlogpsi).
__device__ __forceinline__ float log_uniform(uint32_t w) {
  const uint32_t k = w >> 8;
  return k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
}

// One group of L lanes runs one chain for all sweeps; the block shares one copy of
// the R table in shared memory (or reads it through L2 when it does not fit).
template <int L, int E, bool SMEM>
__global__ void __launch_bounds__(sweep_threads(E), 1) rbm_sweep_f32_kernel(const SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  const float *R = p.R;
  const uint32_t table_bytes = SMEM ? (uint32_t)p.N * p.M_pad * 4u : 0u;
  if constexpr (SMEM) {
    if (!load_table(reinterpret_cast<float *>(smem_raw), p.R, table_bytes, &bar, p.status)) return;
    R = reinterpret_cast<const float *>(smem_raw);
  }
  float2 *saK = reinterpret_cast<float2 *>(smem_raw + table_bytes);
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) saK[i] = p.aK[i];
  __syncthreads();

  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / L, gl = lane % L;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * G;
  const int N = p.N, W = p.W, M_pad = p.M_pad;

  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * G; base < p.C; base += stride) {
    const int64_t c = base + grp;
    const bool valid = c < p.C;
    const int64_t cc = valid ? c : p.C - 1;  // idle groups shadow the last chain and write nothing
    uint32_t sw = gl < W ? p.state[cc * W + gl] : 0u;
    using LY = Lay<L, E>;
    float2 lam[LY::H], mu[LY::H];
    build_cache<L, E>(lam, mu, sw, p.Wt, p.b, N, W, M_pad, gl);
    int64_t nacc = 0;

    for (int t = 0; t < p.n_sweeps; ++t) {
      const uint32_t sweep_id = p.sweep_offset + (uint32_t)t;
      uint32_t abits = 0u;
      for (int p0 = 0; p0 < N; p0 += 2 * L) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(p0 / 2 + gl), sweep_id, (uint32_t)cc, TAG_SWEEP),
                                      p.k0, p.k1);
        const uint32_t site0 = index_from_word(w.x, (uint32_t)N), site1 = index_from_word(w.z, (uint32_t)N);
        const float thr0 = log_uniform(w.y), thr1 = log_uniform(w.w);
        const int np = min(2 * L, N - p0);
        for (int q = 0; q < np; ++q) {
          const int src = q >> 1;
          const uint32_t site = __shfl_sync(FULL_MASK, (q & 1) ? site1 : site0, src, L);
          const float thr = __shfl_sync(FULL_MASK, (q & 1) ? thr1 : thr0, src, L);
          const uint32_t word = __shfl_sync(FULL_MASK, sw, site >> 5, L);
          const bool up = (word >> (site & 31)) & 1u;
          const float tot = flip_logsum<L, E>(up, lam, mu, R + (size_t)site * M_pad, gl);
          const float2 ak = saK[site];
          const float dlt = 2.f * (ak.y - (up ? ak.x : -ak.x)) + tot * LN2F;
          const bool acc = 2.f * dlt > thr;
          if (acc) {
            accept_update<L, E, SMEM>(up, lam, mu, R + (size_t)site * M_pad, gl);
            if (gl == (int)(site >> 5)) sw ^= 1u << (site & 31);
            ++nacc;
          }
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
      }
      if (t >= p.burn_in) {
        const int64_t row = (int64_t)(t - p.burn_in) * p.C + cc;
        if (p.samples && valid && gl < W) p.samples[row * W + gl] = sw;
        if (p.logpsi) {
          const float lp = cache_logpsi<L, E>(lam, mu, sw, saK, N, gl);
          if (valid && gl == 0) p.logpsi[row] = lp;
        }
      }
      if ((t + 1) % p.refresh == 0 && t + 1 < p.n_sweeps) build_cache<L, E>(lam, mu, sw, p.Wt, p.b, N, W, M_pad, gl);
    }
    if (valid && gl < W) p.state[cc * W + gl] = sw;
    if (valid && gl == 0 && p.n_acc) p.n_acc[cc] = nacc;
  }
}

// ------------------------------------------------------------------------------------
// log psi by direct evaluation: log cosh z = |z| + log1p(exp(-2|z|)) - log 2
template <int L, int E>
__global__ void rbm_logpsi_kernel(const uint32_t *__restrict__ cfg, int64_t n, const float *Wt, const float *b,
                                  const float2 *aK, int N, int W, int M_pad, float *out) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, grp = lane / L, gl = lane % L;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x >> 5) * G;
  for (int64_t base = gw * G; base < n; base += stride) {
    const int64_t x = min(base + grp, n - 1);
    const uint32_t sw = gl < W ? cfg[x * W + gl] : 0u;
    float2 th[Lay<L, E>::H];
    compute_theta<L, E>(th, sw, Wt, b, N, W, M_pad, gl);
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < Lay<L, E>::H; ++k) {  // a dummy slot has theta = 0: log cosh 0 = 0
      const float zx = fabsf(th[k].x), zy = fabsf(th[k].y);
      part += (zx + log1pf(expf(-2.f * zx)) - LN2F) + (zy + log1pf(expf(-2.f * zy)) - LN2F);
    }
    const float lp = visible_term<L>(sw, aK, N, gl) + group_allsum<L>(part);
    if (base + grp < n && gl == 0) out[x] = lp;
  }
}

// ------------------------------------------------------------------------------------
// TFIM local energy (Eq. TFIM, App. I Eq. local_energies):
//   eps(x) = J sum_<ij> s_i s_j + h sum_i exp(log psi(flip_i x) - log psi(x)).
template <int L, int E, bool SMEM>
__global__ void __launch_bounds__(eloc_threads(E), 1) rbm_tfim_eloc_kernel(const uint32_t *__restrict__ cfg, int64_t n,
                                                                 const float *Rg, const float2 *aK,
                                                                 const float *Wt, const float *b,
                                                                 const int2 *bonds, int n_bonds, float J,
                                                                 float h, int N, int W, int M_pad, float *eloc,
                                                                 int *status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  const float *R = Rg;
  const uint32_t table_bytes = SMEM ? (uint32_t)N * M_pad * 4u : 0u;
  if constexpr (SMEM) {
    if (!load_table(reinterpret_cast<float *>(smem_raw), Rg, table_bytes, &bar, status)) return;
    R = reinterpret_cast<const float *>(smem_raw);
  }
  float2 *saK = reinterpret_cast<float2 *>(smem_raw + table_bytes);
  for (int i = threadIdx.x; i < N; i += blockDim.x) saK[i] = aK[i];
  __syncthreads();

  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / L, gl = lane % L;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * wpb * G;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + warp) * G; base < n; base += stride) {
    const int64_t x = min(base + grp, n - 1);
    const uint32_t sw = gl < W ? cfg[x * W + gl] : 0u;
    using LY = Lay<L, E>;
    float2 lam[LY::H], mu[LY::H];
    build_cache<L, E>(lam, mu, sw, Wt, b, N, W, M_pad, gl);
    // diagonal: J sum over bonds of s_a s_b
    float d = 0.f;
    for (int b0 = 0; b0 < n_bonds; b0 += L) {
      const int bi = min(b0 + gl, n_bonds - 1);
      const int2 bd = bonds[bi];
      const uint32_t wa = __shfl_sync(FULL_MASK, sw, bd.x >> 5, L);
      const uint32_t wb = __shfl_sync(FULL_MASK, sw, bd.y >> 5, L);
      const uint32_t sa = (wa >> (bd.x & 31)) & 1u, sb = (wb >> (bd.y & 31)) & 1u;
      if (b0 + gl < n_bonds) d += sa == sb ? 1.f : -1.f;
    }
    d = J * group_allsum<L>(d);
    float off = 0.f;
    for (int i = 0; i < N; i += 2) {  // two independent sites per iteration
      const int i1 = min(i + 1, N - 1);
      const uint32_t word0 = __shfl_sync(FULL_MASK, sw, i >> 5, L);
      const uint32_t word1 = __shfl_sync(FULL_MASK, sw, i1 >> 5, L);
      const bool up0 = (word0 >> (i & 31)) & 1u, up1 = (word1 >> (i1 & 31)) & 1u;
      float2 rv0[LY::H], g0[LY::H], rv1[LY::H], g1[LY::H];
      LY::template load<false>(R + (size_t)i * M_pad, gl, rv0, 1.f);
      LY::template load<false>(R + (size_t)i1 * M_pad, gl, rv1, 1.f);
      flip_factors<LY::H>(up0, lam, mu, rv0, g0);
      flip_factors<LY::H>(up1, lam, mu, rv1, g1);
      const float tot0 = sum_log2<L, LY::H>(g0);
      const float tot1 = sum_log2<L, LY::H>(g1);
      const float2 ak0 = saK[i], ak1 = saK[i1];
      off += expf(2.f * (ak0.y - (up0 ? ak0.x : -ak0.x)) + tot0 * LN2F);
      if (i + 1 < N) off += expf(2.f * (ak1.y - (up1 ? ak1.x : -ak1.x)) + tot1 * LN2F);
    }
    if (base + grp < n && gl == 0) eloc[x] = d + h * off;
  }
}

// ------------------------------------------------------------------------------------
// O_k rows (App. I, Eq. forces; closed form for the RBM): O_a = s, O_b = tanh theta,
// O_W[j, i] = tanh(theta_j) s_i, with the FP32 master parameters.  One block per row.
__global__ void rbm_grad_rows_kernel(const uint32_t *__restrict__ cfg, int64_t n, const float *__restrict__ Wm,
                                     const float *__restrict__ bm, int N, int W, int M, int64_t P, float *O) {
  extern __shared__ float sh[];
  float *ss = sh;       // [N] spins as +-1
  float *st = sh + N;   // [M] tanh(theta)
  for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) ss[i] = ((cfg[x * W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      float th = bm[j];
      for (int i = 0; i < N; ++i) th = fmaf(ss[i], Wm[(int64_t)i * M + j], th);
      st[j] = tanhf(th);
    }
    __syncthreads();
    float *row = O + x * P;
    for (int64_t q = threadIdx.x; q < P; q += blockDim.x) {
      float v;
      if (q < N) v = ss[q];
      else if (q < N + M) v = st[q - N];
      else {
        const int64_t r = q - N - M;
        v = st[r / N] * ss[r % N];
      }
      row[q] = v;
    }
    __syncthreads();
  }
}

// Force partials (App. I, Eq. forces).  Block (jt, chunk) owns hidden units
// [32 jt, 32 jt + 32) and one chunk of rows.  Per batch of 64 rows it recomputes
// theta = W s + b for its units, forms t_j e(x) = tanh(theta_j) (eloc(x) - E) and
// accumulates sum_x t_j e(x) s_i (W entries), sum_x t_j e(x) (b entries) and, for
// jt == 0, sum_x s_i e(x) (a entries): FP32 inside a batch, FP64 across batches.
// The FP64 partial sums go to ws[chunk][P]; force_reduce_kernel adds the chunks.
// Thread (warp jg, lane il) owns units 4 jg .. 4 jg + 3 and sites il + 32 k.
constexpr int FT_J = 32;       // hidden units per block
constexpr int FT_THREADS = 256;
constexpr int FT_BATCH = 64;   // rows per FP32 batch
constexpr int FT_MAXI = 8;     // sites per lane: N <= 256

__global__ void __launch_bounds__(FT_THREADS) rbm_force_partial_kernel(
    const uint32_t *__restrict__ cfg, int64_t n, const float *__restrict__ eloc, const double *__restrict__ stats,
    const float *__restrict__ Wm, const float *__restrict__ bm, int N, int W, int M, int64_t P, int n_chunks,
    double *ws) {
  extern __shared__ __align__(16) float sh[];
  float *sW = sh;                     // [N][FT_J] master weights of this tile
  float *ss = sW + N * FT_J;          // [FT_BATCH][N] spins, row-major
  float *ssT = ss + FT_BATCH * N;     // [N][FT_BATCH] spins, site-major
  float *st = ssT + N * FT_BATCH;     // [FT_BATCH][FT_J] tanh(theta) * e(x)
  float *se = st + FT_BATCH * FT_J;   // [FT_BATCH] e(x)
  const int jt = blockIdx.x, chunk = blockIdx.y;
  const int j0 = jt * FT_J;
  const int nj = min(FT_J, M - j0);
  const int jg = threadIdx.x >> 5, il = threadIdx.x & 31;
  for (int q = threadIdx.x; q < N * FT_J; q += FT_THREADS) {
    const int i = q / FT_J, jj = q % FT_J;
    sW[q] = jj < nj ? Wm[(int64_t)i * M + j0 + jj] : 0.f;
  }
  float bj[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) bj[k] = (4 * jg + k < nj) ? bm[j0 + 4 * jg + k] : 0.f;
  const double E = stats[0];
  const int64_t rows_per_chunk = (n + n_chunks - 1) / n_chunks;
  const int64_t r0 = (int64_t)chunk * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  double accW[FT_MAXI][4];
#pragma unroll
  for (int k = 0; k < FT_MAXI; ++k)
#pragma unroll
    for (int m = 0; m < 4; ++m) accW[k][m] = 0.0;
  double accB = 0.0, accA = 0.0;
  __syncthreads();
  for (int64_t xb = r0; xb < r1; xb += FT_BATCH) {
    const int nb = (int)(r1 - xb < FT_BATCH ? r1 - xb : FT_BATCH);
    for (int q = threadIdx.x; q < FT_BATCH * N; q += FT_THREADS) {
      const int r = q / N, i = q % N;
      float v = 0.f;
      if (r < nb) v = ((cfg[(xb + r) * W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
      ss[q] = v;
      ssT[i * FT_BATCH + r] = v;
    }
    for (int r = threadIdx.x; r < FT_BATCH; r += FT_THREADS)
      se[r] = r < nb ? (float)((double)eloc[xb + r] - E) : 0.f;
    __syncthreads();
    {  // theta for rows il, il + 32 and units 4 jg .. 4 jg + 3
      float th0[4], th1[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) th0[k] = th1[k] = bj[k];
      for (int i = 0; i < N; ++i) {
        const float4 w4 = *reinterpret_cast<const float4 *>(sW + i * FT_J + 4 * jg);
        const float s0 = ssT[i * FT_BATCH + il], s1 = ssT[i * FT_BATCH + il + 32];
        th0[0] = fmaf(s0, w4.x, th0[0]); th0[1] = fmaf(s0, w4.y, th0[1]);
        th0[2] = fmaf(s0, w4.z, th0[2]); th0[3] = fmaf(s0, w4.w, th0[3]);
        th1[0] = fmaf(s1, w4.x, th1[0]); th1[1] = fmaf(s1, w4.y, th1[1]);
        th1[2] = fmaf(s1, w4.z, th1[2]); th1[3] = fmaf(s1, w4.w, th1[3]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = 4 * jg + k < nj;
        st[il * FT_J + 4 * jg + k] = ok ? tanhf(th0[k]) * se[il] : 0.f;
        st[(il + 32) * FT_J + 4 * jg + k] = ok ? tanhf(th1[k]) * se[il + 32] : 0.f;
      }
    }
    __syncthreads();
    float acc[FT_MAXI][4];
#pragma unroll
    for (int k = 0; k < FT_MAXI; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[k][m] = 0.f;
    for (int r = 0; r < nb; ++r) {
      const float4 t4 = *reinterpret_cast<const float4 *>(st + r * FT_J + 4 * jg);
#pragma unroll
      for (int k = 0; k < FT_MAXI; ++k) {
        const int i = il + 32 * k;
        if (i < N) {
          const float sv = ss[r * N + i];
          acc[k][0] = fmaf(t4.x, sv, acc[k][0]); acc[k][1] = fmaf(t4.y, sv, acc[k][1]);
          acc[k][2] = fmaf(t4.z, sv, acc[k][2]); acc[k][3] = fmaf(t4.w, sv, acc[k][3]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < FT_MAXI; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) accW[k][m] += acc[k][m];
    if (il < 4) {
      float a = 0.f;
      for (int r = 0; r < nb; ++r) a += st[r * FT_J + 4 * jg + il];
      accB += a;
    }
    if (jt == 0 && threadIdx.x < N) {
      float a = 0.f;
      for (int r = 0; r < nb; ++r) a = fmaf(ss[r * N + threadIdx.x], se[r], a);
      accA += a;
    }
    __syncthreads();
  }
  double *out = ws + (int64_t)chunk * P;
#pragma unroll
  for (int k = 0; k < FT_MAXI; ++k) {
    const int i = il + 32 * k;
    if (i < N) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int jj = 4 * jg + m;
        if (jj < nj) out[N + M + (int64_t)(j0 + jj) * N + i] = accW[k][m];
      }
    }
  }
  if (il < 4 && 4 * jg + il < nj) out[N + j0 + 4 * jg + il] = accB;
  if (jt == 0 && threadIdx.x < N) out[threadIdx.x] = accA;
}

__global__ void force_reduce_kernel(const double *ws, int n_chunks, int64_t P, int64_t n, double *force) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += ws[(int64_t)c * P + k];
    force[k] = s / (double)n;
  }
}

// ------------------------------------------------------------------------------------
// dispatch over (L, E): L = 32 for every instantiated width; L = 16 and L = 8 variants
// (two or four chains per warp) for the widths the tuner may pick.
template <template <int, int> class F, typename... A>
cudaError_t dispatch_le(int L, int E, A... args) {
#define NQS_CASE(LL, EE) \
  if (L == LL && E == EE) return F<LL, EE>::run(args...);
  NQS_CASE(8, 4) NQS_CASE(16, 2) NQS_CASE(16, 4) NQS_CASE(16, 8) NQS_CASE(16, 16) NQS_CASE(16, 26)
  NQS_CASE(16, 28) NQS_CASE(16, 32)
  NQS_CASE(32, 1) NQS_CASE(32, 2) NQS_CASE(32, 3) NQS_CASE(32, 4) NQS_CASE(32, 5) NQS_CASE(32, 6)
  NQS_CASE(32, 7) NQS_CASE(32, 8) NQS_CASE(32, 9) NQS_CASE(32, 10) NQS_CASE(32, 11) NQS_CASE(32, 12)
  NQS_CASE(32, 13) NQS_CASE(32, 14) NQS_CASE(32, 16) NQS_CASE(32, 18) NQS_CASE(32, 20) NQS_CASE(32, 24)
  NQS_CASE(32, 28) NQS_CASE(32, 32)
#undef NQS_CASE
  return cudaErrorInvalidConfiguration;
}
template <template <int, int> class F, typename... A>
cudaError_t dispatch_l32(int E, A... args) {
#define NQS_CASE(EE) \
  if (E == EE) return F<32, EE>::run(args...);
  NQS_CASE(1) NQS_CASE(2) NQS_CASE(3) NQS_CASE(4) NQS_CASE(5) NQS_CASE(6) NQS_CASE(7) NQS_CASE(8) NQS_CASE(9)
  NQS_CASE(10) NQS_CASE(11) NQS_CASE(12) NQS_CASE(13) NQS_CASE(14) NQS_CASE(16) NQS_CASE(18) NQS_CASE(20)
  NQS_CASE(24) NQS_CASE(28) NQS_CASE(32)
#undef NQS_CASE
  return cudaErrorInvalidConfiguration;
}

bool e_instantiated(int E32) {
  switch (E32) {
    case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 9: case 10: case 11: case 12:
    case 13: case 14: case 16: case 18: case 20: case 24: case 28: case 32:
      return true;
    default:
      return false;
  }
}

bool l16_instantiated(int E32) { return E32 == 1 || E32 == 2 || E32 == 4 || E32 == 8 || E32 == 13 || E32 == 14 || E32 == 16; }

// Lanes per chain of the sweep and local-energy kernels.
int pick_lanes(const nqs_ctx *c) {
  const int E32 = c->M_pad / 32;
  if (c->chains_per_warp == 4 && E32 == 1 && c->W <= 8) return 8;
  if (c->chains_per_warp == 2 && l16_instantiated(E32) && c->W <= 16) return 16;
  if (c->chains_per_warp == 0 && E32 == 1 && c->W <= 8) return 8;
  return 32;
}

template <int L, int E>
struct SweepRun {
  static cudaError_t run(const nqs_ctx *c, SweepParams p, cudaStream_t s) {
    const size_t table = (size_t)c->N * c->M_pad * 4;
    const size_t extra = (size_t)c->N * sizeof(float2) + 16;
    const bool smem = table + extra + 256 <= (size_t)c->smem_optin;  // + static mbarrier
    auto kern = smem ? rbm_sweep_f32_kernel<L, E, true> : rbm_sweep_f32_kernel<L, E, false>;
    const size_t shm = (smem ? table : 0) + extra;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int regs = std::max(fa.numRegs, 16);
    const int regs_alloc = (regs + 7) / 8 * 8;
    int warps = 65536 / (regs_alloc * 32);
    warps = std::max(1, std::min(fa.maxThreadsPerBlock / 32, warps));
    constexpr int G = 32 / L;
    const int64_t warps_needed = (p.C + G - 1) / G;
    const int blocks_cap = c->num_sms;  // one CTA per SM shares one table copy
    int64_t blocks = std::min<int64_t>(blocks_cap, (warps_needed + warps - 1) / warps);
    if (blocks < c->num_sms) {  // spread small jobs over more SMs with fewer warps each
      blocks = std::min<int64_t>(c->num_sms, warps_needed);
      warps = (int)std::max<int64_t>(1, (warps_needed + blocks - 1) / blocks);
    } else {  // equal rounds: the fewest warps per CTA that keep the round count
      const int64_t rounds = (warps_needed + blocks * warps - 1) / (blocks * warps);
      warps = (int)((warps_needed + blocks * rounds - 1) / (blocks * rounds));
    }
    kern<<<(unsigned)blocks, warps * 32, shm, s>>>(p);
    return cudaGetLastError();
  }
};

template <int L, int E>
struct LogpsiRun {
  static cudaError_t run(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
    constexpr int G = 32 / L;
    const int64_t warps = (n + G - 1) / G;
    const int64_t blocks = std::min<int64_t>((warps + 7) / 8, (int64_t)c->num_sms * 16);
    rbm_logpsi_kernel<L, E><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
        cfg, n, c->d_Wt, c->d_b, c->d_aK, c->N, c->W, c->M_pad, out);
    return cudaGetLastError();
  }
};

template <int L, int E>
struct ElocRun {
  static cudaError_t run(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s) {
    const size_t table = (size_t)c->N * c->M_pad * 4;
    const size_t extra = (size_t)c->N * sizeof(float2) + 16;
    const bool smem = table + extra + 256 <= (size_t)c->smem_optin;  // + static mbarrier
    auto kern = smem ? rbm_tfim_eloc_kernel<L, E, true> : rbm_tfim_eloc_kernel<L, E, false>;
    const size_t shm = (smem ? table : 0) + extra;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int regs_alloc = (std::max(fa.numRegs, 16) + 7) / 8 * 8;
    int warps = std::max(1, std::min(fa.maxThreadsPerBlock / 32, 65536 / (regs_alloc * 32)));
    constexpr int G = 32 / L;
    const int64_t warps_needed = (n + G - 1) / G;
    int64_t blocks = std::min<int64_t>(c->num_sms, (warps_needed + warps - 1) / warps);
    if (blocks < c->num_sms) {
      blocks = std::min<int64_t>(c->num_sms, warps_needed);
      warps = (int)std::max<int64_t>(1, (warps_needed + blocks - 1) / blocks);
    }
    kern<<<(unsigned)blocks, warps * 32, shm, s>>>(cfg, n, c->d_R ? (const float *)c->d_R : nullptr, c->d_aK,
                                                   c->d_Wt, c->d_b, c->d_bonds, c->n_bonds, (float)c->J1,
                                                   (float)c->h, c->N, c->W, c->M_pad, eloc, c->d_status);
    return cudaGetLastError();
  }
};

int force_chunks(const nqs_ctx *c, int64_t n) {
  const int jt = (c->M + FT_J - 1) / FT_J;
  int64_t want = (2 * (int64_t)c->num_sms + jt - 1) / jt;
  want = std::min<int64_t>(want, (n + FT_BATCH - 1) / FT_BATCH);
  return (int)std::max<int64_t>(1, want);
}

}  // namespace

// ====================================================================================
bool rbm_supported(const nqs_ctx *c, std::string *why) {
  if (c->ham_kind != NQS_TFIM) {
    *why = "the RBM path implements the TFIM Hamiltonian (single-flip moves)";
    return false;
  }
  if (c->dtype != NQS_F32) {
    *why = "the RBM sampler is built for F32 sampling copies";
    return false;
  }
  if (c->N > 256) {
    *why = "RBM path supports N <= 256";
    return false;
  }
  if (!e_instantiated(c->M_pad / 32)) {
    *why = "hidden-layer width not instantiated";
    return false;
  }
  return true;
}

cudaError_t rbm_prepare(nqs_ctx *c, const double *params, cudaStream_t s) {
  const int64_t total = (int64_t)c->N * c->M_pad;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 8);
  rbm_prepare_kernel<float><<<blocks, 256, 0, s>>>(params, c->N, c->M, c->M_pad, c->d_a, c->d_b, c->d_Wt,
                                                   (float *)c->d_R, c->d_Wm, c->d_bm, c->d_status, 20.0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rbm_colsum_kernel<<<(c->N * 32 + 255) / 256, 256, 0, s>>>(c->d_Wt, c->d_a, c->N, c->M_pad, c->d_aK);
  return cudaGetLastError();
}

cudaError_t init_chains(const nqs_ctx *c, uint32_t *state, int64_t n, uint64_t seed, cudaStream_t s) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, (int64_t)c->num_sms * 16));
  if (c->ham_kind == NQS_HEISENBERG)
    init_balanced_kernel<<<blocks, 128, 0, s>>>(state, n, c->N, c->W, k0, k1);
  else
    init_random_kernel<<<blocks, 128, 0, s>>>(state, n, c->N, c->W, k0, k1);
  return cudaGetLastError();
}

cudaError_t rbm_sweep(const nqs_ctx *c, uint32_t *state, int64_t n_chains, int n_sweeps, int burn_in,
                      uint64_t seed, uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc,
                      uint32_t *acc_bits, float *delta, cudaStream_t s) {
  SweepParams p;
  p.R = (const float *)c->d_R;
  p.aK = c->d_aK;
  p.Wt = c->d_Wt;
  p.b = c->d_b;
  p.state = state;
  p.samples = samples;
  p.logpsi = logpsi;
  p.n_acc = n_acc;
  p.acc_bits = acc_bits;
  p.delta = delta;
  p.status = c->d_status;
  p.C = n_chains;
  p.N = c->N;
  p.W = c->W;
  p.M_pad = c->M_pad;
  p.n_sweeps = n_sweeps;
  p.burn_in = burn_in;
  p.refresh = c->refresh;
  p.sweep_offset = sweep_offset;
  p.k0 = (uint32_t)seed;
  p.k1 = (uint32_t)(seed >> 32);
  const int L = pick_lanes(c);
  return dispatch_le<SweepRun>(L, c->M_pad / L, c, p, s);
}

cudaError_t rbm_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  return dispatch_l32<LogpsiRun>(c->M_pad / 32, c, cfg, n, out, s);
}

cudaError_t rbm_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s) {
  const int L = pick_lanes(c);
  return dispatch_le<ElocRun>(L, c->M_pad / L, c, cfg, n, eloc, s);
}

int rbm_force_chunks(const nqs_ctx *c, int64_t n) { return force_chunks(c, n); }

cudaError_t rbm_force_into(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                           double *force, double *scratch, int chunks, cudaStream_t s) {
  const int jt = (c->M + FT_J - 1) / FT_J;
  const size_t shm = (size_t)(c->N * FT_J + 2 * FT_BATCH * c->N + FT_BATCH * FT_J + FT_BATCH) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(rbm_force_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm);
  if (e != cudaSuccess) return e;
  rbm_force_partial_kernel<<<dim3(jt, chunks), FT_THREADS, shm, s>>>(cfg, n, eloc, stats, c->d_Wm, c->d_bm, c->N,
                                                                     c->W, c->M, c->P, chunks, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int rb = (int)std::min<int64_t>((c->P + 255) / 256, (int64_t)c->num_sms * 8);
  force_reduce_kernel<<<rb, 256, 0, s>>>(scratch, chunks, c->P, n, force);
  return cudaGetLastError();
}

size_t rbm_grad_workspace(const nqs_ctx *c, int64_t n) {
  const int chunks = rbm_force_tc_supported(c) ? rbm_force_tc_chunks(c, n) : force_chunks(c, n);
  return (size_t)chunks * (size_t)c->P * sizeof(double);
}

cudaError_t rbm_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                            const double *stats, double *force, void *ws, cudaStream_t s) {
  if (O) {
    const size_t shm = (size_t)(c->N + c->M) * sizeof(float);
    const int64_t blocks = std::min<int64_t>(n, (int64_t)c->num_sms * 8);
    rbm_grad_rows_kernel<<<(unsigned)blocks, 256, shm, s>>>(cfg, n, c->d_Wm, c->d_bm, c->N, c->W, c->M, c->P, O);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (force && rbm_force_tc_supported(c)) {  // tensor-core path (N <= 127)
    const int chunks = rbm_force_tc_chunks(c, n);
    cudaError_t e = rbm_force_tc(c, cfg, n, eloc, stats, (double *)ws, chunks, s);
    if (e != cudaSuccess) return e;
    const int rb = (int)std::min<int64_t>((c->P + 255) / 256, (int64_t)c->num_sms * 8);
    force_reduce_kernel<<<rb, 256, 0, s>>>((const double *)ws, chunks, c->P, n, force);
    return cudaGetLastError();
  }
  if (force) {
    const int chunks = force_chunks(c, n);
    const int jt = (c->M + FT_J - 1) / FT_J;
    const size_t shm = (size_t)(c->N * FT_J + 2 * FT_BATCH * c->N + FT_BATCH * FT_J + FT_BATCH) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(rbm_force_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shm);
    if (e != cudaSuccess) return e;
    rbm_force_partial_kernel<<<dim3(jt, chunks), FT_THREADS, shm, s>>>(cfg, n, eloc, stats, c->d_Wm, c->d_bm, c->N,
                                                                       c->W, c->M, c->P, chunks, (double *)ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rb = (int)std::min<int64_t>((c->P + 255) / 256, (int64_t)c->num_sms * 8);
    force_reduce_kernel<<<rb, 256, 0, s>>>((const double *)ws, chunks, c->P, n, force);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace nqs
