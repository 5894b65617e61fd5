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
#include "rbm_core.cuh"

namespace nqs {
namespace {
using namespace rbmk;
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

// Bounds of the sampling copy for the sweep's cache normalisation interval:
// out[0] = max |W_ji|, out[1] = max_j (sum_i |W_ji| + |b_j|) >= max |theta_j|.  Thread per
// hidden unit; non-negative floats are ordered like their bit patterns (atomicMax on ints).
__global__ void rbm_bounds_kernel(const float *Wt, const float *b, int N, int M_pad, float *out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M_pad; j += gridDim.x * blockDim.x) {
    float s = fabsf(b[j]), m = 0.f;
    for (int i = 0; i < N; ++i) {
      const float w = fabsf(Wt[(int64_t)i * M_pad + j]);
      s += w;
      m = fmaxf(m, w);
    }
    atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
    atomicMax(reinterpret_cast<int *>(out) + 1, __float_as_int(s));
  }
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

// Adds the chunks' partial sums in a fixed order and divides by n, or by *ndiv when given
// (the total sample count of a multi-rank step, held in stats[4]).
__global__ void force_reduce_kernel(const double *ws, int n_chunks, int64_t P, int64_t n, const double *ndiv,
                                    double *force) {
  const double d = ndiv ? *ndiv : (double)n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += ws[(int64_t)c * P + k];
    force[k] = s / d;
  }
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

// Lanes per chain of the FP32 sweep and local-energy kernels (16-bit copies use 32).
int pick_lanes(const nqs_ctx *c) {
  if (c->dtype != NQS_F32) return 32;
  const int E32 = c->M_pad / 32;
  if (c->chains_per_warp == 4 && E32 == 1 && c->W <= 8) return 8;
  if (c->chains_per_warp == 2 && l16_instantiated(E32) && c->W <= 16) return 16;
  if (c->chains_per_warp == 0 && E32 == 1 && c->W <= 8) return 8;
  return 32;
}

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
  if (c->dtype == NQS_FP8E4M3) {
    *why = "the RBM sampler is built for F32, BF16 and F16 sampling copies";
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
  // sampling copy in its dtype
  if (c->dtype == NQS_F16)
    rbm_prepare_kernel<__half><<<blocks, 256, 0, s>>>(params, c->N, c->M, c->M_pad, c->d_a, c->d_b, c->d_Wt,
                                                      (__half *)c->d_R, c->d_Wm, c->d_bm, c->d_status, 2.5);
  else if (c->dtype == NQS_BF16)
    rbm_prepare_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(params, c->N, c->M, c->M_pad, c->d_a, c->d_b, c->d_Wt,
                                                             (__nv_bfloat16 *)c->d_R, c->d_Wm, c->d_bm, c->d_status,
                                                             20.0);
  else
    rbm_prepare_kernel<float><<<blocks, 256, 0, s>>>(params, c->N, c->M, c->M_pad, c->d_a, c->d_b, c->d_Wt,
                                                     (float *)c->d_R, c->d_Wm, c->d_bm, c->d_status, 20.0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rbm_colsum_kernel<<<(c->N * 32 + 255) / 256, 256, 0, s>>>(c->d_Wt, c->d_a, c->N, c->M_pad, c->d_aK);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_bounds, 0, 2 * sizeof(float), s)) != cudaSuccess) return e;
  rbm_bounds_kernel<<<(c->M_pad + 127) / 128, 128, 0, s>>>(c->d_Wt, c->d_b, c->N, c->M_pad, c->d_bounds);
  if ((e = cudaGetLastError()) != cudaSuccess || c->dtype == NQS_F32) return e;
  // FP32 copy for the local energy of a 16-bit context
  rbm_prepare_kernel<float><<<blocks, 256, 0, s>>>(params, c->N, c->M, c->M_pad, c->d_a32, c->d_b32, c->d_Wt32,
                                                   c->d_R32, c->d_Wm, c->d_bm, c->d_status, 20.0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  rbm_colsum_kernel<<<(c->N * 32 + 255) / 256, 256, 0, s>>>(c->d_Wt32, c->d_a32, c->N, c->M_pad, c->d_aK32);
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
  p.R = c->d_R;
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
  p.renorm = c->renorm;
  p.noise_sigma = (float)c->noise_sigma;
  p.noise_k0 = (uint32_t)c->noise_key;
  p.noise_k1 = (uint32_t)(c->noise_key >> 32);
  if (c->noise_sigma > 0.0) return dispatch_l32<Runners<float>::NoisySweep>(c->M_pad / 32, c, p, s);  // F32 only
  if (c->dtype == NQS_F16) return rbm_sweep_f16(c, p, s);
  if (c->dtype == NQS_BF16) return rbm_sweep_bf16(c, p, s);
  const int L = pick_lanes(c);
  return dispatch_le<Runners<float>::Sweep>(L, c->M_pad / L, c, p, s);
}

cudaError_t rbm_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  return dispatch_l32<LogpsiRun>(c->M_pad / 32, c, cfg, n, out, s);
}

static ElocParams eloc_params(const nqs_ctx *c, const uint32_t *cfg, const int32_t *sites, int64_t n, float *out) {
  ElocParams p;
  p.cfg = cfg;
  p.sites = sites;
  p.R = c->d_R;
  p.aK = c->d_aK;
  p.Wt = c->d_Wt;
  p.b = c->d_b;
  p.bonds = c->d_bonds;
  p.out = out;
  p.status = c->d_status;
  p.n = n;
  p.n_bonds = c->n_bonds;
  p.N = c->N;
  p.W = c->W;
  p.M_pad = c->M_pad;
  p.J = (float)c->J1;
  p.h = (float)c->h;
  p.n_chains = 0;
  p.refresh = c->refresh;
  return p;
}

// Local energy with the FP32 copy of the master (Sec. 4.2: a 16-bit copy is used only
// for sampling).
cudaError_t rbm_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s) {
  ElocParams p = eloc_params(c, cfg, nullptr, n, eloc);
  p.R = c->d_R32;
  p.aK = c->d_aK32;
  p.Wt = c->d_Wt32;
  p.b = c->d_b32;
  const int E32 = c->M_pad / 32;
  const int L = (E32 == 1 && c->W <= 8) ? 8 : 32;
  return dispatch_le<Runners<float>::Eloc>(L, c->M_pad / L, c, p, s);
}

// Chain-ordered local energy of sweep-major samples (row k * n_chains + c), FP32 copy.
cudaError_t rbm_local_energy_chains(const nqs_ctx *c, const uint32_t *cfg, int64_t n_chains, int64_t per_chain,
                                    float *eloc, cudaStream_t s) {
  // one group per chain walks its samples in order: with fewer than 16 chains per SM that
  // leaves the GPU mostly idle, and the per-sample kernel (same values to FP32 rounding) is used
  if (n_chains < (int64_t)c->num_sms * 16) return rbm_local_energy(c, cfg, n_chains * per_chain, eloc, s);
  ElocParams p = eloc_params(c, cfg, nullptr, n_chains * per_chain, eloc);
  p.R = c->d_R32;
  p.aK = c->d_aK32;
  p.Wt = c->d_Wt32;
  p.b = c->d_b32;
  p.n_chains = n_chains;
  const int E32 = c->M_pad / 32;
  const int L = (E32 == 1 && c->W <= 8) ? 8 : 32;
  return dispatch_le<Runners<float>::ElocChains>(L, c->M_pad / L, c, p, s);
}

cudaError_t rbm_flip_delta(const nqs_ctx *c, const uint32_t *cfg, const int32_t *sites, int64_t n, float *out,
                           cudaStream_t s) {
  const ElocParams p = eloc_params(c, cfg, sites, n, out);
  if (c->dtype == NQS_F16) return rbm_eloc_f16(c, p, s);
  if (c->dtype == NQS_BF16) return rbm_eloc_bf16(c, p, s);
  return dispatch_l32<Runners<float>::Eloc>(c->M_pad / 32, c, p, s);
}

// Accepted flips between normalisations of the sweep's cache.  Between normalisations a pair
// (lam, mu) drifts by at most e^{4 max|W|} per accepted flip and its smaller entry starts at
// no less than e^{-2 max|theta|} / 2; K is the largest of 8, 4, 2 with a drift
// D = 4 max|W| K that keeps both in range: D <= 8 for an F16 copy (its larger entry, >= 1/2,
// stays above the F16 normal range's bottom), D <= 40 and 2 max|theta| + D <= 80 otherwise
// (FP32 normal range).  K = 1 normalises after every accepted flip.
int rbm_renorm_interval(const nqs_ctx *c, float max_w, float max_theta) {
  for (int K = 8; K > 1; K /= 2) {
    const double D = 4.0 * max_w * K;
    const bool ok = c->dtype == NQS_F16 ? D <= 8.0 && 2.0 * max_theta + D <= 80.0 : D <= 40.0 && 2.0 * max_theta + D <= 80.0;
    if (ok) return K;
  }
  return 1;
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
  force_reduce_kernel<<<rb, 256, 0, s>>>(scratch, chunks, c->P, n, nullptr, force);
  return cudaGetLastError();
}

size_t rbm_grad_workspace(const nqs_ctx *c, int64_t n) {
  const int chunks = rbm_force_tc_supported(c) ? rbm_force_tc_chunks(c, n) : force_chunks(c, n);
  return (size_t)chunks * (size_t)c->P * sizeof(double);
}

cudaError_t rbm_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                            const double *stats, double *force, void *ws, cudaStream_t s, bool share) {
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
    force_reduce_kernel<<<rb, 256, 0, s>>>((const double *)ws, chunks, c->P, n, share ? stats + 4 : nullptr, force);
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
    force_reduce_kernel<<<rb, 256, 0, s>>>((const double *)ws, chunks, c->P, n, share ? stats + 4 : nullptr, force);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace nqs
