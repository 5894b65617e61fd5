// Complex-parameter RBM (App. G with a in C^N, b in C^M, W in C^{M x N}):
//   log psi(s) = a . s + sum_j log cosh(theta_j),  theta = W s + b.
// Sec. 2: the chains sample |psi|^2, so a single-flip proposal is decided on
//   2 Re(log psi(y) - log psi(x)) = -4 s_i Re a_i + sum_j ln(D_j(y) / D_j(x)),
//   D_j = |cosh theta_j|^2 = sinh^2(Re theta_j) + cos^2(Im theta_j)
// (a sum of squares: no cancellation near the zeros of cosh, where the equal form
// (cosh 2x + cos 2y) / 2 loses its accuracy and can even turn negative in FP32).
// Local energies (App. I, Eq. local_energies) of the TFIM (Sec. 4.1) are complex:
//   eps(x) = J sum_<ij> s_i s_j + h sum_i psi(flip_i x) / psi(x),
//   psi(flip_i x) / psi(x) = exp(-2 s_i a_i) prod_j (cosh 2W_ji - s_i tanh(theta_j) sinh 2W_ji).
// The force (App. I, Eq. forces) conjugates the holomorphic log-derivatives:
//   F_k = E[O_k^* (eps - E[eps])],  O_a = s, O_b = tanh theta, O_W[j][i] = tanh(theta_j) s_i.
//
// Sampler cache.  Each lane of a chain's warp keeps, for its hidden units, the four numbers
// sinh x, cosh x, cos y, sin y of theta = x + iy.  Flipping s_i moves x by -2 s_i Re W_ji and
// y by -2 s_i Im W_ji, so the proposal's D_j follows from the addition formulas and a
// per-(site, unit) table of cosh/sinh(2 Re W) and cos/sin(2 Im W): six FMA-type operations
// per unit, no transcendental.  The cache is rebuilt from theta every `refresh` sweeps.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>

#include "common.cuh"
#include "internal.h"

struct nqs_crbm {
  nqs_ctx base;  // device, SM count, sticky status word and statistics scratch
  int N = 0, W = 0, M = 0, M_pad = 0, KU = 0, Lx = 0, Ly = 1;
  double J = 1.0, h = 0.0;
  int64_t P = 0;
  int refresh = 20;
  bool params_set = false;
  float2 *d_a = nullptr;   // [N] visible bias
  float2 *d_b = nullptr;   // [M_pad] hidden bias (zero beyond M)
  float2 *d_Wt = nullptr;  // [N][M_pad] weights, site-major (W^T)
  float4 *d_st = nullptr;  // [N][M_pad] (cosh 2 Re W, sinh 2 Re W, cos 2 Im W, sin 2 Im W)
  float4 *d_et = nullptr;  // [M_pad][N] (cosh 2W, sinh 2W) as complex pairs, unit-major
  int2 *d_nb = nullptr;    // [N] right and down neighbour (-1: none, a chain)
  double *d_imstats = nullptr;  // [5] statistics of Im eps
  double2 *d_fpart = nullptr;   // [force_chunks][P] per-row-chunk partial forces, added in a fixed order
  int force_chunks = 1;
  std::string err;
};

namespace nqs {
namespace {

constexpr int CR_THREADS = 128;
constexpr int CR_SPW = 4;            // samples per warp of the local-energy kernel
constexpr int CR_FU = 16;            // hidden units per force tile
constexpr int CR_FR = 64;            // rows per force block (phase A covers 32 rows per pass)
constexpr int CR_FTHREADS = 288;     // force kernel: sites 0 .. N (N <= 256) in phase B
constexpr double CR_MAX_RE_THETA = 10.0;  // sum_i |Re W_ji| + |Re b_j| (products of D_j stay finite)
constexpr double CR_MAX_RE_W = 1.0;       // |Re W_ji| (conditioning of the hyperbolic update)

__device__ __forceinline__ float spin_of(uint32_t word, int bit) { return (word >> bit) & 1u ? 1.f : -1.f; }

// tanh(x + iy) = (sinh x cosh x + i sin y cos y) / (sinh^2 x + cos^2 y); the denominator is
// |cosh(x + iy)|^2 as a sum of squares (no cancellation near the zeros of cosh).
__device__ __forceinline__ float2 tanh_c(float x, float y) {
  float sy, cy;
  sincosf(y, &sy, &cy);
  const float shx = sinhf(x), chx = coshf(x);
  const float inv = 1.f / fmaf(shx, shx, cy * cy);
  return make_float2(shx * chx * inv, sy * cy * inv);
}

// ---- parameter preparation -----------------------------------------------------------
__global__ void crbm_prepare_kernel(const double2 *__restrict__ p, int N, int M, int M_pad, float2 *a, float2 *b,
                                    float2 *Wt, float4 *st, float4 *et, int *status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)N * M_pad;
  for (int64_t idx = t0; idx < total; idx += stride) {
    const int i = (int)(idx / M_pad), j = (int)(idx % M_pad);
    const double2 w = j < M ? p[N + M + (int64_t)j * N + i] : make_double2(0.0, 0.0);
    Wt[idx] = make_float2((float)w.x, (float)w.y);
    st[idx] = make_float4((float)cosh(2.0 * w.x), (float)sinh(2.0 * w.x), (float)cos(2.0 * w.y), (float)sin(2.0 * w.y));
    // cosh(x + iy) = cosh x cos y + i sinh x sin y, sinh(x + iy) = sinh x cos y + i cosh x sin y
    const double cx = cosh(2.0 * w.x), sx = sinh(2.0 * w.x), cy = cos(2.0 * w.y), sy = sin(2.0 * w.y);
    et[(int64_t)j * N + i] = make_float4((float)(cx * cy), (float)(sx * sy), (float)(sx * cy), (float)(cx * sy));
  }
  for (int64_t i = t0; i < N; i += stride) a[i] = make_float2((float)p[i].x, (float)p[i].y);
  for (int64_t j = t0; j < M_pad; j += stride) {
    if (j >= M) {
      b[j] = make_float2(0.f, 0.f);
      continue;
    }
    const double2 bj = p[N + j];
    b[j] = make_float2((float)bj.x, (float)bj.y);
    double s = fabs(bj.x), wmax = 0.0;
    for (int i = 0; i < N; ++i) {
      const double wr = fabs(p[N + M + j * (int64_t)N + i].x);
      s += wr;
      wmax = fmax(wmax, wr);
    }
    if (!(s <= CR_MAX_RE_THETA) || !(wmax <= CR_MAX_RE_W)) atomicOr(status, STATUS_RANGE);
  }
}

// ---- sampler ---------------------------------------------------------------------------
struct CSweepArgs {
  uint32_t *state;
  int64_t C;
  int N, W, M_pad, T, B, refresh;
  uint32_t k0, k1, sweep_offset;
  const float2 *a, *b, *Wt;
  const float4 *st;
  uint32_t *samples;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
};

// One warp per chain; lane q < W holds word q of the configuration and of the sweep's
// accept bits; lane l holds hidden units l + 32k (k < KU).
template <int KU>
__global__ void __launch_bounds__(CR_THREADS) crbm_sweep_kernel(const CSweepArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (blockIdx.x * (int64_t)CR_THREADS + threadIdx.x) >> 5;
  if (c >= a.C) return;  // warp-uniform
  uint32_t word = lane < a.W ? a.state[c * a.W + lane] : 0u;
  float shx[KU], chx[KU], cy[KU], sy[KU];
  float Lc = 0.f;  // this lane's sum of log2 D_j of the current configuration
  int64_t nacc = 0;
  for (int t = 0; t < a.T; ++t) {
    if (t % a.refresh == 0) {
      float x[KU], y[KU];
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        const float2 bj = a.b[lane + 32 * k];
        x[k] = bj.x;
        y[k] = bj.y;
      }
      for (int i = 0; i < a.N; ++i) {
        const float s = spin_of(__shfl_sync(FULL_MASK, word, i >> 5), i & 31);
        const float2 *row = a.Wt + (int64_t)i * a.M_pad + lane;
#pragma unroll
        for (int k = 0; k < KU; ++k) {
          const float2 w = __ldg(row + 32 * k);
          x[k] = fmaf(s, w.x, x[k]);
          y[k] = fmaf(s, w.y, y[k]);
        }
      }
      Lc = 0.f;
      float prod = 1.f;
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        shx[k] = sinhf(x[k]);
        chx[k] = coshf(x[k]);
        sincosf(y[k], &sy[k], &cy[k]);
        prod *= fmaf(shx[k], shx[k], cy[k] * cy[k]);
        if ((k & 3) == 3 || k == KU - 1) {
          Lc += lg2_approx(prod);
          prod = 1.f;
        }
      }
    }
    uint32_t bits = 0u;
    // lane l draws the Philox block of proposal pair p/2 + l once per 64 proposals; the
    // proposal's two words are then broadcast from that lane (same counters, same draws)
    uint4 r = make_uint4(0, 0, 0, 0);
    for (int p = 0; p < a.N; ++p) {
      if ((p & 63) == 0)
        r = philox4x32_10(make_uint4((uint32_t)((p >> 1) + lane), a.sweep_offset + t, (uint32_t)c, TAG_SWEEP), a.k0,
                          a.k1);
      const int src = (p & 63) >> 1;
      const uint32_t w0 = __shfl_sync(FULL_MASK, (p & 1) ? r.z : r.x, src);
      const uint32_t w1 = __shfl_sync(FULL_MASK, (p & 1) ? r.w : r.y, src);
      const int i = (int)index_from_word(w0, (uint32_t)a.N);
      const float u = (float)(w1 >> 8) * 0x1p-24f;
      const float sg = spin_of(__shfl_sync(FULL_MASK, word, i >> 5), i & 31);
      const float4 *row = a.st + (int64_t)i * a.M_pad + lane;
      float Ln = 0.f, prod = 1.f;
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        const float4 tb = __ldg(row + 32 * k);
        // sinh(x - b) = sinh x cosh b - cosh x sinh b, cos(y - c) = cos y cos c + sin y sin c
        const float shn = fmaf(shx[k], tb.x, -chx[k] * (sg * tb.y));
        const float cyn = fmaf(cy[k], tb.z, sy[k] * (sg * tb.w));
        prod *= fmaf(shn, shn, cyn * cyn);
        if ((k & 3) == 3 || k == KU - 1) {
          Ln += lg2_approx(prod);
          prod = 1.f;
        }
      }
      // every lane ends with the bitwise-identical sum, so the decision is warp-uniform
      const float dsum = group_allsum<32>(Ln - Lc);
      const float d2 = fmaf(LN2F, dsum, -4.f * sg * a.a[i].x);
      const bool acc = (u == 0.f) || (u < ex2_approx(d2 * LOG2EF));
      if (a.delta && lane == 0) a.delta[((int64_t)c * a.T + t) * a.N + p] = 0.5f * d2;
      if (acc) {
#pragma unroll
        for (int k = 0; k < KU; ++k) {
          const float4 tb = __ldg(row + 32 * k);
          const float sb = sg * tb.y, ss = sg * tb.w;
          const float shn = fmaf(shx[k], tb.x, -chx[k] * sb), chn = fmaf(chx[k], tb.x, -shx[k] * sb);
          const float cyn = fmaf(cy[k], tb.z, sy[k] * ss), syn = fmaf(sy[k], tb.z, -cy[k] * ss);
          shx[k] = shn;
          chx[k] = chn;
          cy[k] = cyn;
          sy[k] = syn;
        }
        Lc = Ln;
        if (lane == (i >> 5)) word ^= 1u << (i & 31);
        if (lane == (p >> 5)) bits |= 1u << (p & 31);
        ++nacc;
      }
    }
    if (lane < a.W) {
      if (a.samples && t >= a.B) a.samples[((int64_t)(t - a.B) * a.C + c) * a.W + lane] = word;
      if (a.acc_bits) a.acc_bits[((int64_t)c * a.T + t) * a.W + lane] = bits;
    }
  }
  if (lane < a.W) a.state[c * a.W + lane] = word;
  if (a.n_acc && lane == 0) a.n_acc[c] = nacc;
}

// ---- log psi ---------------------------------------------------------------------------
struct CRowArgs {
  const uint32_t *cfg;
  int64_t n;
  int N, W, M, M_pad;
  const float2 *a, *b, *Wt;
};

// One warp per configuration: out[2x] = Re log psi, out[2x + 1] = Im log psi (the sum of
// principal arguments; defined modulo 2 pi).
__global__ void __launch_bounds__(CR_THREADS) crbm_logpsi_kernel(const CRowArgs a, float *out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * CR_THREADS) >> 5;
  for (int64_t x = (blockIdx.x * (int64_t)CR_THREADS + threadIdx.x) >> 5; x < a.n; x += nw) {
    const uint32_t word = lane < a.W ? a.cfg[x * a.W + lane] : 0u;
    float re = 0.f, im = 0.f;
    // padded units (W = b = 0) add log cosh 0 = 0; every lane runs every iteration
    for (int j = lane; j < a.M_pad; j += 32) {
      float tx = a.b[j].x, ty = a.b[j].y;
      for (int i = 0; i < a.N; ++i) {
        const float s = spin_of(__shfl_sync(FULL_MASK, word, i >> 5), i & 31);
        const float2 w = a.Wt[(int64_t)i * a.M_pad + j];
        tx = fmaf(s, w.x, tx);
        ty = fmaf(s, w.y, ty);
      }
      float sy, cy;
      sincosf(ty, &sy, &cy);
      const float chx = coshf(tx), shx = sinhf(tx);
      re += 0.5f * logf(fmaxf(chx * chx - sy * sy, 0.f));  // |cosh z|^2 = cosh^2 x - sin^2 y
      im += atan2f(shx * sy, chx * cy);
    }
    for (int q = 0; q < (a.N + 31) / 32; ++q) {
      const uint32_t wq = __shfl_sync(FULL_MASK, word, q);
      const int i = 32 * q + lane;
      if (i < a.N) {
        const float s = spin_of(wq, lane);
        re = fmaf(s, a.a[i].x, re);
        im = fmaf(s, a.a[i].y, im);
      }
    }
    re = group_allsum<32>(re);
    im = group_allsum<32>(im);
    if (lane == 0) {
      out[2 * x] = re;
      out[2 * x + 1] = im;
    }
  }
}

// ---- local energies ----------------------------------------------------------------------
struct CElocArgs {
  CRowArgs r;
  const float4 *et;
  const int2 *nb;
  float J, h;
  float *eloc_re, *eloc_im;
  int64_t n_chains;  // CHAIN: rows k C + c of chain c, k < r.n / n_chains (sweep-major samples)
  int refresh;       // CHAIN: theta rebuilt from scratch every `refresh` samples of a chain
};

// |p| pulled into the log2 accumulator L; a zero product marks the ratio as zero.
__device__ __forceinline__ void crbm_normalise(float2 &p, float &L, bool &dead) {
  const float m = fmaf(p.x, p.x, p.y * p.y);
  if (m > 0.f) {
    L = fmaf(0.5f, lg2_approx(m), L);
    const float inv = rsqrtf(m);
    p.x *= inv;
    p.y *= inv;
  } else {
    dead = true;
    p = make_float2(1.f, 0.f);
  }
}

// One warp per CR_SPW configurations.  Phase 1 (lanes over hidden units): theta and
// tanh theta of every sample into the warp's shared-memory slice.  Phase 2 (lanes over
// sites): the flip ratio of site i as a product over all units, read from the unit-major
// (cosh 2W, sinh 2W) table once for the CR_SPW samples.
// CHAIN: a warp walks one chain's sweep-major samples in order, CR_SPW at a time, and keeps
// theta in registers from one sample to the next: it adds 2 s'_i W_i only for the spins that
// changed since the chain's previous sample (theta rebuilt from scratch every `refresh`
// samples).  Phase 2 is the same.
template <int KU, bool CHAIN>
__global__ void __launch_bounds__(CR_THREADS, 4) crbm_eloc_kernel(const CElocArgs a) {
  extern __shared__ float2 crbm_tanh[];  // [warps][CR_SPW][M_pad]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M_pad = a.r.M_pad, N = a.r.N, W = a.r.W;
  float2 *tw = crbm_tanh + (size_t)warp * CR_SPW * M_pad;
  const int64_t gw = (blockIdx.x * (int64_t)CR_THREADS + threadIdx.x) >> 5;  // global warp
  const int64_t nw = ((int64_t)gridDim.x * CR_THREADS) >> 5;
  // work items: groups of CR_SPW rows (grid-stride), or (CHAIN) the blocks of chain gw in order
  const int64_t K = CHAIN ? a.r.n / a.n_chains : 0;
  const int64_t n_items = CHAIN ? (gw < a.n_chains ? (K + CR_SPW - 1) / CR_SPW : 0) : (a.r.n + CR_SPW - 1) / CR_SPW;
  float cx[CHAIN ? KU : 1], cy[CHAIN ? KU : 1];  // CHAIN: the chain's theta after its previous sample
  uint32_t prev = 0u;                            // CHAIN: the word of that sample held by this lane
  for (int64_t it = CHAIN ? 0 : gw; it < n_items; it += CHAIN ? 1 : nw) {
    uint32_t wr[CR_SPW];
    int64_t xr[CR_SPW];  // output row of sample r (clamped), valid when vr[r]
    bool vr[CR_SPW];
#pragma unroll
    for (int r = 0; r < CR_SPW; ++r) {
      const int64_t q = it * CR_SPW + r;
      if constexpr (CHAIN) {
        vr[r] = q < K;
        xr[r] = std::min<int64_t>(q, K - 1) * a.n_chains + gw;
      } else {
        vr[r] = q < a.r.n;
        xr[r] = std::min<int64_t>(q, a.r.n - 1);
      }
      wr[r] = lane < W ? a.r.cfg[xr[r] * W + lane] : 0u;
    }
    if constexpr (CHAIN) {
#pragma unroll
      for (int r = 0; r < CR_SPW; ++r) {
        const int64_t k = std::min<int64_t>(it * CR_SPW + r, K - 1);
        if (k % a.refresh == 0) {  // from scratch: b + sum_i s_i W_i
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            const float2 bj = a.r.b[lane + 32 * u];
            cx[u] = bj.x;
            cy[u] = bj.y;
          }
          for (int i = 0; i < N; ++i) {
            const float si = spin_of(__shfl_sync(FULL_MASK, wr[r], i >> 5), i & 31);
            const float2 *row = a.r.Wt + (int64_t)i * M_pad + lane;
#pragma unroll
            for (int u = 0; u < KU; ++u) {
              const float2 w = __ldg(row + 32 * u);
              cx[u] = fmaf(si, w.x, cx[u]);
              cy[u] = fmaf(si, w.y, cy[u]);
            }
          }
        } else {  // the spins changed since the previous sample: theta += 2 s'_i W_i
          for (int wi = 0; wi < W; ++wi) {
            uint32_t m = __shfl_sync(FULL_MASK, wr[r] ^ prev, wi);
            const uint32_t now = __shfl_sync(FULL_MASK, wr[r], wi);
            while (m) {  // warp-uniform
              const int bit = __ffs(m) - 1;
              m &= m - 1u;
              const float s2 = ((now >> bit) & 1u) ? 2.f : -2.f;
              const float2 *row = a.r.Wt + (int64_t)(32 * wi + bit) * M_pad + lane;
#pragma unroll
              for (int u = 0; u < KU; ++u) {
                const float2 w = __ldg(row + 32 * u);
                cx[u] = fmaf(s2, w.x, cx[u]);
                cy[u] = fmaf(s2, w.y, cy[u]);
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) tw[r * M_pad + lane + 32 * u] = tanh_c(cx[u], cy[u]);
        prev = wr[r];
      }
    } else {
    // theta of two samples at a time: each weight row is loaded once for both
#pragma unroll
    for (int r = 0; r < CR_SPW; r += 2) {
      float tx0[KU], ty0[KU], tx1[KU], ty1[KU];
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        const float2 bj = a.r.b[lane + 32 * k];
        tx0[k] = tx1[k] = bj.x;
        ty0[k] = ty1[k] = bj.y;
      }
      for (int i = 0; i < N; ++i) {
        const float s0 = spin_of(__shfl_sync(FULL_MASK, wr[r], i >> 5), i & 31);
        const float s1 = spin_of(__shfl_sync(FULL_MASK, wr[r + 1], i >> 5), i & 31);
        const float2 *row = a.r.Wt + (int64_t)i * M_pad + lane;
#pragma unroll
        for (int k = 0; k < KU; ++k) {
          const float2 w = __ldg(row + 32 * k);
          tx0[k] = fmaf(s0, w.x, tx0[k]);
          ty0[k] = fmaf(s0, w.y, ty0[k]);
          tx1[k] = fmaf(s1, w.x, tx1[k]);
          ty1[k] = fmaf(s1, w.y, ty1[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        tw[r * M_pad + lane + 32 * k] = tanh_c(tx0[k], ty0[k]);
        tw[(r + 1) * M_pad + lane + 32 * k] = tanh_c(tx1[k], ty1[k]);
      }
    }
    }
    __syncwarp();
    float er[CR_SPW], ei[CR_SPW];
#pragma unroll
    for (int r = 0; r < CR_SPW; ++r) er[r] = ei[r] = 0.f;
    // full passes of 32 sites (every lane takes one site for all CR_SPW samples); a tail of
    // rem < 32 sites with rem * CR_SPW <= 32 runs below as (site, sample) pairs instead, one
    // pair per lane, so that it does not cost a full pass for a few active lanes
    const int rem = N % 32;
    const bool tail_pairs = rem > 0 && rem * CR_SPW <= 32;
    const int n_full = tail_pairs ? N / 32 : (N + 31) / 32;
    for (int q = 0; q < n_full; ++q) {
      const int i = 32 * q + lane;
      const bool active = i < N;
      const int2 nb = a.nb[active ? i : 0];
      float sg[CR_SPW], zz[CR_SPW];
#pragma unroll
      for (int r = 0; r < CR_SPW; ++r) {
        sg[r] = spin_of(__shfl_sync(FULL_MASK, wr[r], q), lane);
        const float sr = spin_of(__shfl_sync(FULL_MASK, wr[r], nb.x >> 5), nb.x & 31);
        const int d = nb.y >= 0 ? nb.y : 0;
        const float sd = nb.y >= 0 ? spin_of(__shfl_sync(FULL_MASK, wr[r], d >> 5), d & 31) : 0.f;
        zz[r] = sg[r] * (sr + sd);
      }
      if (active) {
        float2 p[CR_SPW];
        float L[CR_SPW];
        bool dead[CR_SPW];
#pragma unroll
        for (int r = 0; r < CR_SPW; ++r) {
          p[r] = make_float2(1.f, 0.f);
          L[r] = 0.f;
          dead[r] = false;
        }
        const float4 *col = a.et + i;
        // (cosh 2W, sinh 2W) of (j, i) for the current chunk of 8 units; the next chunk's
        // loads are issued before the current one is consumed (load latency, not bandwidth,
        // bounds this loop)
        float4 cur[8], nxt[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) cur[jj] = __ldg(col + (int64_t)jj * N);
        for (int j0 = 0; j0 < M_pad; j0 += 8) {
          if (j0 + 8 < M_pad) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) nxt[jj] = __ldg(col + (int64_t)(j0 + 8 + jj) * N);
          } else {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) nxt[jj] = cur[jj];
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = j0 + jj;
            const float4 cs = cur[jj];
#pragma unroll
            for (int r = 0; r < CR_SPW; ++r) {
              const float2 t = tw[r * M_pad + j];
              const float tsx = fmaf(t.x, cs.z, -t.y * cs.w), tsy = fmaf(t.x, cs.w, t.y * cs.z);
              const float rx = fmaf(-sg[r], tsx, cs.x), ry = fmaf(-sg[r], tsy, cs.y);
              const float px = fmaf(p[r].x, rx, -p[r].y * ry), py = fmaf(p[r].x, ry, p[r].y * rx);
              p[r] = make_float2(px, py);
            }
          }
#pragma unroll
          for (int r = 0; r < CR_SPW; ++r) crbm_normalise(p[r], L[r], dead[r]);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) cur[jj] = nxt[jj];
        }
        const float2 ai = a.r.a[i];
#pragma unroll
        for (int r = 0; r < CR_SPW; ++r) {
          er[r] = fmaf(a.J, zz[r], er[r]);
          if (!dead[r]) {
            // exp(-2 s_i a_i) prod_j (...) = 2^(L - 2 s_i Re a_i log2 e) e^{-2 i s_i Im a_i} p
            const float mag = ex2_approx(fmaf(-2.f * sg[r] * ai.x, LOG2EF, L[r]));
            float sn, cn;
            sincosf(-2.f * sg[r] * ai.y, &sn, &cn);
            const float rx = fmaf(p[r].x, cn, -p[r].y * sn), ry = fmaf(p[r].x, sn, p[r].y * cn);
            er[r] = fmaf(a.h * mag, rx, er[r]);
            ei[r] = fmaf(a.h * mag, ry, ei[r]);
          }
        }
      }
    }
    if (tail_pairs) {
      const bool act = lane < rem * CR_SPW;
      const int rr = act ? lane / rem : 0;
      const int i = 32 * (N / 32) + (act ? lane % rem : 0);
      const int2 nb = a.nb[i];
      const int d = nb.y >= 0 ? nb.y : 0;
      // this lane's sample's words of sites i, nb.x, nb.y (the shuffles are warp-wide)
      uint32_t wi = 0u, wx = 0u, wd = 0u;
#pragma unroll
      for (int r = 0; r < CR_SPW; ++r) {
        const uint32_t vi = __shfl_sync(FULL_MASK, wr[r], i >> 5);
        const uint32_t vx = __shfl_sync(FULL_MASK, wr[r], nb.x >> 5);
        const uint32_t vd = __shfl_sync(FULL_MASK, wr[r], d >> 5);
        if (r == rr) {
          wi = vi;
          wx = vx;
          wd = vd;
        }
      }
      if (act) {
        const float sg = spin_of(wi, i & 31);
        const float sr = spin_of(wx, nb.x & 31);
        const float sd = nb.y >= 0 ? spin_of(wd, d & 31) : 0.f;
        float2 pp = make_float2(1.f, 0.f);
        float L = 0.f;
        bool dead = false;
        const float4 *col = a.et + i;
        const float2 *tr = tw + rr * M_pad;
        float4 cur[8], nxt[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) cur[jj] = __ldg(col + (int64_t)jj * N);
        for (int j0 = 0; j0 < M_pad; j0 += 8) {
          if (j0 + 8 < M_pad) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) nxt[jj] = __ldg(col + (int64_t)(j0 + 8 + jj) * N);
          } else {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) nxt[jj] = cur[jj];
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const float4 cs = cur[jj];
            const float2 t = tr[j0 + jj];
            const float tsx = fmaf(t.x, cs.z, -t.y * cs.w), tsy = fmaf(t.x, cs.w, t.y * cs.z);
            const float rx = fmaf(-sg, tsx, cs.x), ry = fmaf(-sg, tsy, cs.y);
            const float px = fmaf(pp.x, rx, -pp.y * ry), py = fmaf(pp.x, ry, pp.y * rx);
            pp = make_float2(px, py);
          }
          crbm_normalise(pp, L, dead);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) cur[jj] = nxt[jj];
        }
        const float2 ai = a.r.a[i];
        float dr = a.J * sg * (sr + sd), di = 0.f;
        if (!dead) {
          const float mag = ex2_approx(fmaf(-2.f * sg * ai.x, LOG2EF, L));
          float sn, cn;
          sincosf(-2.f * sg * ai.y, &sn, &cn);
          const float rx = fmaf(pp.x, cn, -pp.y * sn), ry = fmaf(pp.x, sn, pp.y * cn);
          dr = fmaf(a.h * mag, rx, dr);
          di = a.h * mag * ry;
        }
#pragma unroll
        for (int r = 0; r < CR_SPW; ++r)
          if (r == rr) {
            er[r] += dr;
            ei[r] += di;
          }
      }
    }
#pragma unroll
    for (int r = 0; r < CR_SPW; ++r) {
      const float sre = group_allsum<32>(er[r]), sim = group_allsum<32>(ei[r]);
      if (lane == 0 && vr[r]) {
        a.eloc_re[xr[r]] = sre;
        a.eloc_im[xr[r]] = sim;
      }
    }
    __syncwarp();
  }
}

// ---- O rows ------------------------------------------------------------------------------
// One CTA per row: O[x] = [s | tanh theta | tanh(theta_j) s_i], complex FP32 interleaved.
__global__ void __launch_bounds__(CR_THREADS) crbm_grad_rows_kernel(const CRowArgs a, int64_t P, float2 *O) {
  extern __shared__ float2 crbm_rowt[];  // [M_pad]
  __shared__ uint32_t words[8];
  for (int64_t x = blockIdx.x; x < a.n; x += gridDim.x) {
    if (threadIdx.x < a.W) words[threadIdx.x] = a.cfg[x * a.W + threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.x; j < a.M; j += CR_THREADS) {
      float tx = a.b[j].x, ty = a.b[j].y;
      for (int i = 0; i < a.N; ++i) {
        const float s = spin_of(words[i >> 5], i & 31);
        const float2 w = a.Wt[(int64_t)i * a.M_pad + j];
        tx = fmaf(s, w.x, tx);
        ty = fmaf(s, w.y, ty);
      }
      crbm_rowt[j] = tanh_c(tx, ty);
    }
    __syncthreads();
    float2 *row = O + x * P;
    for (int64_t k = threadIdx.x; k < P; k += CR_THREADS) {
      float2 v;
      if (k < a.N) {
        v = make_float2(spin_of(words[k >> 5], (int)(k & 31)), 0.f);
      } else if (k < a.N + a.M) {
        v = crbm_rowt[k - a.N];
      } else {
        const int64_t q = k - a.N - a.M;
        const int j = (int)(q / a.N), i = (int)(q % a.N);
        const float s = spin_of(words[i >> 5], i & 31);
        const float2 t = crbm_rowt[j];
        v = make_float2(s * t.x, s * t.y);
      }
      row[k] = v;
    }
    __syncthreads();
  }
}

// ---- force -------------------------------------------------------------------------------
// The force as one contraction over rows x of the extended matrices
//   G[x][j] = conj(t_j(x)) e(x) (j < M),  G[x][M] = e(x),     e = eps - E,
//   S[x][i] = s_i(x) (i < N),             S[x][N] = 1,
// Fsum = G^T S: F_W = Fsum[j][i], F_b = Fsum[j][N], F_a = Fsum[M][i].  CTA (row range,
// tile of CR_FU units): phase A builds G for CR_FR rows, phase B accumulates site columns
// in FP32 over the block and in FP64 across blocks, then writes its row chunk's slot of the
// partial forces (every entry of a slot is written by exactly one CTA of that chunk);
// crbm_force_reduce_kernel adds the slots in a fixed order, so the result is deterministic.
struct CForceArgs {
  CRowArgs r;
  const float *eloc_re, *eloc_im;
  const double *stats;
  int64_t rows_per_cta;
  double2 *part;  // [gridDim.x][P]
  int64_t P;
};

// HALVES = 2 (N + 1 <= 144): phase B thread (i, h) takes site i and units h*8 .. h*8 + 7 of
// the tile, so 2 (N + 1) threads share the accumulation; HALVES = 1 otherwise.
template <int HALVES>
__global__ void __launch_bounds__(CR_FTHREADS) crbm_force_kernel(const CForceArgs a) {
  constexpr int UPT = CR_FU / HALVES;  // units per phase-B thread
  __shared__ uint32_t sbits[CR_FR][8];
  __shared__ float2 g[CR_FR][CR_FU];
  const int tid = threadIdx.x;
  const int N = a.r.N, M = a.r.M, W = a.r.W;
  const int j0 = blockIdx.y * CR_FU;
  const int64_t x_begin = blockIdx.x * a.rows_per_cta;
  const int64_t x_end = std::min<int64_t>(a.r.n, x_begin + a.rows_per_cta);
  const float Ere = (float)a.stats[0], Eim = (float)a.stats[5];
  const int i = tid % (N + 1), h = tid / (N + 1);
  const bool worker = h < HALVES;
  double accd[UPT][2];
#pragma unroll
  for (int u = 0; u < UPT; ++u) accd[u][0] = accd[u][1] = 0.0;
  for (int64_t r0 = x_begin; r0 < x_end; r0 += CR_FR) {
    for (int idx = tid; idx < CR_FR * W; idx += CR_FTHREADS) {
      const int rr = idx / W, q = idx % W;
      const int64_t x = r0 + rr;
      sbits[rr][q] = x < x_end ? a.r.cfg[x * W + q] : 0u;
    }
    __syncthreads();
#pragma unroll 1
    for (int rr0 = 0; rr0 < CR_FR; rr0 += 32) {
      if (tid >= 32 * (CR_FU / 2)) break;
      const int rr = rr0 + tid / (CR_FU / 2), uu = 2 * (tid % (CR_FU / 2));
      const int64_t x = r0 + rr;
      const bool valid = x < x_end;
      const float ex = valid ? a.eloc_re[x] - Ere : 0.f, ey = valid ? a.eloc_im[x] - Eim : 0.f;
      const int ja = j0 + uu, jb = ja + 1;
      const int ca = std::min(ja, a.r.M_pad - 1), cb = std::min(jb, a.r.M_pad - 1);
      float tax = a.r.b[ca].x, tay = a.r.b[ca].y, tbx = a.r.b[cb].x, tby = a.r.b[cb].y;
#pragma unroll 4
      for (int ii = 0; ii < N; ++ii) {
        const float sp = spin_of(sbits[rr][ii >> 5], ii & 31);
        const float2 wa = a.r.Wt[(int64_t)ii * a.r.M_pad + ca], wb = a.r.Wt[(int64_t)ii * a.r.M_pad + cb];
        tax = fmaf(sp, wa.x, tax);
        tay = fmaf(sp, wa.y, tay);
        tbx = fmaf(sp, wb.x, tbx);
        tby = fmaf(sp, wb.y, tby);
      }
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int j = v ? jb : ja;
        float2 gv = make_float2(0.f, 0.f);
        if (j < M) {
          const float2 t = v ? tanh_c(tbx, tby) : tanh_c(tax, tay);
          // conj(t) e
          gv = make_float2(fmaf(t.x, ex, t.y * ey), fmaf(t.x, ey, -t.y * ex));
        } else if (j == M) {
          gv = make_float2(ex, ey);
        }
        g[rr][uu + v] = gv;
      }
    }
    __syncthreads();
    if (worker) {
      float acc[UPT][2];
#pragma unroll
      for (int u = 0; u < UPT; ++u) acc[u][0] = acc[u][1] = 0.f;
      for (int rr = 0; rr < CR_FR; ++rr) {
        const float sp = i < N ? spin_of(sbits[rr][i >> 5], i & 31) : 1.f;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          const float2 gv = g[rr][h * UPT + u];
          acc[u][0] = fmaf(sp, gv.x, acc[u][0]);
          acc[u][1] = fmaf(sp, gv.y, acc[u][1]);
        }
      }
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        accd[u][0] += (double)acc[u][0];
        accd[u][1] += (double)acc[u][1];
      }
    }
    __syncthreads();
  }
  if (!worker) return;
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int j = j0 + h * UPT + u;
    int64_t k = -1;
    if (j < M && i < N) k = (int64_t)N + M + (int64_t)j * N + i;
    else if (j < M) k = (int64_t)N + j;
    else if (j == M && i < N) k = i;
    if (k >= 0) a.part[blockIdx.x * a.P + k] = make_double2(accd[u][0], accd[u][1]);
  }
}

__global__ void crbm_force_reduce_kernel(const double2 *part, int chunks, int64_t P, double inv_n, double2 *force) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < chunks; ++q) {
      const double2 v = part[q * P + k];
      s.x += v.x;
      s.y += v.y;
    }
    force[k] = make_double2(s.x * inv_n, s.y * inv_n);
  }
}

// Largest instantiated units-per-lane width >= need.
constexpr int KU_LIST[] = {1, 2, 3, 4, 6, 8, 10, 13, 16};

template <int KU>
cudaError_t launch_sweep(const nqs_crbm *c, const CSweepArgs &a, cudaStream_t s) {
  const int64_t blocks = (a.C * 32 + CR_THREADS - 1) / CR_THREADS;
  crbm_sweep_kernel<KU><<<(unsigned)blocks, CR_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int KU>
cudaError_t launch_eloc(const nqs_crbm *c, const CElocArgs &a, cudaStream_t s) {
  const size_t smem = (size_t)(CR_THREADS / 32) * CR_SPW * c->M_pad * sizeof(float2);
  const bool chain = a.n_chains > 0;
  auto k = chain ? crbm_eloc_kernel<KU, true> : crbm_eloc_kernel<KU, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // a warp per chain (CHAIN), else grid-stride warps over groups of CR_SPW rows
  const int64_t warps = chain ? a.n_chains : (a.r.n + CR_SPW - 1) / CR_SPW;
  const int64_t blocks = std::max<int64_t>(1, chain ? (warps * 32 + CR_THREADS - 1) / CR_THREADS
                                                    : std::min<int64_t>((warps * 32 + CR_THREADS - 1) / CR_THREADS,
                                                                        (int64_t)c->base.num_sms * 8));
  k<<<(unsigned)blocks, CR_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

#define CRBM_DISPATCH(KUV, FN, ...)        \
  switch (KUV) {                           \
    case 1: return FN<1>(__VA_ARGS__);     \
    case 2: return FN<2>(__VA_ARGS__);     \
    case 3: return FN<3>(__VA_ARGS__);     \
    case 4: return FN<4>(__VA_ARGS__);     \
    case 6: return FN<6>(__VA_ARGS__);     \
    case 8: return FN<8>(__VA_ARGS__);     \
    case 10: return FN<10>(__VA_ARGS__);   \
    case 13: return FN<13>(__VA_ARGS__);   \
    default: return FN<16>(__VA_ARGS__);   \
  }

cudaError_t dispatch_sweep(const nqs_crbm *c, const CSweepArgs &a, cudaStream_t s) {
  CRBM_DISPATCH(c->KU, launch_sweep, c, a, s)
}
cudaError_t dispatch_eloc(const nqs_crbm *c, const CElocArgs &a, cudaStream_t s) {
  CRBM_DISPATCH(c->KU, launch_eloc, c, a, s)
}

CRowArgs row_args(const nqs_crbm *c, const uint32_t *cfg, int64_t n) {
  CRowArgs r;
  r.cfg = cfg;
  r.n = n;
  r.N = c->N;
  r.W = c->W;
  r.M = c->M;
  r.M_pad = c->M_pad;
  r.a = c->d_a;
  r.b = c->d_b;
  r.Wt = c->d_Wt;
  return r;
}

void crbm_free(nqs_crbm *c) {
  void *ptrs[] = {c->d_a, c->d_b, c->d_Wt, c->d_st, c->d_et, c->d_nb, c->d_imstats, c->base.d_status,
                  c->base.d_scratch, c->d_fpart};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace
}  // namespace nqs

namespace {

thread_local std::string g_crbm_error;

nqs_status cfail(nqs_crbm *c, nqs_status st, const std::string &msg) {
  if (c) c->err = msg;
  else g_crbm_error = msg;
  return st;
}
nqs_status ccuda(nqs_crbm *c, cudaError_t e, const char *where) {
  return cfail(c, NQS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

const char *nqs_crbm_last_error(const nqs_crbm *c) { return c ? c->err.c_str() : g_crbm_error.c_str(); }
int64_t nqs_crbm_n_params(const nqs_crbm *c) { return c ? c->P : 0; }
int32_t nqs_crbm_words_per_config(const nqs_crbm *c) { return c ? c->W : 0; }

nqs_status nqs_crbm_create(nqs_crbm **out, const nqs_ham_desc *ham, int32_t n_hidden) {
  using namespace nqs;
  if (!out || !ham) return cfail(nullptr, NQS_EINVAL, "nqs_crbm_create: null argument");
  *out = nullptr;
  if (ham->kind != NQS_TFIM) return cfail(nullptr, NQS_EUNSUPPORTED, "the complex RBM is built for the TFIM");
  if (ham->Lx < 3 || !(ham->Ly == 1 || ham->Ly >= 3))
    return cfail(nullptr, NQS_EINVAL, "periodic lattice needs Lx >= 3 and Ly == 1 or Ly >= 3");
  const int64_t N64 = (int64_t)ham->Lx * ham->Ly;
  if (N64 > 256) return cfail(nullptr, NQS_EUNSUPPORTED, "the complex RBM takes at most 256 sites");
  if (n_hidden < 1 || n_hidden > 512) return cfail(nullptr, NQS_EUNSUPPORTED, "the complex RBM needs 1 <= n_hidden <= 512");
  nqs_crbm *c = new (std::nothrow) nqs_crbm();
  if (!c) return cfail(nullptr, NQS_ENOMEM, "host allocation failed");
  c->N = (int)N64;
  c->W = (c->N + 31) / 32;
  c->M = n_hidden;
  const int need = (c->M + 31) / 32;
  c->KU = 16;
  for (int v : KU_LIST)
    if (v >= need) {
      c->KU = v;
      break;
    }
  c->M_pad = 32 * c->KU;
  c->Lx = ham->Lx;
  c->Ly = ham->Ly;
  c->J = ham->J1;
  c->h = ham->h;
  c->P = (int64_t)c->N + c->M + (int64_t)c->M * c->N;
  nqs_ctx &b = c->base;
  b.model_kind = NQS_RBM;
  b.ham_kind = NQS_TFIM;
  b.N = c->N;
  b.W = c->W;
  b.Lx = c->Lx;
  b.Ly = c->Ly;
  cudaError_t e;
  if ((e = cudaGetDevice(&b.device)) != cudaSuccess) {
    delete c;
    return ccuda(nullptr, e, "cudaGetDevice");
  }
  cudaDeviceGetAttribute(&b.num_sms, cudaDevAttrMultiProcessorCount, b.device);
  std::vector<int2> nb(c->N);
  for (int y = 0; y < c->Ly; ++y)
    for (int x = 0; x < c->Lx; ++x)
      nb[x + c->Lx * y] = make_int2((x + 1) % c->Lx + c->Lx * y, c->Ly > 1 ? x + c->Lx * ((y + 1) % c->Ly) : -1);
  const size_t NM = (size_t)c->N * c->M_pad;
  const int tiles = (c->M + 1 + CR_FU - 1) / CR_FU;
  // row chunks of the SIMT force, and of the tensor-core force (at most one per SM and unit tile)
  c->force_chunks = std::max(std::max(1, (b.num_sms * 4 + tiles - 1) / tiles), b.num_sms);
  if ((e = cudaMalloc(&c->d_fpart, (size_t)c->force_chunks * c->P * sizeof(double2))) ||
      (e = cudaMalloc(&c->d_a, c->N * sizeof(float2))) || (e = cudaMalloc(&c->d_b, c->M_pad * sizeof(float2))) ||
      (e = cudaMalloc(&c->d_Wt, NM * sizeof(float2))) || (e = cudaMalloc(&c->d_st, NM * sizeof(float4))) ||
      (e = cudaMalloc(&c->d_et, NM * sizeof(float4))) || (e = cudaMalloc(&c->d_nb, c->N * sizeof(int2))) ||
      (e = cudaMalloc(&c->d_imstats, 5 * sizeof(double))) || (e = cudaMalloc(&b.d_status, sizeof(int))) ||
      (e = cudaMalloc(&b.d_scratch, 5 * STATS_MAX_BLOCKS * sizeof(double))) ||
      (e = cudaMemset(b.d_status, 0, sizeof(int))) ||
      (e = cudaMemcpy(c->d_nb, nb.data(), nb.size() * sizeof(int2), cudaMemcpyHostToDevice))) {
    crbm_free(c);
    delete c;
    return cfail(nullptr, NQS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  *out = c;
  return NQS_OK;
}

void nqs_crbm_destroy(nqs_crbm *c) {
  if (!c) return;
  nqs::crbm_free(c);
  delete c;
}

nqs_status nqs_crbm_set_refresh(nqs_crbm *c, int32_t refresh) {
  if (!c) return NQS_EINVAL;
  if (refresh < 1) return cfail(c, NQS_EINVAL, "refresh must be >= 1");
  c->refresh = refresh;
  return NQS_OK;
}

nqs_status nqs_crbm_set_params(nqs_crbm *c, const double *params, nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!params) return cfail(c, NQS_EINVAL, "nqs_crbm_set_params: null params");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = 0;
  cudaError_t e = cudaMemsetAsync(c->base.d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return ccuda(c, e, "nqs_crbm_set_params");
  const int64_t total = (int64_t)c->N * c->M_pad;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)c->base.num_sms * 8));
  crbm_prepare_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2 *>(params), c->N, c->M, c->M_pad, c->d_a,
                                             c->d_b, c->d_Wt, c->d_st, c->d_et, c->base.d_status);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&st, c->base.d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return ccuda(c, e, "nqs_crbm_set_params");
  if (st & STATUS_RANGE) {
    c->params_set = false;
    cudaMemsetAsync(c->base.d_status, 0, sizeof(int), s);
    return cfail(c, NQS_EINVAL, "a weight is outside the complex sampler's range (|Re W| <= 1, sum_i |Re W_ji| + |Re b_j| <= 10)");
  }
  c->params_set = true;
  return NQS_OK;
}

nqs_status nqs_crbm_init_chains(nqs_crbm *c, uint32_t *state, int64_t n, uint64_t seed, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n < 0 || (n > 0 && !state)) return cfail(c, NQS_EINVAL, "nqs_crbm_init_chains: bad state/n");
  if (n > (int64_t)UINT32_MAX) return cfail(c, NQS_EINVAL, "at most 2^32 chains");
  if (n == 0) return NQS_OK;
  cudaError_t e = nqs::init_chains(&c->base, state, n, seed, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_init_chains");
}

nqs_status nqs_crbm_sweep(nqs_crbm *c, uint32_t *state, int64_t n_chains, int32_t n_sweeps, int32_t burn_in,
                          uint64_t seed, uint32_t sweep_offset, uint32_t *samples, int64_t *n_accepted,
                          const nqs_sweep_trace *trace, nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return cfail(c, NQS_EINVAL, "nqs_crbm_sweep: parameters not set");
  if (n_chains < 0 || n_sweeps < 0 || burn_in < 0) return cfail(c, NQS_EINVAL, "nqs_crbm_sweep: negative size");
  if (n_chains > (int64_t)UINT32_MAX) return cfail(c, NQS_EINVAL, "at most 2^32 chains");
  if ((uint64_t)sweep_offset + (uint64_t)n_sweeps > (1ull << 32)) return cfail(c, NQS_EINVAL, "sweep counter overflow");
  if (n_chains == 0 || n_sweeps == 0) return NQS_OK;
  if (!state) return cfail(c, NQS_EINVAL, "nqs_crbm_sweep: null state");
  CSweepArgs a;
  a.state = state;
  a.C = n_chains;
  a.N = c->N;
  a.W = c->W;
  a.M_pad = c->M_pad;
  a.T = n_sweeps;
  a.B = burn_in;
  a.refresh = c->refresh;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.sweep_offset = sweep_offset;
  a.a = c->d_a;
  a.b = c->d_b;
  a.Wt = c->d_Wt;
  a.st = c->d_st;
  a.samples = samples;
  a.n_acc = n_accepted;
  a.acc_bits = trace ? trace->accept_bits : nullptr;
  a.delta = trace ? trace->delta : nullptr;
  cudaError_t e = dispatch_sweep(c, a, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_sweep");
}

nqs_status nqs_crbm_logpsi(nqs_crbm *c, const uint32_t *cfg, int64_t n, float *out, nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return cfail(c, NQS_EINVAL, "nqs_crbm_logpsi: parameters not set");
  if (n < 0 || (n > 0 && (!cfg || !out))) return cfail(c, NQS_EINVAL, "nqs_crbm_logpsi: bad arguments");
  if (n == 0) return NQS_OK;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n * 32 + CR_THREADS - 1) / CR_THREADS, (int64_t)c->base.num_sms * 16));
  crbm_logpsi_kernel<<<(unsigned)blocks, CR_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(row_args(c, cfg, n), out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_logpsi");
}

nqs_status nqs_crbm_local_energy(nqs_crbm *c, const uint32_t *cfg, int64_t n, float *eloc_re, float *eloc_im,
                                 nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return cfail(c, NQS_EINVAL, "nqs_crbm_local_energy: parameters not set");
  if (n < 0 || (n > 0 && (!cfg || !eloc_re || !eloc_im))) return cfail(c, NQS_EINVAL, "nqs_crbm_local_energy: bad arguments");
  if (n == 0) return NQS_OK;
  CElocArgs a;
  a.r = row_args(c, cfg, n);
  a.et = c->d_et;
  a.nb = c->d_nb;
  a.J = (float)c->J;
  a.h = (float)c->h;
  a.eloc_re = eloc_re;
  a.eloc_im = eloc_im;
  a.n_chains = 0;
  a.refresh = c->refresh;
  cudaError_t e = dispatch_eloc(c, a, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_local_energy");
}

nqs_status nqs_crbm_local_energy_chains(nqs_crbm *c, const uint32_t *samples, int64_t n_chains, int64_t per_chain,
                                        float *eloc_re, float *eloc_im, nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return cfail(c, NQS_EINVAL, "nqs_crbm_local_energy_chains: parameters not set");
  if (n_chains < 0 || per_chain < 0) return cfail(c, NQS_EINVAL, "nqs_crbm_local_energy_chains: negative size");
  if (n_chains == 0 || per_chain == 0) return NQS_OK;
  if (!samples || !eloc_re || !eloc_im) return cfail(c, NQS_EINVAL, "nqs_crbm_local_energy_chains: null argument");
  // a warp per chain: with fewer than 16 chains per SM that leaves the GPU mostly idle, so the
  // per-sample evaluation (the same values to FP32 rounding) is used
  if (n_chains < (int64_t)c->base.num_sms * 16)
    return nqs_crbm_local_energy(c, samples, n_chains * per_chain, eloc_re, eloc_im, stream);
  CElocArgs a;
  a.r = row_args(c, samples, n_chains * per_chain);
  a.et = c->d_et;
  a.nb = c->d_nb;
  a.J = (float)c->J;
  a.h = (float)c->h;
  a.eloc_re = eloc_re;
  a.eloc_im = eloc_im;
  a.n_chains = n_chains;
  a.refresh = c->refresh;
  cudaError_t e = dispatch_eloc(c, a, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_local_energy_chains");
}

nqs_status nqs_crbm_stats(nqs_crbm *c, const float *eloc_re, const float *eloc_im, int64_t n, int64_t n_chains,
                          const int64_t *n_accepted, int64_t proposals_per_chain, double *out, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n <= 0 || n_chains <= 0 || n % n_chains != 0 || !eloc_re || !eloc_im || !out)
    return cfail(c, NQS_EINVAL, "nqs_crbm_stats: need n > 0 a multiple of n_chains and non-null eloc/out");
  if (n_accepted && proposals_per_chain <= 0) return cfail(c, NQS_EINVAL, "nqs_crbm_stats: proposals_per_chain must be > 0");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = nqs::energy_stats(&c->base, eloc_re, n, n_chains, n_accepted, proposals_per_chain, out, s);
  if (e == cudaSuccess) e = nqs::energy_stats(&c->base, eloc_im, n, n_chains, nullptr, 1, c->d_imstats, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out + 5, c->d_imstats, sizeof(double), cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_stats");
}

nqs_status nqs_crbm_logpsi_grad(nqs_crbm *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc_re,
                                const float *eloc_im, const double *stats, double *force, nqs_stream stream) {
  using namespace nqs;
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return cfail(c, NQS_EINVAL, "nqs_crbm_logpsi_grad: parameters not set");
  if (n < 0 || (n > 0 && !cfg)) return cfail(c, NQS_EINVAL, "nqs_crbm_logpsi_grad: bad arguments");
  if (force && n > 0 && (!eloc_re || !eloc_im || !stats))
    return cfail(c, NQS_EINVAL, "nqs_crbm_logpsi_grad: the force needs eloc and stats");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (n == 0) {
    if (force) e = cudaMemsetAsync(force, 0, (size_t)c->P * 2 * sizeof(double), s);
    return e == cudaSuccess ? NQS_OK : ccuda(c, e, "nqs_crbm_logpsi_grad");
  }
  const CRowArgs r = row_args(c, cfg, n);
  if (O) {
    const int64_t blocks = std::min<int64_t>(n, (int64_t)c->base.num_sms * 16);
    crbm_grad_rows_kernel<<<(unsigned)blocks, CR_THREADS, c->M_pad * sizeof(float2), s>>>(
        r, c->P, reinterpret_cast<float2 *>(O));
    if ((e = cudaGetLastError()) != cudaSuccess) return ccuda(c, e, "nqs_crbm_logpsi_grad");
  }
  if (force && c->N <= 127) {  // tensor-core path: spins, the constant site and the weights in K = 128
    const int chunks = std::min(c->force_chunks, crbm_force_tc_chunks(c->M, c->base.num_sms, n));
    e = crbm_force_tc(cfg, n, c->N, c->W, c->M, c->M_pad, c->P, c->d_Wt, c->d_b, eloc_re, eloc_im, stats, c->d_fpart,
                      chunks, reinterpret_cast<double2 *>(force), c->base.d_status, s);
    if (e != cudaSuccess) return ccuda(c, e, "nqs_crbm_logpsi_grad");
  } else if (force) {
    CForceArgs a;
    a.r = r;
    a.eloc_re = eloc_re;
    a.eloc_im = eloc_im;
    a.stats = stats;
    a.part = c->d_fpart;
    a.P = c->P;
    const int tiles = (c->M + 1 + CR_FU - 1) / CR_FU;
    const int64_t blocks_rows = (n + CR_FR - 1) / CR_FR;
    const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(blocks_rows, c->force_chunks));
    a.rows_per_cta = ((blocks_rows + chunks - 1) / chunks) * CR_FR;
    const int64_t gx = (n + a.rows_per_cta - 1) / a.rows_per_cta;
    if (2 * (c->N + 1) <= CR_FTHREADS)
      crbm_force_kernel<2><<<dim3((unsigned)gx, (unsigned)tiles), CR_FTHREADS, 0, s>>>(a);
    else
      crbm_force_kernel<1><<<dim3((unsigned)gx, (unsigned)tiles), CR_FTHREADS, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return ccuda(c, e, "nqs_crbm_logpsi_grad");
    crbm_force_reduce_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((c->P + 255) / 256, 1024)), 256, 0,
                               s>>>(c->d_fpart, (int)gx, c->P, 1.0 / (double)n, reinterpret_cast<double2 *>(force));
    if ((e = cudaGetLastError()) != cudaSuccess) return ccuda(c, e, "nqs_crbm_logpsi_grad");
  }
  return NQS_OK;
}

nqs_status nqs_crbm_check_status(nqs_crbm *c, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  nqs_status st = nqs_check_status(&c->base, stream);
  if (st != NQS_OK) c->err = c->base.err;
  return st;
}

}  // extern "C"
