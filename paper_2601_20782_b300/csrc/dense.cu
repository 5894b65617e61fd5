// Dense feed-forward ansatz: sampling copy, forward passes, local energies, the
// exchange-move sampler and the FP32 backward for O_k.
//
//   a_0 = log cosh(W_0 s + b_0),  a_l = tanh(W_l a_{l-1} + b_l) (l >= 1),  log psi = w_out . a_{L-1} + b_out
// (the paper names feed-forward networks without fixing an architecture; this is the
// reading used throughout).  Parameters, flat FP64: [W_0 (H0 x N) | b_0 | W_1 (H1 x H0) |
// b_1 | ... | w_out (H_{L-1}) | b_out].
//
// Sampling copy (Sec. 4.2): W_l (l >= 1) in BF16 for the tensor cores, W_0 rounded to BF16
// and kept in FP32 for the layer-0 pre-activations z0 = W_0 s + b_0, which are cached per
// chain in FP32 and updated incrementally on an accepted move (two columns for an
// exchange, one for a flip).  Rows of a pass = configurations whose log psi is needed:
// the cached z0 of a source configuration plus the move's column difference, then
// log cosh -> BF16 -> GEMM chain (dense_gemm.cu) -> log psi.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nqs {
namespace {

constexpr float LN2 = 0.693147180559945309f;

__device__ __forceinline__ float log_cosh_f(float z) {
  z = fabsf(z);
  return z + log1pf(expf(-2.f * z)) - LN2;
}
// MUFU form for activations that are rounded to BF16 right after (error ~1e-6 << 2^-9)
__device__ __forceinline__ float log_cosh_fast(float z) {
  z = fabsf(z);
  return z + __logf(1.f + __expf(-2.f * z)) - LN2;
}

// Two adjacent activations of a layer's input row, in the activation type of the copy:
// BF16 (the BF16 copy) or E4M3 (the FP8 copy).
__device__ __forceinline__ void store_act2(__nv_bfloat16 *row, int k, float v0, float v1) {
  *reinterpret_cast<__nv_bfloat162 *>(row + k) = __floats2bfloat162_rn(v0, v1);
}
__device__ __forceinline__ void store_act2(uint8_t *row, int k, float v0, float v1) {
  *reinterpret_cast<uint16_t *>(row + k) = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
}

// ------------------------------------------------------------------------------------
// sampling copy and FP32 master from the FP64 parameters
__global__ void dense_prepare_kernel(const double *__restrict__ p, int64_t P, int N, int H0, float *master, float *W1t,
                                     float *b1, float *status_unused) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    master[k] = (float)p[k];
    if (k < (int64_t)H0 * N) {  // W_0[j][i] -> site-major, rounded to BF16
      const int j = (int)(k / N), i = (int)(k % N);
      W1t[(int64_t)i * H0 + j] = __bfloat162float(__double2bfloat16(p[k]));
    } else if (k < (int64_t)H0 * N + H0) {
      b1[k - (int64_t)H0 * N] = __bfloat162float(__double2bfloat16(p[k]));
    }
  }
}

// layer l >= 1: W_l [H x K] (flat at off) -> BF16 [H][Kp] (padding stays zero); bias, w_out
__global__ void dense_prepare_layer_kernel(const double *__restrict__ p, int64_t off, int H, int K, int Kp,
                                           __nv_bfloat16 *Wl, float *bl, const double *w_out_src, float *w_out,
                                           int last) {
  const int64_t total = (int64_t)H * K;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / K), kk = (int)(k % K);
    Wl[(int64_t)n * Kp + kk] = __double2bfloat16(p[off + k]);
    if (kk == 0) {
      bl[n] = __bfloat162float(__double2bfloat16(p[off + total + n]));
      if (last) w_out[n] = __bfloat162float(__double2bfloat16(w_out_src[n]));
    }
  }
}

// FP8 copy.  max |W_l| of each weight matrix (l = 0: W_0 [H0 x N] at 0; l >= 1 at its offset),
// as FP32 bits (non-negative floats order as integers)
__global__ void dense_wmax_kernel(const double *__restrict__ p, int64_t off, int64_t count, unsigned *wmax) {
  float m = 0.f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)p[off + k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(wmax, __float_as_uint(m));
}
// s_l = the largest power of two with max |W_l| s_l <= 448 (the E4M3 maximum); 1 for W_l = 0
__global__ void dense_scale8_kernel(const unsigned *wmax, int L, float *scale) {
  const int l = threadIdx.x;
  if (l >= L) return;
  const float m = __uint_as_float(wmax[l]);
  const float sc = m > 0.f ? exp2f(floorf(log2f(448.f / m))) : 1.f;
  scale[l] = sc;
  scale[L + l] = 1.f / sc;
}
__device__ __forceinline__ float e4m3_round(float v) {
  const __nv_fp8_e4m3 q(v);  // round to nearest even, saturating
  return (float)q;
}
// layer 0 of the FP8 copy: W1t8[i][j] = E4M3(W_0[j][i] s_0) / s_0 (FP32 values, site-major)
__global__ void dense_prepare8_l0_kernel(const double *__restrict__ p, int N, int H0, const float *scale,
                                         float *W1t8) {
  const float s0 = scale[0];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)H0 * N; k += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / N), i = (int)(k % N);
    W1t8[(int64_t)i * H0 + j] = e4m3_round((float)p[k] * s0) / s0;
  }
}
// layer l >= 1: W_l [H x K] (flat at off) -> E4M3 of W_l s_l, [H][Kp8] (padding stays zero)
__global__ void dense_prepare8_layer_kernel(const double *__restrict__ p, int64_t off, int H, int K, int Kp8,
                                            const float *scale_l, uint8_t *Wl8) {
  const float sl = *scale_l;
  const int64_t total = (int64_t)H * K;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k / K), kk = (int)(k % K);
    Wl8[(int64_t)n * Kp8 + kk] = __nv_cvt_float_to_fp8((float)p[off + k] * sl, __NV_SATFINITE, __NV_E4M3);
  }
}

// ------------------------------------------------------------------------------------
// z0 = W_0 s + b_0 for n configurations, FP32.  Block (row block, column block): Z0_ROWS
// configurations x 128 hidden units, thread per unit with Z0_ROWS accumulators; the spin
// words of the block's rows are read once per 32 sites into registers.
constexpr int Z0_ROWS = 8;
constexpr int Z0_COLS = 128;
__global__ void __launch_bounds__(Z0_COLS) dense_z0_kernel(const uint32_t *__restrict__ cfg, int64_t n,
                                                           const float *__restrict__ W1t,
                                                           const float *__restrict__ b1, int N, int W, int H0,
                                                           float *z0) {
  const int n_cb = (H0 + Z0_COLS - 1) / Z0_COLS;
  const int64_t n_blocks = (n + Z0_ROWS - 1) / Z0_ROWS * n_cb;
  for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int64_t x0 = blk / n_cb * Z0_ROWS;
    const int j = (int)(blk % n_cb) * Z0_COLS + threadIdx.x;
    const int nr = (int)(n - x0 < Z0_ROWS ? n - x0 : Z0_ROWS);
    if (j >= H0) continue;
    float acc[Z0_ROWS];
    const float bj = b1[j];
#pragma unroll
    for (int r = 0; r < Z0_ROWS; ++r) acc[r] = bj;
    for (int w = 0; w < W; ++w) {
      uint32_t word[Z0_ROWS];
#pragma unroll
      for (int r = 0; r < Z0_ROWS; ++r) word[r] = r < nr ? __ldg(cfg + (x0 + r) * W + w) : 0u;
      const int i1 = N - 32 * w < 32 ? N - 32 * w : 32;
      const float *wp = W1t + (int64_t)(32 * w) * H0 + j;
#pragma unroll 4
      for (int b = 0; b < i1; ++b) {
        const float wv = __ldg(wp + (int64_t)b * H0);
#pragma unroll
        for (int r = 0; r < Z0_ROWS; ++r) acc[r] += ((word[r] >> b) & 1u) ? wv : -wv;
      }
    }
#pragma unroll
    for (int r = 0; r < Z0_ROWS; ++r)
      if (r < nr) z0[(x0 + r) * H0 + j] = acc[r];
  }
}

static unsigned z0_grid(int64_t n, int H0, int num_sms) {
  const int64_t blocks = (n + Z0_ROWS - 1) / Z0_ROWS * ((H0 + Z0_COLS - 1) / Z0_COLS);
  const int64_t cap = (int64_t)num_sms * 16;
  return (unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

// A move: flip site i (j < 0) or exchange sites i and j; valid only if the spins differ
// for an exchange (otherwise the move is the identity).
struct Move {
  int i, j;
};

__device__ __forceinline__ int spin_of(const uint32_t *cfg, int W, int64_t x, int i) {
  return ((cfg[x * W + (i >> 5)] >> (i & 31)) & 1u) ? 1 : -1;
}

// Row r of the layer-0 output: log cosh(z0[src] + move delta) in BF16, [R][Kp1].
// mode 0: plain rows (src = r).  mode 1: local-energy rows r = x * (1 + nconn) + k; k = 0 is
// the configuration itself, k >= 1 the k-1-th connected move (site flip for TFIM, bond
// exchange for Heisenberg).  The sampler's rows come from dense_propose_kernel.
struct A1Args {
  const uint32_t *cfg;
  const float *z0;
  const float *W1t;
  const int2 *bonds;
  void *act;  // BF16 or E4M3 rows (the kernel's activation type)
  int64_t R;
  int N, W, H0, Kp1, nconn, mode, exchange;
};

__device__ __forceinline__ bool row_move(const A1Args &a, int64_t r, int64_t *src, Move *mv) {
  if (a.mode == 0) {
    *src = r;
    return false;
  }
  *src = r / (1 + a.nconn);
  const int m = (int)(r % (1 + a.nconn)) - 1;
  if (m < 0) return false;
  if (a.exchange) {
    const int2 b = a.bonds[m];
    mv->i = b.x;
    mv->j = b.y;
    return spin_of(a.cfg, a.W, *src, b.x) != spin_of(a.cfg, a.W, *src, b.y);
  }
  mv->i = m;
  mv->j = -1;
  return true;
}

template <typename TA>
__global__ void dense_a1_kernel(const A1Args a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < a.R; r += nw) {
    int64_t src;
    Move mv{0, -1};
    const bool moved = row_move(a, r, &src, &mv);
    const float si = moved ? (float)spin_of(a.cfg, a.W, src, mv.i) : 0.f;
    const float *zr = a.z0 + src * a.H0;
    const float *wi = a.W1t + (int64_t)mv.i * a.H0;
    const float *wj = a.W1t + (int64_t)(mv.j < 0 ? 0 : mv.j) * a.H0;
    TA *out = static_cast<TA *>(a.act) + r * a.Kp1;
    // flip: s_i -> -s_i; exchange: s_i -> -s_i and s_j = -s_i -> s_i
    if ((a.H0 & 3) == 0) {  // four units per lane per step, 16-byte loads (rows 16-byte aligned)
      for (int k = 4 * lane; k < a.H0; k += 128) {
        float4 z = *reinterpret_cast<const float4 *>(zr + k);
        if (moved) {
          float4 d = *reinterpret_cast<const float4 *>(wi + k);
          if (mv.j >= 0) {
            const float4 e = *reinterpret_cast<const float4 *>(wj + k);
            d = make_float4(d.x - e.x, d.y - e.y, d.z - e.z, d.w - e.w);
          }
          z = make_float4(fmaf(-2.f * si, d.x, z.x), fmaf(-2.f * si, d.y, z.y), fmaf(-2.f * si, d.z, z.z),
                          fmaf(-2.f * si, d.w, z.w));
        }
        store_act2(out, k, log_cosh_fast(z.x), log_cosh_fast(z.y));
        store_act2(out, k + 2, log_cosh_fast(z.z), log_cosh_fast(z.w));
      }
    } else {
      for (int k = 2 * lane; k < a.H0; k += 64) {  // two units per lane per step (H0 even)
        float z0v = zr[k], z1v = zr[k + 1];
        if (moved) {
          const float d0 = mv.j < 0 ? wi[k] : wi[k] - wj[k];
          const float d1 = mv.j < 0 ? wi[k + 1] : wi[k + 1] - wj[k + 1];
          z0v = fmaf(-2.f * si, d0, z0v);
          z1v = fmaf(-2.f * si, d1, z1v);
        }
        store_act2(out, k, log_cosh_fast(z0v), log_cosh_fast(z1v));
      }
    }
  }
}

// log psi of the rows: sum of the last layer's range partials + b_out
__global__ void dense_sum_kernel(const float *part, int64_t R, int n_ranges, const float *b_out, float *out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    float s = b_out[0];
    for (int q = 0; q < 2 * n_ranges; ++q) s += part[r * 2 * n_ranges + q];
    out[r] = s;
  }
}

// ------------------------------------------------------------------------------------
// Local energy from the rows' log psi (App. I, Eq. local_energies).  TFIM (Eq. TFIM):
// J sum s_i s_j + h sum_i psi(flip_i x)/psi(x).  Heisenberg (App. E): sum_b J_b s_i s_j
// + sum over anti-aligned bonds of 2 J_b sign_b psi(x_b)/psi(x), sign_b = -1 when the
// Marshall rule is on and the bond joins the two sublattices.
__global__ void dense_eloc_combine_kernel(const uint32_t *__restrict__ cfg, int64_t n, const float *lp_rows,
                                          const int2 *bonds, const float *bondJ, int n_bonds, int N, int W, int Lx,
                                          int exchange, int marshall, float J, float h, float *eloc) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nconn = exchange ? n_bonds : N;
  for (int64_t x = gw; x < n; x += nw) {
    const float *lp = lp_rows + x * (1 + nconn);
    const float l0 = lp[0];
    float acc = 0.f;
    for (int b = lane; b < n_bonds; b += 32) {
      const int2 bd = bonds[b];
      const int si = spin_of(cfg, W, x, bd.x), sj = spin_of(cfg, W, x, bd.y);
      const float Jb = exchange ? bondJ[b] : J;
      acc += Jb * (float)(si * sj);
      if (exchange && si != sj) {
        float sign = 1.f;
        if (marshall) {
          const int pi_ = (bd.x % Lx + bd.x / Lx) & 1, pj = (bd.y % Lx + bd.y / Lx) & 1;
          if (pi_ != pj) sign = -1.f;
        }
        acc += 2.f * Jb * sign * expf(lp[1 + b] - l0);
      }
    }
    if (!exchange)
      for (int i = lane; i < N; i += 32) acc += h * expf(lp[1 + i] - l0);
    acc = group_allsum<32>(acc);
    if (lane == 0) eloc[x] = acc;
  }
}

// ------------------------------------------------------------------------------------
// Sampler.  Proposal p of sweep t of chain c: Philox counter (p/2, sweep, c, TAG_SWEEP),
// words (0,1) for even p and (2,3) for odd p: move = (w * n_moves) >> 32 (a bond of the
// Hamiltonian for Heisenberg, a site for TFIM), u = (w' >> 8) 2^-24.  The draw happens
// in dense_a1_kernel (mode 2), which also writes the proposal's layer-0 row.
// ------------------------------------------------------------------------------------
// One Metropolis step of every chain for the dense ansatz (Sec. 2.2 sampler, App. I
// incremental layer 0).  Warp per chain c; the chain's layer-0 pre-activations z0[c] live
// in FP32 and are updated by the accepted move only.  In order:
//  1. decision of the previous step (decide): log psi(y) = b_out + the last layer's range
//     partials of row c, accepted iff 2 (log psi(y) - log psi(x)) > log u (u = 0 always);
//     bookkeeping (accept count, accept bits, increments) for proposal (t_prev, p_prev);
//  2. the accepted move (pending): z0 += -2 s_i (W_i - W_j) (W_j only for an exchange),
//     spins moved;
//  3. the configuration after a completed sweep (emit_row >= 0) written to the samples;
//  4. proposal p of sweep sweep_id (propose): Philox words (0,1) / (2,3) of counter
//     (p/2, sweep_id, chain, TAG_SWEEP) give the move and u; the proposal's layer-0 row
//     log cosh(z0 + its delta) is written in BF16 for the GEMM chain.  An exchange of
//     equal spins is the identity (prop = -1, accepted without evaluation).
struct ProposeArgs {
  uint32_t *state;
  float *z0;
  const float *W1t;
  const int2 *bonds;
  int32_t *prop;
  float *thr;
  float *lp;
  void *act;  // BF16 or E4M3 rows (the kernel's activation type)
  const float *part;
  const float *b_out;
  int n_ranges;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
  uint32_t *samples;
  float *logpsi;
  int64_t C;
  int N, W, H0, Kp1, exchange, n_moves, n_sweeps;
  int decide, first, t_prev, p_prev;
  int emit_row;
  int propose, p;
  uint32_t sweep_id, k0, k1;
};

template <int NJ, typename TA>  // column block of 64 * NJ units held in registers, two per lane per j
__global__ void __launch_bounds__(256, 4) dense_propose_kernel(const ProposeArgs a) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < a.C; c += nw) {
    // ---- every load that does not depend on the decision is issued first
    uint32_t word = lane < a.W ? a.state[c * a.W + lane] : 0u;
    const float lp0 = a.lp[c];
    const int mp = a.decide ? a.prop[c] : -1;
    const float thr_old = a.decide ? a.thr[c] : 0.f;
    int m = 0;
    float thr_new = 0.f;
    int2 nb = make_int2(0, -1);
    if (a.propose) {  // this step's proposal: Philox, then its bond
      const uint4 w = philox4x32_10(make_uint4((uint32_t)(a.p / 2), a.sweep_id, (uint32_t)c, TAG_SWEEP), a.k0, a.k1);
      const uint32_t wm = (a.p & 1) ? w.z : w.x, wu = (a.p & 1) ? w.w : w.y;
      m = (int)index_from_word(wm, (uint32_t)a.n_moves);
      const uint32_t k = wu >> 8;
      thr_new = k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
      nb = a.exchange ? a.bonds[m] : make_int2(m, -1);
    }
    // the previous proposal's bond, fetched before knowing whether it was accepted
    const int2 pbc = mp >= 0 ? (a.exchange ? a.bonds[mp] : make_int2(mp, -1)) : make_int2(0, -1);
    float part = 0.f;
    if (mp >= 0)
      for (int q = lane; q < 2 * a.n_ranges; q += 32) part += a.part[c * 2 * a.n_ranges + q];
    // ---- decision of the previous proposal
    bool pending = false;
    float lp_c = lp0;
    if (a.decide) {
      bool acc = true;
      float dlt = 0.f;
      if (mp >= 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(full, part, o);
        const float lpn = a.b_out[0] + part;
        dlt = lpn - lp0;
        acc = 2.f * dlt > thr_old;
        if (acc) {
          lp_c = lpn;
          pending = true;
        }
      }
      __syncwarp();  // every lane has read prop/thr/lp of chain c
      if (lane == 0) {
        if (pending) a.lp[c] = lp_c;
        if (a.n_acc) a.n_acc[c] = (a.first ? 0 : a.n_acc[c]) + (acc ? 1 : 0);
        if (a.acc_bits) {
          const int64_t wi = ((int64_t)c * a.n_sweeps + a.t_prev) * a.W + (a.p_prev >> 5);
          const uint32_t bit = 1u << (a.p_prev & 31);
          a.acc_bits[wi] = ((a.p_prev & 31) == 0 ? 0u : a.acc_bits[wi]) | (acc ? bit : 0u);
        }
        if (a.delta) a.delta[((int64_t)c * a.n_sweeps + a.t_prev) * a.N + a.p_prev] = dlt;
      }
    }
    const int2 pb = pending ? pbc : make_int2(0, -1);
    float gp = 0.f;  // pending move: z0 += gp (W_i - W_j)
    if (pending) {
      gp = ((__shfl_sync(full, word, pb.x >> 5) >> (pb.x & 31)) & 1u) ? -2.f : 2.f;
      if (lane == (pb.x >> 5)) word ^= 1u << (pb.x & 31);
      if (pb.y >= 0 && lane == (pb.y >> 5)) word ^= 1u << (pb.y & 31);
      if (lane < a.W) a.state[c * a.W + lane] = word;
    }
    if (a.emit_row >= 0) {
      const int64_t row = (int64_t)a.emit_row * a.C + c;
      if (a.samples && lane < a.W) a.samples[row * a.W + lane] = word;
      if (a.logpsi && lane == 0) a.logpsi[row] = lp_c;
    }
    bool moved = false;
    float gn = 0.f;  // proposal: z = z0 + gn (W_i - W_j)
    if (a.propose) {
      const int sx = (__shfl_sync(full, word, nb.x >> 5) >> (nb.x & 31)) & 1u;
      moved = true;
      if (nb.y >= 0) moved = sx != (int)((__shfl_sync(full, word, nb.y >> 5) >> (nb.y & 31)) & 1u);
      gn = sx ? -2.f : 2.f;
      __syncwarp();
      if (lane == 0) {
        a.thr[c] = thr_new;
        a.prop[c] = moved ? m : -1;
      }
    }
    if (!pending && !a.propose) continue;
    float *zr = a.z0 + c * a.H0;
    const float *pi = a.W1t + (int64_t)pb.x * a.H0, *pj = a.W1t + (int64_t)(pb.y < 0 ? 0 : pb.y) * a.H0;
    const float *ni = a.W1t + (int64_t)nb.x * a.H0, *nj = a.W1t + (int64_t)(nb.y < 0 ? 0 : nb.y) * a.H0;
    TA *out = static_cast<TA *>(a.act) + c * a.Kp1;
    const bool use_new = a.propose && moved;
    for (int kb = 0; kb < a.H0; kb += 64 * NJ) {
      // all loads of the block (z row, the two moves' weight differences) before any store
      float2 z[NJ], dp[NJ], dn[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int k = kb + 64 * j + 2 * lane;
        const bool in = k < a.H0;
        z[j] = in ? *reinterpret_cast<const float2 *>(zr + k) : make_float2(0.f, 0.f);
        dp[j] = make_float2(0.f, 0.f);
        dn[j] = make_float2(0.f, 0.f);
        if (pending && in) {
          dp[j] = *reinterpret_cast<const float2 *>(pi + k);
          if (pb.y >= 0) {
            const float2 t = *reinterpret_cast<const float2 *>(pj + k);
            dp[j].x -= t.x;
            dp[j].y -= t.y;
          }
        }
        if (use_new && in) {
          dn[j] = *reinterpret_cast<const float2 *>(ni + k);
          if (nb.y >= 0) {
            const float2 t = *reinterpret_cast<const float2 *>(nj + k);
            dn[j].x -= t.x;
            dn[j].y -= t.y;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int k = kb + 64 * j + 2 * lane;
        if (k < a.H0) {
          if (pending) {
            z[j].x = fmaf(gp, dp[j].x, z[j].x);
            z[j].y = fmaf(gp, dp[j].y, z[j].y);
            *reinterpret_cast<float2 *>(zr + k) = z[j];
          }
          if (a.propose) {
            const float vx = fmaf(gn, dn[j].x, z[j].x), vy = fmaf(gn, dn[j].y, z[j].y);
            store_act2(out, k, log_cosh_fast(vx), log_cosh_fast(vy));
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// O_k rows in FP32 (App. I, Eq. forces), one block per configuration: forward with the
// FP32 master, then the hand-written backward
//   delta_{L-1} = w_out (1 - a_{L-1}^2),  delta_{l-1} = (W_l^T delta_l) f'_{l-1}(z_{l-1}),
//   f'_0 = tanh (log cosh), f'_l = 1 - tanh^2 (l >= 1);
//   O_{W_l} = delta_l a_{l-1}^T (a_{-1} = s),  O_{b_l} = delta_l,  O_{w_out} = a_{L-1},  O_{b_out} = 1.
struct GradArgs {
  const uint32_t *cfg;
  const float *master;
  float *O;        // [n][P]
  int64_t n, P;
  int N, W, L;
  int H[8];
  int64_t offW[8], offb[8], offw_out;
};

__global__ void __launch_bounds__(256) dense_grad_kernel(const GradArgs g) {
  extern __shared__ float sh[];
  float *s = sh;  // [N]
  float *za = s + g.N;  // per layer: z then a (2 * H[l] each)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t x = blockIdx.x; x < g.n; x += gridDim.x) {
    for (int i = tid; i < g.N; i += blockDim.x) s[i] = ((g.cfg[x * g.W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    __syncthreads();
    // forward
    const float *in = s;
    int K = g.N;
    float *zl = za;
    for (int l = 0; l < g.L; ++l) {
      const int Hl = g.H[l];
      float *al = zl + Hl;
      const float *Wl = g.master + g.offW[l];
      for (int nn = warp; nn < Hl; nn += 8) {  // warp per output unit, lanes over the input
        float acc = 0.f;
        for (int k = lane; k < K; k += 32) acc = fmaf(Wl[(int64_t)nn * K + k], in[k], acc);
        acc = group_allsum<32>(acc);
        if (lane == 0) {
          const float z = acc + g.master[g.offb[l] + nn];
          zl[nn] = z;
          al[nn] = l == 0 ? log_cosh_f(z) : tanhf(z);
        }
      }
      __syncthreads();
      in = al;
      K = Hl;
      zl = al + Hl;
    }
    // backward: delta of the last layer into the z slot (z no longer needed there)
    float *row = g.O + x * g.P;
    {
      const int l = g.L - 1;
      float *zL = za;
      for (int q = 0; q < l; ++q) zL += 2 * g.H[q];
      const float *aL = zL + g.H[l];
      for (int nn = tid; nn < g.H[l]; nn += blockDim.x) {
        row[g.offw_out + nn] = aL[nn];
        zL[nn] = g.master[g.offw_out + nn] * (1.f - aL[nn] * aL[nn]);
      }
      if (tid == 0) row[g.P - 1] = 1.f;
    }
    __syncthreads();
    for (int l = g.L - 1; l >= 0; --l) {
      float *zl2 = za;
      for (int q = 0; q < l; ++q) zl2 += 2 * g.H[q];
      const float *dl = zl2;  // delta_l
      const int Hl = g.H[l];
      const int Kl = l == 0 ? g.N : g.H[l - 1];
      const float *ain = l == 0 ? s : zl2 - Kl;  // a_{l-1}
      // O_{W_l} = delta_l a_{l-1}^T (row n of the block = delta_l[n] a_{l-1}) and O_{b_l} = delta_l
      for (int nn = warp; nn < Hl; nn += 8) {
        const float dn = dl[nn];
        float *dst = row + g.offW[l] + (int64_t)nn * Kl;
        for (int k = lane; k < Kl; k += 32) dst[k] = dn * ain[k];
      }
      for (int nn = tid; nn < Hl; nn += blockDim.x) row[g.offb[l] + nn] = dl[nn];
      if (l > 0) {
        // delta_{l-1} = (W_l^T delta_l) f'(z_{l-1}) into the z slot of layer l-1
        float *zprev = zl2 - 2 * Kl;
        const float *aprev = zprev + Kl;
        const float *Wl = g.master + g.offW[l];
        __syncthreads();
        float *tmp = zl2 + Hl;  // a_l slot, free now
        for (int k = tid; k < Kl; k += blockDim.x) {
          float acc = 0.f;
          for (int nn = 0; nn < Hl; ++nn) acc = fmaf(Wl[(int64_t)nn * Kl + k], dl[nn], acc);
          const float fp = (l - 1 == 0) ? tanhf(zprev[k]) : (1.f - aprev[k] * aprev[k]);
          tmp[k] = acc * fp;
        }
        __syncthreads();
        for (int k = tid; k < Kl; k += blockDim.x) zprev[k] = tmp[k];
      }
      __syncthreads();
    }
  }
}

// F_k (+)= sum_x O[x][k] (eloc[x] - E) / n over a chunk of rows.  Block (column tile of
// 256, row slice of at most 256 rows): FP32 products and sum within the slice (FP64 arithmetic
// is a small fraction of the FP32 rate on this GPU), FP64 across slices: part[slice][k],
// added in a fixed order by dense_force_sum_kernel.
constexpr int FORCE_SLICES = 64;
__global__ void __launch_bounds__(256) dense_force_part_kernel(const float *O, int64_t rows, int64_t P,
                                                               const float *eloc, const double *stats, double *part) {
  __shared__ float se[256];
  const double E = stats[0];
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int slice = blockIdx.y;
  const int64_t per = (rows + FORCE_SLICES - 1) / FORCE_SLICES;
  const int64_t x0 = slice * per, x1 = min(rows, x0 + per);
  double s = 0.0;
  for (int64_t xb = x0; xb < x1; xb += 256) {
    const int nb = (int)(x1 - xb < 256 ? x1 - xb : 256);
    __syncthreads();
    if (threadIdx.x < nb) se[threadIdx.x] = (float)((double)eloc[xb + threadIdx.x] - E);
    __syncthreads();
    if (k < P) {
      float f0 = 0.f, f1 = 0.f;
      const float *col = O + xb * P + k;
      int x = 0;
      for (; x + 1 < nb; x += 2) {
        f0 = fmaf(col[(int64_t)x * P], se[x], f0);
        f1 = fmaf(col[(int64_t)(x + 1) * P], se[x + 1], f1);
      }
      if (x < nb) f0 = fmaf(col[(int64_t)x * P], se[x], f0);
      s += (double)f0 + (double)f1;
    }
  }
  if (k < P) part[slice * P + k] = s;
}
// ndiv: when given, the divisor is *ndiv (stats[4], the total sample count of a multi-rank step)
__global__ void dense_force_sum_kernel(const double *part, int64_t P, int64_t n_total, const double *ndiv,
                                       int accumulate, double *force) {
  const double d = ndiv ? *ndiv : (double)n_total;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < FORCE_SLICES; ++q) s += part[q * P + k];
    s /= d;
    force[k] = accumulate ? force[k] + s : s;
  }
}

int grid_for(int64_t work, int per_block, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, (int64_t)num_sms * 16));
}

// GEMM chain over layers 1..L-1 for R rows whose layer-0 output is in act[0]; writes log psi
// (out == nullptr: leaves the last layer's partials in d_part and returns their range count).
// With fewer row tiles than half the SMs each layer uses its split configuration (N-ranges
// of half the width) so that more CTAs share the work; with enough row tiles for every SM
// to take two of them per N-range, the tall configuration (two row tiles per CTA on the
// half-width ranges, more products per byte of operands).
// f8: the FP8 copy's E4M3 activations, weights and scales.
cudaError_t run_chain(const nqs_ctx *c, int64_t R, float *out, const float *b_out_dev, cudaStream_t s,
                      int *n_ranges_out = nullptr, bool f8 = false) {
  int cur = 0;
  cudaError_t e;
  const int64_t n_tiles = (R + 127) / 128;
  const bool split = n_tiles < c->num_sms / 2;
  int n_ranges = 1;
  for (int l = 1; l < c->L; ++l) {
    const bool last = l == c->L - 1;
    const std::vector<int> &Kp = f8 ? c->Kp8 : c->Kp;
    const int ld_out = last ? 0 : Kp[l + 1];
    const bool tall = !split && c->NRs[l] > 0 && c->NRs[l] <= 256 &&
                      (n_tiles / 2) * ((c->H[l] + c->NRs[l] - 1) / c->NRs[l]) >= c->num_sms;
    const bool sp = (split || tall) && c->NRs[l] > 0;
    const int NR = sp ? c->NRs[l] : c->NR[l];
    const CUtensorMap &m0 = f8 ? (sp ? c->mBs0_8[l] : c->mB0_8[l]) : (sp ? c->mBs0[l] : c->mB0[l]);
    const CUtensorMap &m1 = f8 ? (sp ? c->mBs1_8[l] : c->mB1_8[l]) : (sp ? c->mBs1[l] : c->mB1[l]);
    const void *A = f8 ? (const void *)c->d_act8[cur] : (const void *)c->d_act[cur];
    void *next = f8 ? (void *)c->d_act8[cur ^ 1] : (void *)c->d_act[cur ^ 1];
    if ((e = dense_gemm(c, A, (int)R, Kp[l], m0, m1, c->H[l], NR, sp ? c->p0s[l] : c->p0[l],
                        sp ? c->p1s[l] : c->p1[l], last ? 1 : 0, c->d_bl[l], last ? c->d_wout : nullptr,
                        last ? nullptr : next, ld_out, last ? c->d_part : nullptr, s,
                        f8 ? c->d_scale8 + c->L + l : nullptr, tall)) != cudaSuccess)
      return e;
    if (last) n_ranges = (c->H[l] + NR - 1) / NR;
    cur ^= 1;
  }
  if (n_ranges_out) *n_ranges_out = n_ranges;
  if (!out) return cudaSuccess;
  dense_sum_kernel<<<grid_for(R, 256, c->num_sms), 256, 0, s>>>(c->d_part, R, n_ranges, b_out_dev, out);
  return cudaGetLastError();
}

A1Args a1_args(const nqs_ctx *c, const uint32_t *cfg, int64_t R, int mode, bool f8 = false) {
  A1Args a;
  a.cfg = cfg;
  a.z0 = c->d_z1;
  a.W1t = f8 ? c->d_W1t8 : c->d_W1t;
  a.bonds = c->d_bonds;
  a.act = f8 ? (void *)c->d_act8[0] : (void *)c->d_act[0];
  a.R = R;
  a.N = c->N;
  a.W = c->W;
  a.H0 = c->H[0];
  a.Kp1 = f8 ? c->Kp8[1] : c->Kp[1];
  a.nconn = c->ham_kind == NQS_HEISENBERG ? c->n_bonds : c->N;
  a.mode = mode;
  a.exchange = c->ham_kind == NQS_HEISENBERG;
  return a;
}

cudaError_t launch_propose(const nqs_ctx *c, const ProposeArgs &a, cudaStream_t s) {
  const dim3 grid = grid_for(a.C, 8, c->num_sms);
  const bool f8 = c->dtype == NQS_FP8E4M3;
  if (a.H0 <= 128)
    f8 ? dense_propose_kernel<2, uint8_t><<<grid, 256, 0, s>>>(a) : dense_propose_kernel<2, __nv_bfloat16><<<grid, 256, 0, s>>>(a);
  else if (a.H0 <= 256)
    f8 ? dense_propose_kernel<4, uint8_t><<<grid, 256, 0, s>>>(a) : dense_propose_kernel<4, __nv_bfloat16><<<grid, 256, 0, s>>>(a);
  else
    f8 ? dense_propose_kernel<8, uint8_t><<<grid, 256, 0, s>>>(a) : dense_propose_kernel<8, __nv_bfloat16><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// ====================================================================================
bool dense_setup(nqs_ctx *c, const nqs_model_desc *m, std::string *why) {
  if (m->n_layers < 2 || m->n_layers > 8 || !m->widths) {
    *why = "dense ansatz needs 2..8 hidden layers";
    return false;
  }
  if (c->dtype != NQS_BF16 && c->dtype != NQS_FP8E4M3) {
    *why = "the dense ansatz is built for BF16 and FP8 (E4M3) sampling copies";
    return false;
  }
  c->L = m->n_layers;
  c->H.assign(m->widths, m->widths + c->L);
  c->Kp.assign(c->L, 0);
  c->Kp8.assign(c->L, 0);
  int64_t P = 0;
  int fan = c->N;
  for (int l = 0; l < c->L; ++l) {
    if (c->H[l] < 16 || c->H[l] > 4096 || c->H[l] % 16) {
      *why = "dense widths must be multiples of 16 in [16, 4096]";
      return false;
    }
    if (l >= 1) {
      c->Kp[l] = ((c->H[l - 1] + 63) / 64) * 64;
      c->Kp8[l] = ((c->H[l - 1] + 127) / 128) * 128;
    }
    P += (int64_t)c->H[l] * fan + c->H[l];
    fan = c->H[l];
  }
  c->P = P + fan + 1;
  c->NR.assign(c->L, 0);
  c->p0.assign(c->L, 0);
  c->p1.assign(c->L, 0);
  c->NRs.assign(c->L, 0);
  c->p0s.assign(c->L, 0);
  c->p1s.assign(c->L, 0);
  for (int l = 1; l < c->L; ++l) {
    const int NR = std::min(c->H[l], 512);
    c->NR[l] = NR;
    c->p0[l] = std::min(256, 16 * ((NR + 31) / 32));
    c->p1[l] = NR - c->p0[l];
    const int NRs = 16 * ((NR / 2 + 15) / 16);  // split configuration: half the range
    if (NRs >= 32 && NRs < NR) {
      c->NRs[l] = NRs;
      c->p0s[l] = std::min(256, 16 * ((NRs + 31) / 32));
      c->p1s[l] = NRs - c->p0s[l];
    }
  }
  return true;
}

void dense_free(nqs_ctx *c) {
  void *ptrs[] = {c->d_W1t, c->d_b1,   c->d_wout, c->d_master,     c->d_act[0],     c->d_act[1], c->d_part,
                  c->d_out, c->d_z1,   c->d_lp,   c->d_prop,       c->d_thr,        c->d_grad_scratch,
                  c->d_force_part, c->d_z1b, c->d_W1d};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto p : c->d_Wl)
    if (p) cudaFree(p);
  for (auto p : c->d_bl)
    if (p) cudaFree(p);
  void *p8[] = {c->d_W1t8, c->d_scale8, c->d_wmax8, c->d_act8[0], c->d_act8[1]};
  for (void *p : p8)
    if (p) cudaFree(p);
  for (auto p : c->d_Wl8)
    if (p) cudaFree(p);
}

cudaError_t dense_alloc_rows(nqs_ctx *c, int64_t rows) {
  void *old[] = {c->d_act[0], c->d_act[1], c->d_part, c->d_out, c->d_z1, c->d_lp, c->d_prop, c->d_thr,
                 c->d_act8[0], c->d_act8[1], c->d_z1b};
  for (void *p : old)
    if (p) cudaFree(p);
  c->d_act8[0] = c->d_act8[1] = nullptr;
  c->d_z1b = nullptr;
  int maxKp = 64, max_ranges = 1;
  for (int l = 1; l < c->L; ++l) {
    maxKp = std::max(maxKp, c->Kp[l]);
    max_ranges = std::max(max_ranges, (c->H[l] + c->NR[l] - 1) / c->NR[l]);
    if (c->NRs[l]) max_ranges = std::max(max_ranges, (c->H[l] + c->NRs[l] - 1) / c->NRs[l]);
  }
  cudaError_t e;
  const size_t act = (size_t)rows * maxKp * sizeof(__nv_bfloat16);
  if ((e = cudaMalloc(&c->d_act[0], act)) || (e = cudaMalloc(&c->d_act[1], act)) ||
      (e = cudaMalloc(&c->d_part, (size_t)rows * max_ranges * 2 * 4)) || (e = cudaMalloc(&c->d_out, (size_t)rows * 4)) ||
      (e = cudaMalloc(&c->d_z1, (size_t)rows * c->H[0] * 4)) || (e = cudaMalloc(&c->d_lp, (size_t)rows * 4 + 16)) ||
      (e = cudaMalloc(&c->d_prop, (size_t)rows * 4)) || (e = cudaMalloc(&c->d_thr, (size_t)rows * 4)))
    return e;
  if ((e = cudaMemset(c->d_act[0], 0, act)) || (e = cudaMemset(c->d_act[1], 0, act))) return e;
  if (dense_fused_supported(c) && (e = cudaMalloc(&c->d_z1b, (size_t)rows * c->H[0] * 4)) != cudaSuccess) return e;
  if (c->dtype == NQS_FP8E4M3) {  // E4M3 rows; the padding columns stay zero
    int maxKp8 = 128;
    for (int l = 1; l < c->L; ++l) maxKp8 = std::max(maxKp8, c->Kp8[l]);
    const size_t act8 = (size_t)rows * maxKp8;
    if ((e = cudaMalloc(&c->d_act8[0], act8)) || (e = cudaMalloc(&c->d_act8[1], act8)) ||
        (e = cudaMemset(c->d_act8[0], 0, act8)) || (e = cudaMemset(c->d_act8[1], 0, act8)))
      return e;
  }
  c->max_rows = rows;
  return cudaSuccess;
}

cudaError_t dense_alloc_params(nqs_ctx *c) {
  cudaError_t e;
  if ((e = cudaMalloc(&c->d_W1t, (size_t)c->N * c->H[0] * 4)) || (e = cudaMalloc(&c->d_b1, (size_t)c->H[0] * 4)) ||
      (e = cudaMalloc(&c->d_wout, (size_t)c->H[c->L - 1] * 4 + 16)) ||
      (e = cudaMalloc(&c->d_master, (size_t)c->P * 4)))
    return e;
  if (c->ham_kind == NQS_HEISENBERG && c->n_bonds > 0 && dense_fused_supported(c) &&
      (e = cudaMalloc(&c->d_W1d, (size_t)c->n_bonds * c->H[0] * 4)))
    return e;
  c->d_Wl.assign(c->L, nullptr);
  c->d_bl.assign(c->L, nullptr);
  c->mB0.resize(c->L);
  c->mB1.resize(c->L);
  c->mBs0.resize(c->L);
  c->mBs1.resize(c->L);
  for (int l = 1; l < c->L; ++l) {
    const size_t wbytes = (size_t)c->H[l] * c->Kp[l] * sizeof(__nv_bfloat16);
    if ((e = cudaMalloc(&c->d_Wl[l], wbytes)) || (e = cudaMemset(c->d_Wl[l], 0, wbytes)) ||
        (e = cudaMalloc(&c->d_bl[l], (size_t)c->H[l] * 4)))
      return e;
    if (!make_tmap_bf16_2d(&c->mB0[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p0[l]) ||
        !make_tmap_bf16_2d(&c->mB1[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p1[l] ? c->p1[l] : c->p0[l]))
      return cudaErrorInvalidValue;
    if (c->NRs[l] &&
        (!make_tmap_bf16_2d(&c->mBs0[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p0s[l]) ||
         !make_tmap_bf16_2d(&c->mBs1[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p1s[l] ? c->p1s[l] : c->p0s[l])))
      return cudaErrorInvalidValue;
  }
  if (c->dtype == NQS_FP8E4M3) {
    c->d_Wl8.assign(c->L, nullptr);
    c->mB0_8.resize(c->L);
    c->mB1_8.resize(c->L);
    c->mBs0_8.resize(c->L);
    c->mBs1_8.resize(c->L);
    if ((e = cudaMalloc(&c->d_W1t8, (size_t)c->N * c->H[0] * 4)) || (e = cudaMalloc(&c->d_scale8, 2 * c->L * 4)) ||
        (e = cudaMalloc(&c->d_wmax8, c->L * 4)))
      return e;
    for (int l = 1; l < c->L; ++l) {
      const size_t wbytes = (size_t)c->H[l] * c->Kp8[l];
      if ((e = cudaMalloc(&c->d_Wl8[l], wbytes)) || (e = cudaMemset(c->d_Wl8[l], 0, wbytes))) return e;
      if (!make_tmap_u8_2d(&c->mB0_8[l], c->d_Wl8[l], c->H[l], c->Kp8[l], c->p0[l]) ||
          !make_tmap_u8_2d(&c->mB1_8[l], c->d_Wl8[l], c->H[l], c->Kp8[l], c->p1[l] ? c->p1[l] : c->p0[l]))
        return cudaErrorInvalidValue;
      if (c->NRs[l] &&
          (!make_tmap_u8_2d(&c->mBs0_8[l], c->d_Wl8[l], c->H[l], c->Kp8[l], c->p0s[l]) ||
           !make_tmap_u8_2d(&c->mBs1_8[l], c->d_Wl8[l], c->H[l], c->Kp8[l], c->p1s[l] ? c->p1s[l] : c->p0s[l])))
        return cudaErrorInvalidValue;
    }
  }
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(256, (int64_t)(256u << 20) / (c->P * 4)));
  c->grad_chunk = chunk;
  if ((e = cudaMalloc(&c->d_grad_scratch, (size_t)chunk * c->P * 4))) return e;
  if ((e = cudaMalloc(&c->d_force_part, (size_t)FORCE_SLICES * c->P * 8))) return e;
  return dense_alloc_rows(c, 262144);
}

cudaError_t dense_prepare(nqs_ctx *c, const double *params, cudaStream_t s) {
  const int H0 = c->H[0];
  dense_prepare_kernel<<<grid_for(c->P, 256, c->num_sms), 256, 0, s>>>(params, c->P, c->N, H0, c->d_master,
                                                                        c->d_W1t, c->d_b1, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t off = (int64_t)H0 * c->N + H0;
  for (int l = 1; l < c->L; ++l) {
    const int K = c->H[l - 1];
    const int64_t wout_off = c->P - 1 - c->H[c->L - 1];
    dense_prepare_layer_kernel<<<grid_for((int64_t)c->H[l] * K, 256, c->num_sms), 256, 0, s>>>(
        params, off, c->H[l], K, c->Kp[l], c->d_Wl[l], c->d_bl[l], params + wout_off, c->d_wout, l == c->L - 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    off += (int64_t)c->H[l] * K + c->H[l];
  }
  if (c->dtype == NQS_FP8E4M3) {  // the FP8 copy: per-layer scales, then E4M3 weights
    if ((e = cudaMemsetAsync(c->d_wmax8, 0, c->L * 4, s)) != cudaSuccess) return e;
    int64_t o = 0;
    for (int l = 0; l < c->L; ++l) {
      const int64_t cnt = (int64_t)c->H[l] * (l == 0 ? c->N : c->H[l - 1]);
      dense_wmax_kernel<<<grid_for(cnt, 256, c->num_sms), 256, 0, s>>>(params, o, cnt, c->d_wmax8 + l);
      o += cnt + c->H[l];
    }
    dense_scale8_kernel<<<1, 32, 0, s>>>(c->d_wmax8, c->L, c->d_scale8);
    dense_prepare8_l0_kernel<<<grid_for((int64_t)H0 * c->N, 256, c->num_sms), 256, 0, s>>>(params, c->N, H0, c->d_scale8,
                                                                                         c->d_W1t8);
    o = (int64_t)H0 * c->N + H0;
    for (int l = 1; l < c->L; ++l) {
      const int K = c->H[l - 1];
      dense_prepare8_layer_kernel<<<grid_for((int64_t)c->H[l] * K, 256, c->num_sms), 256, 0, s>>>(
          params, o, c->H[l], K, c->Kp8[l], c->d_scale8 + l, c->d_Wl8[l]);
      o += (int64_t)c->H[l] * K + c->H[l];
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c->d_W1d && (e = dense_fused_prepare(c, s)) != cudaSuccess) return e;
  // b_out (= master[P - 1]) is kept on the device right after w_out
  return cudaMemcpyAsync(c->d_wout + c->H[c->L - 1], c->d_master + (c->P - 1), sizeof(float), cudaMemcpyDeviceToDevice,
                         s);
}

// log psi of rows through the sampling copy (BF16, or the FP8 copy of an FP8 context)
static cudaError_t logpsi_rows(const nqs_ctx *c, const uint32_t *cfg, int64_t R, float *out, cudaStream_t s) {
  const bool f8 = c->dtype == NQS_FP8E4M3;
  const float *b_out = c->d_wout + c->H[c->L - 1];
  dense_z0_kernel<<<z0_grid(R, c->H[0], c->num_sms), Z0_COLS, 0, s>>>(cfg, R, f8 ? c->d_W1t8 : c->d_W1t, c->d_b1, c->N,
                                                                     c->W, c->H[0], c->d_z1);
  const A1Args a = a1_args(c, cfg, R, 0, f8);
  if (f8) dense_a1_kernel<uint8_t><<<grid_for(R, 8, c->num_sms), 256, 0, s>>>(a);
  else dense_a1_kernel<__nv_bfloat16><<<grid_for(R, 8, c->num_sms), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return run_chain(c, R, out, b_out, s, nullptr, f8);
}

cudaError_t dense_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  cudaError_t e;
  for (int64_t x0 = 0; x0 < n; x0 += c->max_rows) {
    const int64_t R = std::min<int64_t>(c->max_rows, n - x0);
    if ((e = logpsi_rows(c, cfg + x0 * c->W, R, out + x0, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t dense_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s) {
  const bool exch = c->ham_kind == NQS_HEISENBERG;
  const int nconn = exch ? c->n_bonds : c->N;
  const int64_t per = 1 + nconn;
  const int64_t chunk = std::max<int64_t>(1, c->max_rows / per);
  const float *b_out = c->d_wout + c->H[c->L - 1];
  cudaError_t e;
  for (int64_t x0 = 0; x0 < n; x0 += chunk) {
    const int64_t ns = std::min<int64_t>(chunk, n - x0);
    const uint32_t *cx = cfg + x0 * c->W;
    dense_z0_kernel<<<z0_grid(ns, c->H[0], c->num_sms), Z0_COLS, 0, s>>>(cx, ns, c->d_W1t, c->d_b1, c->N, c->W, c->H[0],
                                                                c->d_z1);
    A1Args a = a1_args(c, cx, ns * per, 1);  // the BF16 copy (also for an FP8 context)
    dense_a1_kernel<__nv_bfloat16><<<grid_for(ns * per, 8, c->num_sms), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = run_chain(c, ns * per, c->d_out, b_out, s)) != cudaSuccess) return e;
    dense_eloc_combine_kernel<<<grid_for(ns, 8, c->num_sms), 256, 0, s>>>(
        cx, ns, c->d_out, c->d_bonds, c->d_bondJ, c->n_bonds, c->N, c->W, c->Lx, exch, c->marshall, (float)c->J1,
        (float)c->h, eloc + x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t dense_sweep(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int burn_in, uint64_t seed,
                        uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc, uint32_t *acc_bits,
                        float *delta, cudaStream_t s) {
  if (C > c->max_rows) return cudaErrorInvalidValue;
  const float *b_out = c->d_wout + c->H[c->L - 1];
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  cudaError_t e;
  const bool f8 = c->dtype == NQS_FP8E4M3;  // the sampler runs on the FP8 copy
  auto refresh = [&]() -> cudaError_t { return logpsi_rows(c, state, C, c->d_lp, s); };  // z0, log psi from scratch
  if ((e = refresh()) != cudaSuccess) return e;
  if (c->dense_fused && c->d_z1b && dense_fused_supported(c)) {
    // persistent fused sampler, one launch per stretch of sweeps between two refreshes (the
    // refresh points of the multi-launch path below: after sweep t when (t + 1) % refresh == 0)
    for (int t = 0; t < n_sweeps;) {
      const int next = (t / c->refresh + 1) * c->refresh;
      const int t1 = next < n_sweeps ? next : n_sweeps;
      if ((e = dense_fused_sweeps(c, state, C, n_sweeps, t, t1, burn_in, seed, sweep_offset, samples, logpsi, n_acc,
                                  acc_bits, delta, t > 0, s)) != cudaSuccess)
        return e;
      if (t1 < n_sweeps && (e = refresh()) != cudaSuccess) return e;
      t = t1;
    }
    return cudaSuccess;
  }
  ProposeArgs a;
  a.state = state;
  a.z0 = c->d_z1;
  a.W1t = f8 ? c->d_W1t8 : c->d_W1t;
  a.bonds = c->d_bonds;
  a.prop = c->d_prop;
  a.thr = c->d_thr;
  a.lp = c->d_lp;
  a.act = f8 ? (void *)c->d_act8[0] : (void *)c->d_act[0];
  a.part = c->d_part;
  a.b_out = b_out;
  a.n_ranges = 1;
  a.n_acc = n_acc;
  a.acc_bits = acc_bits;
  a.delta = delta;
  a.samples = samples;
  a.logpsi = logpsi;
  a.C = C;
  a.N = c->N;
  a.W = c->W;
  a.H0 = c->H[0];
  a.Kp1 = f8 ? c->Kp8[1] : c->Kp[1];
  a.exchange = c->ham_kind == NQS_HEISENBERG;
  a.n_moves = a.exchange ? c->n_bonds : c->N;
  a.n_sweeps = n_sweeps;
  a.decide = 0;
  a.first = 1;
  a.t_prev = a.p_prev = 0;
  a.emit_row = -1;
  a.k0 = k0;
  a.k1 = k1;
  for (int t = 0; t < n_sweeps; ++t) {
    a.sweep_id = sweep_offset + (uint32_t)t;
    for (int p = 0; p < c->N; ++p) {
      a.propose = 1;
      a.p = p;
      if ((e = launch_propose(c, a, s)) != cudaSuccess) return e;
      if (a.decide) a.first = 0;
      a.emit_row = -1;
      if ((e = run_chain(c, C, nullptr, b_out, s, &a.n_ranges, f8)) != cudaSuccess) return e;
      a.decide = 1;
      a.t_prev = t;
      a.p_prev = p;
    }
    if (t >= burn_in) a.emit_row = t - burn_in;
    if ((t + 1) % c->refresh == 0 && t + 1 < n_sweeps) {  // decide, apply, emit, then rebuild the caches
      a.propose = 0;
      if ((e = launch_propose(c, a, s)) != cudaSuccess) return e;
      a.decide = 0;
      a.first = 0;
      a.emit_row = -1;
      if ((e = refresh()) != cudaSuccess) return e;
    }
  }
  a.propose = 0;  // closing pass: last decision and last sample
  return launch_propose(c, a, s);
}

cudaError_t force_rows(const nqs_ctx *c, const float *O, int64_t rows, const float *eloc, const double *stats,
                              int64_t n_total, bool share, int accumulate, double *force, cudaStream_t s) {
  double *part = reinterpret_cast<double *>(c->d_force_part);
  dense_force_part_kernel<<<dim3((unsigned)((c->P + 255) / 256), FORCE_SLICES), 256, 0, s>>>(O, rows, c->P, eloc, stats,
                                                                                             part);
  dense_force_sum_kernel<<<grid_for(c->P, 256, c->num_sms), 256, 0, s>>>(part, c->P, n_total, share ? stats + 4 : nullptr,
                                                                        accumulate, force);
  return cudaGetLastError();
}

cudaError_t dense_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                              const double *stats, double *force, cudaStream_t s, bool share) {
  GradArgs g;
  g.cfg = cfg;
  g.master = c->d_master;
  g.P = c->P;
  g.N = c->N;
  g.W = c->W;
  g.L = c->L;
  int64_t off = 0;
  int fan = c->N;
  size_t shm = (size_t)c->N;
  for (int l = 0; l < c->L; ++l) {
    g.H[l] = c->H[l];
    g.offW[l] = off;
    off += (int64_t)c->H[l] * fan;
    g.offb[l] = off;
    off += c->H[l];
    fan = c->H[l];
    shm += 2 * (size_t)c->H[l];
  }
  g.offw_out = off;
  shm *= sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(dense_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  const int64_t chunk = O ? n : c->grad_chunk;
  for (int64_t x0 = 0; x0 < n; x0 += chunk) {
    const int64_t rows = std::min<int64_t>(chunk, n - x0);
    g.cfg = cfg + x0 * c->W;
    g.O = O ? O + x0 * c->P : c->d_grad_scratch;
    g.n = rows;
    dense_grad_kernel<<<(unsigned)std::min<int64_t>(rows, (int64_t)c->num_sms * 8), 256, shm, s>>>(g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (force && !O && (e = force_rows(c, g.O, rows, eloc + x0, stats, n, share, x0 > 0, force, s)) != cudaSuccess)
      return e;
  }
  if (force && O) return force_rows(c, O, n, eloc, stats, n, share, 0, force, s);
  return cudaSuccess;
}

}  // namespace nqs
