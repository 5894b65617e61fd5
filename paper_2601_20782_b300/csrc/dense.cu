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

// ------------------------------------------------------------------------------------
// z0 = W_0 s + b_0 for n configurations (one warp per configuration, FP32)
__global__ void dense_z0_kernel(const uint32_t *__restrict__ cfg, int64_t n, const float *__restrict__ W1t,
                                const float *__restrict__ b1, int N, int W, int H0, float *z0) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = gw; x < n; x += nw) {
    for (int j0 = 0; j0 < H0; j0 += 32 * 4) {
      float acc[4];
      for (int u = 0; u < 4; ++u) acc[u] = (j0 + lane + 32 * u < H0) ? b1[j0 + lane + 32 * u] : 0.f;
      for (int w = 0; w < W; ++w) {
        const uint32_t word = cfg[x * W + w];
        const int nb = min(32, N - 32 * w);
        for (int bit = 0; bit < nb; ++bit) {
          const float s = ((word >> bit) & 1u) ? 1.f : -1.f;
          const float *row = W1t + (int64_t)(32 * w + bit) * H0 + j0 + lane;
          for (int u = 0; u < 4; ++u)
            if (j0 + lane + 32 * u < H0) acc[u] = fmaf(s, row[32 * u], acc[u]);
        }
      }
      for (int u = 0; u < 4; ++u)
        if (j0 + lane + 32 * u < H0) z0[x * H0 + j0 + lane + 32 * u] = acc[u];
    }
  }
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
// exchange for Heisenberg).  mode 2: sampler rows r = chain, move prop[r] (< 0: identity).
struct A1Args {
  const uint32_t *cfg;
  const float *z0;
  const float *W1t;
  const int2 *bonds;
  const int32_t *prop;
  __nv_bfloat16 *act;
  int64_t R;
  int N, W, H0, Kp1, nconn, mode, exchange;
};

__device__ __forceinline__ bool row_move(const A1Args &a, int64_t r, int64_t *src, Move *mv) {
  if (a.mode == 0) {
    *src = r;
    return false;
  }
  int m;
  if (a.mode == 1) {
    *src = r / (1 + a.nconn);
    m = (int)(r % (1 + a.nconn)) - 1;
  } else {
    *src = r;
    m = a.prop[r];
  }
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
    __nv_bfloat16 *out = a.act + r * a.Kp1;
    for (int k = 2 * lane; k < a.H0; k += 64) {  // two units per lane per step (H0 even)
      float z0v = zr[k], z1v = zr[k + 1];
      if (moved) {
        // flip: s_i -> -s_i; exchange: s_i -> -s_i and s_j = -s_i -> s_i
        const float d0 = mv.j < 0 ? wi[k] : wi[k] - wj[k];
        const float d1 = mv.j < 0 ? wi[k + 1] : wi[k + 1] - wj[k + 1];
        z0v = fmaf(-2.f * si, d0, z0v);
        z1v = fmaf(-2.f * si, d1, z1v);
      }
      *reinterpret_cast<__nv_bfloat162 *>(out + k) = __floats2bfloat162_rn(log_cosh_f(z0v), log_cosh_f(z1v));
    }
  }
}

// log psi of the rows: sum of the last layer's range partials + b_out
__global__ void dense_sum_kernel(const float *part, int64_t R, int n_ranges, const float *b_out, float *out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    float s = b_out[0];
    for (int q = 0; q < n_ranges; ++q) s += part[r * n_ranges + q];
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
// Hamiltonian for Heisenberg, a site for TFIM), u = (w' >> 8) 2^-24.
__global__ void dense_propose_kernel(const uint32_t *__restrict__ state, int64_t C, int W, int exchange, int n_moves,
                                     const int2 *bonds, int p, uint32_t sweep_id, uint32_t k0, uint32_t k1,
                                     int32_t *prop, float *thr) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(p / 2), sweep_id, (uint32_t)c, TAG_SWEEP), k0, k1);
    const uint32_t wm = (p & 1) ? w.z : w.x, wu = (p & 1) ? w.w : w.y;
    const int m = (int)index_from_word(wm, (uint32_t)n_moves);
    const uint32_t k = wu >> 8;
    thr[c] = k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
    int mv = m;
    if (exchange) {
      const int2 b = bonds[m];
      if (spin_of(state, W, c, b.x) == spin_of(state, W, c, b.y)) mv = -1;  // identity: always accepted
    }
    prop[c] = mv;
  }
}

struct AcceptArgs {
  uint32_t *state;
  float *z0;
  float *lp;
  const float *lp_new;
  const int32_t *prop;
  const float *thr;
  const float *W1t;
  const int2 *bonds;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
  uint32_t *samples;
  float *logpsi;
  int64_t C;
  int N, W, H0, exchange, p, t, n_sweeps, emit_row;  // emit_row < 0: no sample this step
  int first;  // reset n_acc
};

// One warp per chain: decision u < exp(2 (log psi(y) - log psi(x))), then on accept the
// FP32 z0 update (one or two columns of W_0), the spin move and the cached log psi.
__global__ void dense_accept_kernel(const AcceptArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < a.C; c += nw) {
    const int m = a.prop[c];
    bool acc;
    float dlt = 0.f;
    if (m < 0) {
      acc = true;
    } else {
      dlt = a.lp_new[c] - a.lp[c];
      acc = 2.f * dlt > a.thr[c];
    }
    if (acc && m >= 0) {
      int i, j;
      if (a.exchange) {
        const int2 b = a.bonds[m];
        i = b.x;
        j = b.y;
      } else {
        i = m;
        j = -1;
      }
      const float si = (float)spin_of(a.state, a.W, c, i);
      float *z = a.z0 + c * a.H0;
      const float *wi = a.W1t + (int64_t)i * a.H0;
      const float *wj = a.W1t + (int64_t)(j < 0 ? 0 : j) * a.H0;
      for (int k = lane; k < a.H0; k += 32) z[k] = fmaf(-2.f * si, j < 0 ? wi[k] : wi[k] - wj[k], z[k]);
      __syncwarp();
      if (lane == 0) {
        a.state[c * a.W + (i >> 5)] ^= 1u << (i & 31);
        if (j >= 0) a.state[c * a.W + (j >> 5)] ^= 1u << (j & 31);
        a.lp[c] = a.lp_new[c];
      }
    }
    if (lane == 0) {
      if (a.n_acc) a.n_acc[c] = (a.first ? 0 : a.n_acc[c]) + (acc ? 1 : 0);
      if (a.acc_bits) {
        const int64_t wi = ((int64_t)c * a.n_sweeps + a.t) * a.W + (a.p >> 5);
        const uint32_t bit = 1u << (a.p & 31);
        a.acc_bits[wi] = ((a.p & 31) == 0 ? 0u : a.acc_bits[wi]) | (acc ? bit : 0u);
      }
      if (a.delta) a.delta[((int64_t)c * a.n_sweeps + a.t) * a.N + a.p] = dlt;
    }
    __syncwarp();
    if (a.emit_row >= 0) {
      const int64_t row = (int64_t)a.emit_row * a.C + c;
      if (a.samples)
        for (int w = lane; w < a.W; w += 32) a.samples[row * a.W + w] = a.state[c * a.W + w];
      if (lane == 0 && a.logpsi) a.logpsi[row] = a.lp[c];
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
      // O_{W_l} = delta_l a_{l-1}^T and O_{b_l} = delta_l
      for (int64_t q = tid; q < (int64_t)Hl * Kl; q += blockDim.x) row[g.offW[l] + q] = dl[q / Kl] * ain[q % Kl];
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

// F_k (+)= sum_x O[x][k] (eloc[x] - E) / n over a chunk of rows (FP64, fixed order)
__global__ void dense_force_kernel(const float *O, int64_t rows, int64_t P, const float *eloc, const double *stats,
                                   int64_t n_total, int accumulate, double *force) {
  const double E = stats[0];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t x = 0; x < rows; ++x) s += (double)O[x * P + k] * ((double)eloc[x] - E);
    s /= (double)n_total;
    force[k] = accumulate ? force[k] + s : s;
  }
}

int grid_for(int64_t work, int per_block, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, (int64_t)num_sms * 16));
}

// GEMM chain over layers 1..L-1 for R rows whose layer-0 output is in act[0]; writes log psi.
cudaError_t run_chain(const nqs_ctx *c, int64_t R, float *out, const float *b_out_dev, cudaStream_t s) {
  int cur = 0;
  cudaError_t e;
  for (int l = 1; l < c->L; ++l) {
    const bool last = l == c->L - 1;
    const int ld_out = last ? 0 : c->Kp[l + 1];
    if ((e = dense_gemm(c, c->d_act[cur], (int)R, c->Kp[l], c->mB0[l], c->mB1[l], c->H[l], c->NR[l], c->p0[l],
                        c->p1[l], last ? 1 : 0, c->d_bl[l], last ? c->d_wout : nullptr,
                        last ? nullptr : c->d_act[cur ^ 1], ld_out, last ? c->d_part : nullptr, s)) != cudaSuccess)
      return e;
    cur ^= 1;
  }
  const int n_ranges = (c->H[c->L - 1] + c->NR[c->L - 1] - 1) / c->NR[c->L - 1];
  dense_sum_kernel<<<grid_for(R, 256, c->num_sms), 256, 0, s>>>(c->d_part, R, n_ranges, b_out_dev, out);
  return cudaGetLastError();
}

A1Args a1_args(const nqs_ctx *c, const uint32_t *cfg, int64_t R, int mode) {
  A1Args a;
  a.cfg = cfg;
  a.z0 = c->d_z1;
  a.W1t = c->d_W1t;
  a.bonds = c->d_bonds;
  a.prop = c->d_prop;
  a.act = c->d_act[0];
  a.R = R;
  a.N = c->N;
  a.W = c->W;
  a.H0 = c->H[0];
  a.Kp1 = c->Kp[1];
  a.nconn = c->ham_kind == NQS_HEISENBERG ? c->n_bonds : c->N;
  a.mode = mode;
  a.exchange = c->ham_kind == NQS_HEISENBERG;
  return a;
}

}  // namespace

// ====================================================================================
bool dense_setup(nqs_ctx *c, const nqs_model_desc *m, std::string *why) {
  if (m->n_layers < 2 || m->n_layers > 8 || !m->widths) {
    *why = "dense ansatz needs 2..8 hidden layers";
    return false;
  }
  if (c->dtype != NQS_BF16) {
    *why = "the dense ansatz is built for a BF16 sampling copy";
    return false;
  }
  c->L = m->n_layers;
  c->H.assign(m->widths, m->widths + c->L);
  c->Kp.assign(c->L, 0);
  int64_t P = 0;
  int fan = c->N;
  for (int l = 0; l < c->L; ++l) {
    if (c->H[l] < 16 || c->H[l] > 4096 || c->H[l] % 16) {
      *why = "dense widths must be multiples of 16 in [16, 4096]";
      return false;
    }
    if (l >= 1) c->Kp[l] = ((c->H[l - 1] + 63) / 64) * 64;
    P += (int64_t)c->H[l] * fan + c->H[l];
    fan = c->H[l];
  }
  c->P = P + fan + 1;
  c->NR.assign(c->L, 0);
  c->p0.assign(c->L, 0);
  c->p1.assign(c->L, 0);
  for (int l = 1; l < c->L; ++l) {
    const int NR = std::min(c->H[l], 512);
    c->NR[l] = NR;
    c->p0[l] = std::min(256, 16 * ((NR + 31) / 32));
    c->p1[l] = NR - c->p0[l];
  }
  return true;
}

void dense_free(nqs_ctx *c) {
  void *ptrs[] = {c->d_W1t, c->d_b1, c->d_wout, c->d_master, c->d_act[0], c->d_act[1], c->d_part, c->d_out,
                  c->d_z1,  c->d_lp, c->d_prop, c->d_thr,    c->d_grad_scratch};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto p : c->d_Wl)
    if (p) cudaFree(p);
  for (auto p : c->d_bl)
    if (p) cudaFree(p);
}

cudaError_t dense_alloc_rows(nqs_ctx *c, int64_t rows) {
  void *old[] = {c->d_act[0], c->d_act[1], c->d_part, c->d_out, c->d_z1, c->d_lp, c->d_prop, c->d_thr};
  for (void *p : old)
    if (p) cudaFree(p);
  int maxKp = 64, max_ranges = 1;
  for (int l = 1; l < c->L; ++l) {
    maxKp = std::max(maxKp, c->Kp[l]);
    max_ranges = std::max(max_ranges, (c->H[l] + c->NR[l] - 1) / c->NR[l]);
  }
  cudaError_t e;
  const size_t act = (size_t)rows * maxKp * sizeof(__nv_bfloat16);
  if ((e = cudaMalloc(&c->d_act[0], act)) || (e = cudaMalloc(&c->d_act[1], act)) ||
      (e = cudaMalloc(&c->d_part, (size_t)rows * max_ranges * 4)) || (e = cudaMalloc(&c->d_out, (size_t)rows * 4)) ||
      (e = cudaMalloc(&c->d_z1, (size_t)rows * c->H[0] * 4)) || (e = cudaMalloc(&c->d_lp, (size_t)rows * 4 + 16)) ||
      (e = cudaMalloc(&c->d_prop, (size_t)rows * 4)) || (e = cudaMalloc(&c->d_thr, (size_t)rows * 4)))
    return e;
  if ((e = cudaMemset(c->d_act[0], 0, act)) || (e = cudaMemset(c->d_act[1], 0, act))) return e;
  c->max_rows = rows;
  return cudaSuccess;
}

cudaError_t dense_alloc_params(nqs_ctx *c) {
  cudaError_t e;
  if ((e = cudaMalloc(&c->d_W1t, (size_t)c->N * c->H[0] * 4)) || (e = cudaMalloc(&c->d_b1, (size_t)c->H[0] * 4)) ||
      (e = cudaMalloc(&c->d_wout, (size_t)c->H[c->L - 1] * 4 + 16)) ||
      (e = cudaMalloc(&c->d_master, (size_t)c->P * 4)))
    return e;
  c->d_Wl.assign(c->L, nullptr);
  c->d_bl.assign(c->L, nullptr);
  c->mB0.resize(c->L);
  c->mB1.resize(c->L);
  for (int l = 1; l < c->L; ++l) {
    const size_t wbytes = (size_t)c->H[l] * c->Kp[l] * sizeof(__nv_bfloat16);
    if ((e = cudaMalloc(&c->d_Wl[l], wbytes)) || (e = cudaMemset(c->d_Wl[l], 0, wbytes)) ||
        (e = cudaMalloc(&c->d_bl[l], (size_t)c->H[l] * 4)))
      return e;
    if (!make_tmap_bf16_2d(&c->mB0[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p0[l]) ||
        !make_tmap_bf16_2d(&c->mB1[l], c->d_Wl[l], c->H[l], c->Kp[l], c->p1[l] ? c->p1[l] : c->p0[l]))
      return cudaErrorInvalidValue;
  }
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(256, (int64_t)(256u << 20) / (c->P * 4)));
  c->grad_chunk = chunk;
  if ((e = cudaMalloc(&c->d_grad_scratch, (size_t)chunk * c->P * 4))) return e;
  return dense_alloc_rows(c, 65536);
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
  // b_out (= master[P - 1]) is kept on the device right after w_out
  return cudaMemcpyAsync(c->d_wout + c->H[c->L - 1], c->d_master + (c->P - 1), sizeof(float), cudaMemcpyDeviceToDevice,
                         s);
}

cudaError_t dense_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  cudaError_t e;
  const float *b_out = c->d_wout + c->H[c->L - 1];
  for (int64_t x0 = 0; x0 < n; x0 += c->max_rows) {
    const int64_t R = std::min<int64_t>(c->max_rows, n - x0);
    dense_z0_kernel<<<grid_for(R, 8, c->num_sms), 256, 0, s>>>(cfg + x0 * c->W, R, c->d_W1t, c->d_b1, c->N, c->W,
                                                               c->H[0], c->d_z1);
    A1Args a = a1_args(c, cfg + x0 * c->W, R, 0);
    dense_a1_kernel<<<grid_for(R, 8, c->num_sms), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = run_chain(c, R, out + x0, b_out, s)) != cudaSuccess) return e;
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
    dense_z0_kernel<<<grid_for(ns, 8, c->num_sms), 256, 0, s>>>(cx, ns, c->d_W1t, c->d_b1, c->N, c->W, c->H[0],
                                                                c->d_z1);
    A1Args a = a1_args(c, cx, ns * per, 1);
    dense_a1_kernel<<<grid_for(ns * per, 8, c->num_sms), 256, 0, s>>>(a);
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
  const bool exch = c->ham_kind == NQS_HEISENBERG;
  const int n_moves = exch ? c->n_bonds : c->N;
  const float *b_out = c->d_wout + c->H[c->L - 1];
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  cudaError_t e;
  auto refresh = [&]() -> cudaError_t {  // z0 and log psi of the chains from scratch
    dense_z0_kernel<<<grid_for(C, 8, c->num_sms), 256, 0, s>>>(state, C, c->d_W1t, c->d_b1, c->N, c->W, c->H[0],
                                                               c->d_z1);
    A1Args a = a1_args(c, state, C, 0);
    dense_a1_kernel<<<grid_for(C, 8, c->num_sms), 256, 0, s>>>(a);
    cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return e2;
    return run_chain(c, C, c->d_lp, b_out, s);
  };
  if ((e = refresh()) != cudaSuccess) return e;
  for (int t = 0; t < n_sweeps; ++t) {
    const uint32_t sweep_id = sweep_offset + (uint32_t)t;
    for (int p = 0; p < c->N; ++p) {
      dense_propose_kernel<<<grid_for(C, 256, c->num_sms), 256, 0, s>>>(state, C, c->W, exch, n_moves, c->d_bonds, p,
                                                                        sweep_id, k0, k1, c->d_prop, c->d_thr);
      A1Args a = a1_args(c, state, C, 2);
      dense_a1_kernel<<<grid_for(C, 8, c->num_sms), 256, 0, s>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = run_chain(c, C, c->d_out, b_out, s)) != cudaSuccess) return e;
      AcceptArgs ac;
      ac.state = state;
      ac.z0 = c->d_z1;
      ac.lp = c->d_lp;
      ac.lp_new = c->d_out;
      ac.prop = c->d_prop;
      ac.thr = c->d_thr;
      ac.W1t = c->d_W1t;
      ac.bonds = c->d_bonds;
      ac.n_acc = n_acc;
      ac.acc_bits = acc_bits;
      ac.delta = delta;
      ac.samples = samples;
      ac.logpsi = logpsi;
      ac.C = C;
      ac.N = c->N;
      ac.W = c->W;
      ac.H0 = c->H[0];
      ac.exchange = exch;
      ac.p = p;
      ac.t = t;
      ac.n_sweeps = n_sweeps;
      ac.emit_row = (p == c->N - 1 && t >= burn_in) ? t - burn_in : -1;
      ac.first = (t == 0 && p == 0);
      dense_accept_kernel<<<grid_for(C, 8, c->num_sms), 256, 0, s>>>(ac);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((t + 1) % c->refresh == 0 && t + 1 < n_sweeps && (e = refresh()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t dense_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                              const double *stats, double *force, cudaStream_t s) {
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
    if (force && !O) {
      dense_force_kernel<<<grid_for(c->P, 256, c->num_sms), 256, 0, s>>>(g.O, rows, c->P, eloc + x0, stats, n,
                                                                         x0 > 0, force);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  if (force && O) {
    dense_force_kernel<<<grid_for(c->P, 256, c->num_sms), 256, 0, s>>>(O, n, c->P, eloc, stats, n, 0, force);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace nqs
