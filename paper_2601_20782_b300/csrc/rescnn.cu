// Residual convolutional ansatz (App. H, "ResCNN") on a periodic Lx x Ly lattice:
//   h(0) = Conv(s),  h(l+1) = h(l) + Conv[phi(Conv(phi(LN(h(l)))))],  log psi = sum LN(h(B)),
// 3 x 3 periodic cross-correlations with a bias, F = 16 filters, LN over the 16 channels of a
// site (eps 1e-6, scale and shift), phi the tanh form of GELU.
//
// This file holds the FP32 sampling copy on the CUDA cores: one thread per (configuration,
// site) row keeps that row's residual stream h in registers; the input of each convolution
// sits in shared memory as FP32 rows, and a thread reads its nine periodic neighbour rows
// (computed from its site's coordinates) for each of the 16 x 16 x 9 multiply-adds.  The same forward pass serves three modes: log psi of given
// configurations, the N + 1 configurations of each sample's TFIM local energy, and the
// Metropolis sweep (a CTA owns a group of chains for all its sweeps; each step proposes one
// flip per chain, evaluates the proposed configurations and decides).
//
// Kernel order of the FP32 parameter copy (floats; tap = 3 dy + dx):
//   k0 [tap][F] | b0 [F] | per block: gamma [F] | beta [F] | K1 [tap][ci][co] | b1 [F] |
//   K2 [tap][ci][co] | b2 [F] | final gamma [F] | final beta [F]
// i.e. the master order with each kernel K[co][ci][dy][dx] stored as [tap][ci][co].
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "rescnn.cuh"

namespace nqs {
namespace cnn {
namespace {

// Master -> kernel order (F = 16).  One thread per element of the kernel-order array.
__global__ void rescnn_prepare_f32_kernel(const double *master, int n_blocks, float *cw) {
  const int P = n_params(n_blocks);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    int src = k;
    if (k < 9 * CF) {  // k0[tap][co] <- K0[co][0][tap]
      const int tap = k / CF, co = k % CF;
      src = co * 9 + tap;
    } else if (k >= 10 * CF && k < 10 * CF + n_blocks * BLOCK_FLOATS) {
      const int base = 10 * CF + ((k - 10 * CF) / BLOCK_FLOATS) * BLOCK_FLOATS;
      const int r = k - base;
      int kb = -1;
      if (r >= OFF_K1 && r < OFF_K1 + 9 * CF * CF) kb = OFF_K1;
      if (r >= OFF_K2 && r < OFF_K2 + 9 * CF * CF) kb = OFF_K2;
      if (kb >= 0) {  // [tap][ci][co] <- [co][ci][tap]
        const int e = r - kb, tap = e / (CF * CF), ci = (e / CF) % CF, co = e % CF;
        src = base + kb + (co * CF + ci) * 9 + tap;
      }
    }
    cw[k] = (float)master[src];
  }
}

__device__ __forceinline__ float gelu_f32(float y) {  // tanh form, accurate tanhf
  return 0.5f * y * (1.f + tanhf(GELU_C * fmaf(0.044715f * y * y, y, y)));
}

// LN over the 16 channels of one site: (v - mean) / sqrt(var + eps) * gamma + beta
__device__ __forceinline__ void layer_norm16(const float (&v)[CF], const float *g, const float *be,
                                             float (&y)[CF]) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) m += v[c];
  m *= 1.f / CF;
  float var = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) {
    const float d = v[c] - m;
    var = fmaf(d, d, var);
  }
  const float rs = rsqrtf(fmaf(var, 1.f / CF, LN_EPS));
#pragma unroll
  for (int c = 0; c < CF; ++c) y[c] = fmaf((v[c] - m) * rs, g[c], be[c]);
}

// Row of the periodic neighbour (dy, dx) of site (x, y) in a configuration whose rows start at row0.
struct RowPos {
  int row0, x, y, Lx, Ly;
  __device__ __forceinline__ int nb(int tap) const {
    const int dy = tap / 3, dx = tap - 3 * dy;
    int xx = x + dx - 1, yy = y + dy - 1;
    xx += xx < 0 ? Lx : (xx >= Lx ? -Lx : 0);
    yy += yy < 0 ? Ly : (yy >= Ly ? -Ly : 0);
    return row0 + xx + Lx * yy;
  }
};

// z = bias + sum_tap sum_ci K[tap][ci][co] act[nb(tap)][ci] (act rows of 16 FP32 in shared memory)
__device__ __forceinline__ void conv_row_f32(const float *K, const float *bias, const float *act, const RowPos &rp,
                                             float (&z)[CF]) {
#pragma unroll
  for (int c = 0; c < CF; ++c) z[c] = bias[c];
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const float4 *a4 = reinterpret_cast<const float4 *>(act + rp.nb(tap) * CF);
    float a[CF];
#pragma unroll
    for (int q = 0; q < CF / 4; ++q) {
      const float4 v = a4[q];
      a[4 * q] = v.x;
      a[4 * q + 1] = v.y;
      a[4 * q + 2] = v.z;
      a[4 * q + 3] = v.w;
    }
    const float4 *k4 = reinterpret_cast<const float4 *>(K + tap * CF * CF);
#pragma unroll
    for (int ci = 0; ci < CF; ++ci) {
#pragma unroll
      for (int q = 0; q < CF / 4; ++q) {
        const float4 w = k4[ci * (CF / 4) + q];
        z[4 * q] = fmaf(w.x, a[ci], z[4 * q]);
        z[4 * q + 1] = fmaf(w.y, a[ci], z[4 * q + 1]);
        z[4 * q + 2] = fmaf(w.z, a[ci], z[4 * q + 2]);
        z[4 * q + 3] = fmaf(w.w, a[ci], z[4 * q + 3]);
      }
    }
  }
}

__device__ __forceinline__ void store_row(float *act, int r, const float (&v)[CF]) {
  float4 *d = reinterpret_cast<float4 *>(act + r * CF);
#pragma unroll
  for (int q = 0; q < CF / 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Shared-memory state of one CTA's group of G configurations (G N <= blockDim.x rows).
struct GroupSmem {
  float *w;       // [P] kernel-order parameters
  float *act;     // [blockDim.x][16] convolution input rows
  float *spin;    // [G][N] +-1 of the group's configurations
  float *rowsum;  // [blockDim.x] per-row sum of the final LN
  int *flip;      // [G] site flipped for the evaluated configuration (-1: none)
  float *lp;      // [G] log psi of the evaluated configurations
};

// log psi of the group's G configurations (spin with flip applied) into sm.lp.  Every thread
// of the CTA calls it (it synchronises); row r = g N + site belongs to thread r.
__device__ void forward_group_f32(const GroupSmem &sm, int G, int N, int Lx, int Ly, int n_blocks, int r) {
  const int g = r / N;
  const bool live = g < G;
  const int site = r - g * N;
  const RowPos rp{live ? g * N : 0, site % Lx, site / Lx, Lx, Ly};
  const float *w = sm.w;
  float h[CF];
  {  // embedding: h = b0 + sum_tap k0[tap] s(neighbour)
#pragma unroll
    for (int c = 0; c < CF; ++c) h[c] = w[9 * CF + c];
    if (live) {
      const int fl = g * N + sm.flip[g];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int j = rp.nb(t);
        float s = sm.spin[j];
        if (j == fl) s = -s;
#pragma unroll
        for (int c = 0; c < CF; ++c) h[c] = fmaf(w[t * CF + c], s, h[c]);
      }
    }
  }
  float a[CF], z[CF];
#pragma unroll 1
  for (int l = 0; l < n_blocks; ++l) {
    const float *bw = w + 10 * CF + l * BLOCK_FLOATS;
    layer_norm16(h, bw + OFF_G, bw + OFF_BE, a);
#pragma unroll
    for (int c = 0; c < CF; ++c) a[c] = gelu_f32(a[c]);
    store_row(sm.act, r, a);
    __syncthreads();
    conv_row_f32(bw + OFF_K1, bw + OFF_B1, sm.act, rp, z);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CF; ++c) a[c] = gelu_f32(z[c]);
    store_row(sm.act, r, a);
    __syncthreads();
    conv_row_f32(bw + OFF_K2, bw + OFF_B2, sm.act, rp, z);
#pragma unroll
    for (int c = 0; c < CF; ++c) h[c] += z[c];
    __syncthreads();
  }
  const float *fw = w + 10 * CF + n_blocks * BLOCK_FLOATS;
  layer_norm16(h, fw, fw + CF, a);
  float rs = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) rs += a[c];
  sm.rowsum[r] = rs;
  __syncthreads();
  // one warp per configuration adds its N rows in a fixed order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int gg = warp; gg < G; gg += nw) {
    float v = 0.f;
    for (int i = lane; i < N; i += 32) v += sm.rowsum[gg * N + i];
    v = group_allsum<32>(v);
    if (lane == 0) sm.lp[gg] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ float log_uniform_cnn(uint32_t w) {  // log u, u = (w >> 8) 2^-24; u = 0 -> -inf
  const uint32_t k = w >> 8;
  return k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
}

struct Smem {
  GroupSmem sm;
  float *thr;  // [G]
  float *lpx;  // [G]
  uint4 *pw;   // [G] Philox block of the current proposal pair
  int *acc;    // [G]
};

__device__ Smem carve(unsigned char *raw, int P, int rows, int G, int N) {
  Smem s;
  float *f = reinterpret_cast<float *>(raw);
  s.sm.w = f;
  f += (P + 3) & ~3;
  s.sm.act = f;
  f += rows * CF;
  s.sm.rowsum = f;
  f += rows;
  s.sm.spin = f;
  f += (G * N + 3) & ~3;
  s.sm.lp = f;
  f += (G + 3) & ~3;
  s.thr = f;
  f += (G + 3) & ~3;
  s.lpx = f;
  f += (G + 3) & ~3;
  s.pw = reinterpret_cast<uint4 *>(f);
  f += 4 * G;
  s.sm.flip = reinterpret_cast<int *>(f);
  f += (G + 3) & ~3;
  s.acc = reinterpret_cast<int *>(f);
  return s;
}

__device__ void load_params(float *dst, const float *src, int P) {
  for (int k = threadIdx.x; k < P; k += blockDim.x) dst[k] = src[k];
}

// Configurations from packed words: MODE 0 = log psi of cfg[q]; MODE 1 = the N + 1 local-energy
// configurations of sample q / (N + 1) (k = q mod (N + 1): 0 unflipped, else site k - 1 flipped).
template <int MODE>
__global__ void __launch_bounds__(CN_THREADS) rescnn_eval_f32_kernel(const CnnArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, G = a.G, P = n_params(a.n_blocks);
  Smem s = carve(smem_raw, P, blockDim.x, G, N);
  load_params(s.sm.w, a.cw, P);
  const int r = threadIdx.x;
  const int64_t n_groups = (a.n_cfg + G - 1) / G;
  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t q0 = grp * G;
    const int Gv = (int)std::min<int64_t>(G, a.n_cfg - q0);
    __syncthreads();  // previous group's reads of spin / flip are done
    for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
      const int g = e / N, i = e % N;
      const int64_t q = q0 + std::min(g, Gv - 1);
      const int64_t x = MODE == 0 ? q : q / (N + 1);
      const uint32_t word = a.cfg[x * a.W + (i >> 5)];
      s.sm.spin[e] = ((word >> (i & 31)) & 1u) ? 1.f : -1.f;
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x)
      s.sm.flip[g] = MODE == 0 ? -1 : (int)((q0 + std::min(g, Gv - 1)) % (N + 1)) - 1;
    __syncthreads();
    forward_group_f32(s.sm, G, N, a.Lx, a.Ly, a.n_blocks, r);
    for (int g = threadIdx.x; g < Gv; g += blockDim.x) a.out[q0 + g] = s.sm.lp[g];
  }
}

// eps(x) = J sum_<ij> s_i s_j + h sum_k exp(lp[x][k] - lp[x][0]) for the configurations of
// rescnn_eval_f32_kernel<1> (TFIM, Sec. 4.1 Eq. TFIM; App. I Eq. local_energies)
__global__ void rescnn_eloc_combine_kernel(const uint32_t *cfg, int64_t n, int N, int W, const int2 *bonds,
                                           int n_bonds, float J, float hx, const float *lp, float *eloc) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t *sw = cfg + x * W;
    float d = 0.f;
    for (int b = 0; b < n_bonds; ++b) {
      const int2 bd = bonds[b];
      const uint32_t si = (sw[bd.x >> 5] >> (bd.x & 31)) & 1u, sj = (sw[bd.y >> 5] >> (bd.y & 31)) & 1u;
      d += si == sj ? 1.f : -1.f;
    }
    const float *l = lp + x * (N + 1);
    float off = 0.f;
    for (int k = 1; k <= N; ++k) off += expf(l[k] - l[0]);
    eloc[x] = J * d + hx * off;
  }
}

// Metropolis sweeps (Sec. 3.1): a CTA takes groups of G chains and runs all their sweeps.
// Proposal p of sweep t of chain c: Philox4x32-10 block (p / 2, sweep_offset + t, c, TAG_SWEEP)
// under key (seed lo, seed hi); words (0, 1) for even p, (2, 3) for odd p: the site by the
// multiply-shift map, log u from the 24-bit uniform; accept iff 2 (lp(y) - lp(x)) > log u.
__global__ void __launch_bounds__(CN_THREADS) rescnn_sweep_f32_kernel(const CnnArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, G = a.G, W = a.W, P = n_params(a.n_blocks);
  Smem s = carve(smem_raw, P, blockDim.x, G, N);
  load_params(s.sm.w, a.cw, P);
  const int r = threadIdx.x;
  const int64_t n_groups = (a.C + G - 1) / G;
  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t c0 = grp * G;
    const int Gv = (int)std::min<int64_t>(G, a.C - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
      const int g = e / N, i = e % N;
      const int64_t c = c0 + std::min(g, Gv - 1);
      s.sm.spin[e] = ((a.state[c * W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      s.sm.flip[g] = -1;
      s.acc[g] = 0;
    }
    __syncthreads();
    forward_group_f32(s.sm, G, N, a.Lx, a.Ly, a.n_blocks, r);
    for (int g = threadIdx.x; g < G; g += blockDim.x) s.lpx[g] = s.sm.lp[g];
    int64_t nacc = 0;  // thread g < Gv: accepted proposals of chain c0 + g
    uint32_t abits = 0u;
    for (int t = 0; t < a.n_sweeps; ++t) {
      const uint32_t sweep_id = a.sweep_offset + (uint32_t)t;
      for (int p = 0; p < N; ++p) {
        if (threadIdx.x < G) {
          const int g = threadIdx.x;
          const int64_t c = c0 + std::min(g, Gv - 1);
          if ((p & 1) == 0)
            s.pw[g] = philox4x32_10(make_uint4((uint32_t)(p / 2), sweep_id, (uint32_t)c, TAG_SWEEP), a.k0, a.k1);
          const uint4 w4 = s.pw[g];
          s.sm.flip[g] = (int)index_from_word((p & 1) ? w4.z : w4.x, (uint32_t)N);
          s.thr[g] = log_uniform_cnn((p & 1) ? w4.w : w4.y);
        }
        __syncthreads();
        forward_group_f32(s.sm, G, N, a.Lx, a.Ly, a.n_blocks, r);
        if (threadIdx.x < Gv) {
          const int g = threadIdx.x;
          const int64_t c = c0 + g;
          const float dlt = s.sm.lp[g] - s.lpx[g];
          const bool acc = 2.f * dlt > s.thr[g];
          if (acc) {
            const int site = s.sm.flip[g];
            s.sm.spin[g * N + site] = -s.sm.spin[g * N + site];
            s.lpx[g] = s.sm.lp[g];
            ++nacc;
          }
          if (a.acc_bits) {
            abits |= (acc ? 1u : 0u) << (p & 31);
            if ((p & 31) == 31 || p == N - 1) {
              a.acc_bits[(c * a.n_sweeps + t) * W + (p >> 5)] = abits;
              abits = 0u;
            }
          }
          if (a.delta) a.delta[(c * a.n_sweeps + t) * N + p] = dlt;
        }
        __syncthreads();
      }
      if (t >= a.burn_in) {
        const int64_t row0 = (int64_t)(t - a.burn_in) * a.C;
        for (int e = threadIdx.x; e < Gv * W; e += blockDim.x) {
          const int g = e / W, wi = e % W;
          uint32_t word = 0u;
          for (int b = 0; b < 32 && 32 * wi + b < N; ++b)
            if (s.sm.spin[g * N + 32 * wi + b] > 0.f) word |= 1u << b;
          if (a.samples) a.samples[(row0 + c0 + g) * W + wi] = word;
        }
        if (a.logpsi)
          for (int g = threadIdx.x; g < Gv; g += blockDim.x) a.logpsi[row0 + c0 + g] = s.lpx[g];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Gv * W; e += blockDim.x) {
      const int g = e / W, wi = e % W;
      uint32_t word = 0u;
      for (int b = 0; b < 32 && 32 * wi + b < N; ++b)
        if (s.sm.spin[g * N + 32 * wi + b] > 0.f) word |= 1u << b;
      a.state[(c0 + g) * W + wi] = word;
    }
    if (threadIdx.x < Gv && a.n_acc) a.n_acc[c0 + threadIdx.x] = nacc;
  }
}

size_t smem_bytes_f32(int P, int rows, int G, int N) {
  size_t f = ((P + 3) & ~3) + (size_t)rows * CF + rows + ((G * N + 3) & ~3) + 3 * ((G + 3) & ~3) + 4 * G +
             2 * ((G + 3) & ~3);
  return f * sizeof(float);
}

// ---- O_k = d log psi / d theta_k (App. I, Eq. forces), FP32 ----------------------------------
// One CTA per configuration, thread = site.  The forward pass keeps the residual streams
// h(0) .. h(B) in shared memory; the backward pass takes the blocks from the last, recomputing
// each block's LN, GELU and first convolution from its h(l), and writes the row of O in the
// master order ([co][ci][dy][dx] kernels).  With g = d log psi / d(.):
//   final LN: d gamma_F = sum_sites zhat, d beta_F = N, g_h = LN'(1);
//   block l (h' = h + Conv2(c), c = GELU(z1), z1 = Conv1(a), a = GELU(y), y = LN(h)):
//     dK2 = sum_sites c(nb) g_h', db2 = sum g_h', g_c = Conv2^T(g_h'), g_z1 = g_c GELU'(z1),
//     dK1 = sum_sites a(nb) g_z1, db1 = sum g_z1, g_a = Conv1^T(g_z1), g_y = g_a GELU'(y),
//     d gamma = sum g_y zhat, d beta = sum g_y, g_h = g_h' + LN'(g_y);
//   embedding: dK0 = sum_sites s(nb) g_h(0), db0 = sum g_h(0).
// Conv^T reads the neighbour at the opposite offset (tap 8 - t) with K[t] transposed.

__device__ __forceinline__ float gelu_grad_f32(float z) {
  const float u = GELU_C * fmaf(0.044715f * z * z, z, z);
  const float t = tanhf(u);
  return fmaf(0.5f, 1.f + t, 0.5f * z * (1.f - t * t) * GELU_C * fmaf(3.f * 0.044715f, z * z, 1.f));
}

// LN of one site's 16 channels: zhat and 1 / sqrt(var + eps)
__device__ __forceinline__ void ln_stats16(const float (&v)[CF], float (&zh)[CF], float &rs) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) m += v[c];
  m *= 1.f / CF;
  float var = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) var = fmaf(v[c] - m, v[c] - m, var);
  rs = rsqrtf(fmaf(var, 1.f / CF, LN_EPS));
#pragma unroll
  for (int c = 0; c < CF; ++c) zh[c] = (v[c] - m) * rs;
}

// input gradient of y = zhat gamma + beta given g_y: rs (g_z - mean g_z - zhat mean(g_z zhat))
__device__ __forceinline__ void ln_back16(const float (&gy)[CF], const float (&zh)[CF], float rs, const float *g,
                                          float (&gv)[CF]) {
  float mg = 0.f, mgz = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) {
    const float gz = gy[c] * g[c];
    mg += gz;
    mgz = fmaf(gz, zh[c], mgz);
  }
  mg *= 1.f / CF;
  mgz *= 1.f / CF;
#pragma unroll
  for (int c = 0; c < CF; ++c) gv[c] = rs * (gy[c] * g[c] - mg - zh[c] * mgz);
}

struct GradSmem {
  float *w;      // [P] kernel order
  float *hs;     // [(B + 1)][N][CF] residual streams
  float *act;    // [N][CF]
  float *aux;    // [N][CF]
  float *gb;     // [N][CF]
  float *spin;   // [N]
  int *nbt;      // [9][N] neighbour site of (tap, site)
  float *stage;  // [9 CF CF] one kernel gradient in kernel order, before the ordered store
  float *red;    // [16][CF] partial channel sums
};

// sum over the N sites of buf[site][c] (or of buf[site][c] * buf2[site][c]) -> dst[c] (global)
__device__ void channel_sums(const GradSmem &sm, int N, const float *buf, const float *buf2, float *dst) {
  const int t = threadIdx.x, c = t & (CF - 1), part = t >> 4;
  const int parts = blockDim.x >> 4;
  float v = 0.f;
  if (part < 16)
    for (int i = part; i < N; i += min(parts, 16)) v += buf2 ? buf[i * CF + c] * buf2[i * CF + c] : buf[i * CF + c];
  __syncthreads();
  if (part < 16) sm.red[part * CF + c] = v;
  __syncthreads();
  if (t < CF) {
    float s = 0.f;
    for (int q = 0; q < min(parts, 16); ++q) s += sm.red[q * CF + t];
    dst[t] = s;
  }
  __syncthreads();
}

// dK[tap][ci][co] = sum_sites in[nb(tap, site)][ci] g[site][co], stored in the master order
// ([co][ci][tap]) at dst
__device__ void kernel_grad(const GradSmem &sm, int N, const float *in, const float *g, float *dst) {
  for (int e = threadIdx.x; e < 9 * CF * CF; e += blockDim.x) {
    const int tap = e / (CF * CF), ci = (e / CF) % CF, co = e % CF;
    const int *nb = sm.nbt + tap * N;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;  // four chains of FMAs over the sites
    int i = 0;
    for (; i + 3 < N; i += 4) {
      v0 = fmaf(in[nb[i] * CF + ci], g[i * CF + co], v0);
      v1 = fmaf(in[nb[i + 1] * CF + ci], g[(i + 1) * CF + co], v1);
      v2 = fmaf(in[nb[i + 2] * CF + ci], g[(i + 2) * CF + co], v2);
      v3 = fmaf(in[nb[i + 3] * CF + ci], g[(i + 3) * CF + co], v3);
    }
    for (; i < N; ++i) v0 = fmaf(in[nb[i] * CF + ci], g[i * CF + co], v0);
    sm.stage[e] = (v0 + v1) + (v2 + v3);
  }
  __syncthreads();
  for (int m = threadIdx.x; m < 9 * CF * CF; m += blockDim.x) {  // master order: m = (co CF + ci) 9 + tap
    const int tap = m % 9, ci = (m / 9) % CF, co = m / (9 * CF);
    dst[m] = sm.stage[(tap * CF + ci) * CF + co];
  }
  __syncthreads();
}

// g_in[site][ci] = sum_tap sum_co K[tap][ci][co] g[nb(8 - tap, site)][co]
__device__ __forceinline__ void conv_transpose_row(const float *K, const float *g, const GradSmem &sm, int N, int site,
                                                   float (&out)[CF]) {
#pragma unroll
  for (int c = 0; c < CF; ++c) out[c] = 0.f;
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const float *gr = g + sm.nbt[(8 - tap) * N + site] * CF;
    float gv[CF];
#pragma unroll
    for (int c = 0; c < CF; ++c) gv[c] = gr[c];
    const float *k = K + tap * CF * CF;
#pragma unroll
    for (int ci = 0; ci < CF; ++ci) {
      float s = 0.f;
#pragma unroll
      for (int co = 0; co < CF; ++co) s = fmaf(k[ci * CF + co], gv[co], s);
      out[ci] += s;
    }
  }
}

__global__ void __launch_bounds__(CN_THREADS) rescnn_grad_f32_kernel(const CnnArgs a, float *O) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, B = a.n_blocks, P = n_params(B), Lx = a.Lx, Ly = a.Ly;
  GradSmem sm;
  {
    float *f = reinterpret_cast<float *>(smem_raw);
    sm.w = f;
    f += (P + 3) & ~3;
    sm.hs = f;
    f += (B + 1) * N * CF;
    sm.act = f;
    f += N * CF;
    sm.aux = f;
    f += N * CF;
    sm.gb = f;
    f += N * CF;
    sm.spin = f;
    f += (N + 3) & ~3;
    sm.stage = f;
    f += 9 * CF * CF;
    sm.red = f;
    f += 16 * CF;
    sm.nbt = reinterpret_cast<int *>(f);
  }
  load_params(sm.w, a.cw, P);
  for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
    const int tap = e / N, i = e % N;
    const RowPos rp{0, i % Lx, i / Lx, Lx, Ly};
    sm.nbt[e] = rp.nb(tap);
  }
  const int r = threadIdx.x;
  const bool live = r < N;
  const float *w = sm.w;
  const float *fw = w + 10 * CF + B * BLOCK_FLOATS;
  for (int64_t x = blockIdx.x; x < a.n_cfg; x += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm.spin[i] = ((a.cfg[x * a.W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    __syncthreads();
    float *Orow = O + x * P;
    // ---- forward, keeping h(0) .. h(B)
    float h[CF], v[CF], z[CF];
#pragma unroll
    for (int c = 0; c < CF; ++c) h[c] = w[9 * CF + c];
    if (live) {
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
        const float sv = sm.spin[sm.nbt[t * N + r]];
#pragma unroll
        for (int c = 0; c < CF; ++c) h[c] = fmaf(w[t * CF + c], sv, h[c]);
      }
      store_row(sm.hs, r, h);
    }
#pragma unroll 1
    for (int l = 0; l < B; ++l) {
      const float *bw = w + 10 * CF + l * BLOCK_FLOATS;
      layer_norm16(h, bw + OFF_G, bw + OFF_BE, v);
#pragma unroll
      for (int c = 0; c < CF; ++c) v[c] = gelu_f32(v[c]);
      if (live) store_row(sm.act, r, v);
      __syncthreads();
      if (live) conv_row_f32(bw + OFF_K1, bw + OFF_B1, sm.act, RowPos{0, r % Lx, r / Lx, Lx, Ly}, z);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < CF; ++c) v[c] = gelu_f32(z[c]);
      if (live) store_row(sm.act, r, v);
      __syncthreads();
      if (live) {
        conv_row_f32(bw + OFF_K2, bw + OFF_B2, sm.act, RowPos{0, r % Lx, r / Lx, Lx, Ly}, z);
#pragma unroll
        for (int c = 0; c < CF; ++c) h[c] += z[c];
        store_row(sm.hs + (l + 1) * N * CF, r, h);
      }
      __syncthreads();
    }
    // ---- final LN: d gamma_F = sum zhat, d beta_F = N, g_h = LN'(1)
    {
      float zh[CF], rs, ones[CF], gh[CF];
      ln_stats16(h, zh, rs);
#pragma unroll
      for (int c = 0; c < CF; ++c) ones[c] = 1.f;
      ln_back16(ones, zh, rs, fw, gh);
      if (live) {
        store_row(sm.aux, r, zh);
        store_row(sm.gb, r, gh);
      }
      __syncthreads();
      channel_sums(sm, N, sm.aux, nullptr, Orow + 10 * CF + B * BLOCK_FLOATS);
      for (int c = threadIdx.x; c < CF; c += blockDim.x) Orow[10 * CF + B * BLOCK_FLOATS + CF + c] = (float)N;
    }
    // ---- residual blocks, the last first
#pragma unroll 1
    for (int l = B - 1; l >= 0; --l) {
      const float *bw = w + 10 * CF + l * BLOCK_FLOATS;
      float *ob = Orow + 10 * CF + l * BLOCK_FLOATS;
      float hl[CF], zh[CF], rs, y[CF], gnext[CF];
#pragma unroll
      for (int c = 0; c < CF; ++c) hl[c] = live ? sm.hs[(l * N + r) * CF + c] : 0.f;
      ln_stats16(hl, zh, rs);
#pragma unroll
      for (int c = 0; c < CF; ++c) {
        y[c] = fmaf(zh[c], bw[OFF_G + c], bw[OFF_BE + c]);
        v[c] = gelu_f32(y[c]);
      }
      if (live) {
        store_row(sm.act, r, v);  // a = GELU(LN(h))
#pragma unroll
        for (int c = 0; c < CF; ++c) gnext[c] = sm.gb[r * CF + c];
      }
      __syncthreads();
      if (live) conv_row_f32(bw + OFF_K1, bw + OFF_B1, sm.act, RowPos{0, r % Lx, r / Lx, Lx, Ly}, z);  // z1
#pragma unroll
      for (int c = 0; c < CF; ++c) v[c] = gelu_f32(z[c]);
      if (live) store_row(sm.aux, r, v);  // c = GELU(z1)
      __syncthreads();
      kernel_grad(sm, N, sm.aux, sm.gb, ob + OFF_K2);     // dK2
      channel_sums(sm, N, sm.gb, nullptr, ob + OFF_B2);  // db2
      float gz[CF];
      if (live) {
        conv_transpose_row(bw + OFF_K2, sm.gb, sm, N, r, gz);  // g_c
#pragma unroll
        for (int c = 0; c < CF; ++c) gz[c] *= gelu_grad_f32(z[c]);  // g_z1
      }
      __syncthreads();  // every read of aux (c) and gb done
      if (live) store_row(sm.aux, r, gz);
      __syncthreads();
      kernel_grad(sm, N, sm.act, sm.aux, ob + OFF_K1);    // dK1
      channel_sums(sm, N, sm.aux, nullptr, ob + OFF_B1);  // db1
      float gy[CF], gh[CF];
      if (live) {
        conv_transpose_row(bw + OFF_K1, sm.aux, sm, N, r, gy);  // g_a
#pragma unroll
        for (int c = 0; c < CF; ++c) gy[c] *= gelu_grad_f32(y[c]);  // g_y
        ln_back16(gy, zh, rs, bw + OFF_G, gh);
#pragma unroll
        for (int c = 0; c < CF; ++c) gh[c] += gnext[c];
      }
      __syncthreads();  // every read of aux (g_z1) and act done
      if (live) {
        store_row(sm.act, r, gy);
        store_row(sm.aux, r, zh);
      }
      __syncthreads();
      channel_sums(sm, N, sm.act, sm.aux, ob + OFF_G);    // d gamma = sum g_y zhat
      channel_sums(sm, N, sm.act, nullptr, ob + OFF_BE);  // d beta = sum g_y
      if (live) store_row(sm.gb, r, gh);
      __syncthreads();
    }
    // ---- embedding: dK0[co][tap] = sum_sites s(nb(tap)) g_h(0)[co], db0 = sum g_h(0)
    channel_sums(sm, N, sm.gb, nullptr, Orow + 9 * CF);
    for (int e = threadIdx.x; e < 9 * CF; e += blockDim.x) {
      const int co = e / 9, tap = e % 9;
      const int *nb = sm.nbt + tap * N;
      float acc = 0.f;
      for (int i = 0; i < N; ++i) acc = fmaf(sm.spin[nb[i]], sm.gb[i * CF + co], acc);
      Orow[e] = acc;
    }
  }
}

size_t grad_smem_bytes(int P, int N, int B) {
  return 4 * ((size_t)((P + 3) & ~3) + (size_t)(B + 1) * N * CF + 3 * (size_t)N * CF + ((N + 3) & ~3) + 9 * CF * CF +
              16 * CF + 9 * (size_t)N);
}

template <typename K>
cudaError_t launch_groups(const nqs_ctx *c, K kern, int64_t groups, size_t shm, cudaStream_t s, const CnnArgs &a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, a.rows, shm)) != cudaSuccess) return e;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)std::max(per_sm, 1) * c->num_sms));
  kern<<<(unsigned)grid, a.rows, shm, s>>>(a);
  return cudaGetLastError();
}

CnnArgs base_args(const nqs_ctx *c) {
  CnnArgs a{};
  a.cw = c->d_cw;
  a.N = c->N;
  a.W = c->W;
  a.Lx = c->Lx;
  a.Ly = c->Ly;
  a.n_blocks = c->n_blocks;
  a.G = std::max(1, CN_THREADS / c->N);
  a.rows = ((a.G * c->N + 31) / 32) * 32;
  return a;
}

}  // namespace
}  // namespace cnn

bool rescnn_setup(nqs_ctx *c, const nqs_model_desc *m, std::string *why) {
  if (c->ham_kind != NQS_TFIM) {
    *why = "the ResCNN path implements the TFIM (single-flip moves)";
    return false;
  }
  if (c->Ly < 3) {
    *why = "the ResCNN acts on a two-dimensional lattice (Ly >= 3)";
    return false;
  }
  if (c->N > cnn::CN_THREADS) {
    *why = "the ResCNN path takes at most 512 sites";
    return false;
  }
  if (m->n_hidden != cnn::CF) {
    *why = "the ResCNN kernels are built for 16 filters (n_hidden = 16)";
    return false;
  }
  if (m->n_layers < 0 || m->n_layers > cnn::MAX_BLOCKS) {
    *why = "the ResCNN takes 0 .. 8 residual blocks (n_layers)";
    return false;
  }
  c->n_blocks = m->n_layers;
  if (c->dtype != NQS_F32 && !rescnn_lp_supported(c)) {
    *why = "the ResCNN sampling copy is F32, BF16 or F16 (16-bit copies: lattices whose padded rows fit the "
           "tensor-core kernel's tiles and shared memory)";
    return false;
  }
  c->P = cnn::n_params(c->n_blocks);
  c->cnn_rows = (int64_t)1 << 20;
  return true;
}

cudaError_t rescnn_alloc(nqs_ctx *c) {
  cudaError_t e = cudaMalloc(&c->d_cw, (size_t)c->P * sizeof(float));
  if (e != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_clp, (size_t)c->cnn_rows * sizeof(float))) != cudaSuccess) return e;
  // the force without caller O rows: chunks of grad_chunk rows in d_grad_scratch, partials in d_force_part
  c->grad_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)(256u << 20) / (c->P * 4)));
  if ((e = cudaMalloc(&c->d_grad_scratch, (size_t)c->grad_chunk * c->P * sizeof(float))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->d_force_part, (size_t)64 * c->P * sizeof(double))) != cudaSuccess) return e;
  return c->dtype == NQS_F32 ? cudaSuccess : rescnn_lp_alloc(c);
}

void rescnn_free(nqs_ctx *c) {
  if (c->d_cw) cudaFree(c->d_cw);
  if (c->d_clp) cudaFree(c->d_clp);
  if (c->d_grad_scratch) cudaFree(c->d_grad_scratch);
  if (c->d_force_part) cudaFree(c->d_force_part);
  c->d_grad_scratch = nullptr;
  c->d_force_part = nullptr;
  rescnn_lp_free(c);
  c->d_cw = nullptr;
  c->d_clp = nullptr;
}

cudaError_t rescnn_prepare(nqs_ctx *c, const double *params, cudaStream_t s) {
  cnn::rescnn_prepare_f32_kernel<<<(unsigned)std::min<int64_t>((c->P + 255) / 256, 1024), 256, 0, s>>>(
      params, c->n_blocks, c->d_cw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || c->dtype == NQS_F32) return e;
  return rescnn_lp_prepare(c, params, s);
}

cudaError_t rescnn_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  if (c->dtype != NQS_F32) return rescnn_lp_logpsi(c, cfg, n, out, s);
  cnn::CnnArgs a = cnn::base_args(c);
  a.cfg = cfg;
  a.n_cfg = n;
  a.out = out;
  const size_t shm = cnn::smem_bytes_f32((int)c->P, a.rows, a.G, c->N);
  return cnn::launch_groups(c, cnn::rescnn_eval_f32_kernel<0>, (n + a.G - 1) / a.G, shm, s, a);
}

cudaError_t rescnn_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s) {
  const int64_t per = c->N + 1;
  const int64_t chunk = std::max<int64_t>(1, c->cnn_rows / per);
  for (int64_t x0 = 0; x0 < n; x0 += chunk) {
    const int64_t nx = std::min(chunk, n - x0);
    cudaError_t e;
    if (c->dtype != NQS_F32) {
      e = rescnn_lp_eval_flips(c, cfg + x0 * c->W, nx, c->d_clp, s);
    } else {
      cnn::CnnArgs a = cnn::base_args(c);
      a.cfg = cfg + x0 * c->W;
      a.n_cfg = nx * per;
      a.out = c->d_clp;
      const size_t shm = cnn::smem_bytes_f32((int)c->P, a.rows, a.G, c->N);
      e = cnn::launch_groups(c, cnn::rescnn_eval_f32_kernel<1>, (a.n_cfg + a.G - 1) / a.G, shm, s, a);
    }
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nx + 127) / 128, (int64_t)c->num_sms * 8));
    cnn::rescnn_eloc_combine_kernel<<<blocks, 128, 0, s>>>(cfg + x0 * c->W, nx, c->N, c->W, c->d_bonds, c->n_bonds,
                                                           (float)c->J1, (float)c->h, c->d_clp, eloc + x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t rescnn_sweep(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int burn_in, uint64_t seed,
                         uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc, uint32_t *acc_bits,
                         float *delta, cudaStream_t s) {
  if (c->dtype != NQS_F32)
    return rescnn_lp_sweep(c, state, C, n_sweeps, burn_in, seed, sweep_offset, samples, logpsi, n_acc, acc_bits,
                           delta, s);
  cnn::CnnArgs a = cnn::base_args(c);
  a.state = state;
  a.C = C;
  a.n_sweeps = n_sweeps;
  a.burn_in = burn_in;
  a.sweep_offset = sweep_offset;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.samples = samples;
  a.logpsi = logpsi;
  a.n_acc = n_acc;
  a.acc_bits = acc_bits;
  a.delta = delta;
  const size_t shm = cnn::smem_bytes_f32((int)c->P, a.rows, a.G, c->N);
  return cnn::launch_groups(c, cnn::rescnn_sweep_f32_kernel, (C + a.G - 1) / a.G, shm, s, a);
}

bool rescnn_grad_supported(const nqs_ctx *c) {
  return cnn::grad_smem_bytes((int)c->P, c->N, c->n_blocks) <= (size_t)c->smem_optin;
}

cudaError_t rescnn_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                               const double *stats, double *force, cudaStream_t s, bool share) {
  cnn::CnnArgs a = cnn::base_args(c);
  // a CTA per configuration: a thread per site for the site-wise passes, and every thread of
  // the CTA for the parameter gradients' sums over sites
  a.rows = cnn::CN_THREADS;
  const size_t shm = cnn::grad_smem_bytes((int)c->P, c->N, c->n_blocks);
  cudaError_t e = cudaFuncSetAttribute(cnn::rescnn_grad_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  const int64_t chunk = O ? n : c->grad_chunk;
  for (int64_t x0 = 0; x0 < n; x0 += chunk) {
    const int64_t rows = std::min<int64_t>(chunk, n - x0);
    a.cfg = cfg + x0 * c->W;
    a.n_cfg = rows;
    float *Ob = O ? O + x0 * c->P : c->d_grad_scratch;
    cnn::rescnn_grad_f32_kernel<<<(unsigned)std::min<int64_t>(rows, (int64_t)c->num_sms * 8), a.rows, shm, s>>>(a, Ob);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (force && !O && (e = force_rows(c, Ob, rows, eloc + x0, stats, n, share, x0 > 0, force, s)) != cudaSuccess)
      return e;
  }
  if (force && O) return force_rows(c, O, n, eloc, stats, n, share, 0, force, s);
  return cudaSuccess;
}

}  // namespace nqs
