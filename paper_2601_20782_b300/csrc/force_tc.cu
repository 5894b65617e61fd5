// Force of the RBM (App. I, Eq. forces) on the tensor cores:
//     F_k = (1/n) sum_x O_k(x) (eloc(x) - E),  O_a = s, O_b = tanh(theta), O_W[j, i] = tanh(theta_j) s_i.
//
// Block (jt, chunk) owns hidden units j0 = 128 jt .. j0 + 127 and one chunk of rows; per
// tile of 128 rows (samples x) it runs two tcgen05 products with FP32 accumulation in TMEM:
//   GEMM1  theta[x, j] = sum_i s[x, i] W[j, i]             A1 = spins (exact in BF16),
//                                                          B1 = W as three BF16 terms (hi + mid + lo)
//   GEMM2  G[j, i]    += sum_x a[x, j] s[x, i]             a = tanh(theta + b) (eloc - E), three BF16 terms
// Column i = N of the spin tile is a constant +1 (its W column is zero), so G[j, N] = sum_x a[x, j]
// gives the b-entries; the extra hidden row j = M carries a = eloc - E, so G[M, i] gives the a-entries.
// The spin tile serves as the K-major A of GEMM1 and, read MN-major, as the B of GEMM2.
// The hi term of a accumulates in one TMEM accumulator and the mid + lo terms in a second one,
// so that the small terms are not rounded away against the large running sum.  Every DRAIN
// tiles both are added into the block's FP64 slice of the workspace (rows chunk * P ...),
// which force_reduce_kernel then sums over chunks in a fixed order.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace nqs {
namespace {

constexpr int FTC_THREADS = 256;
constexpr int FTC_DRAIN = 16;  // tiles between FP64 drains of the accumulators
constexpr uint32_t FTC_POLLS = 1u << 24;

struct ForceTcParams {
  const uint32_t *cfg;
  const float *eloc;
  const double *stats;
  const float *Wm;  // [N][M] FP32 master, site-major
  const float *bm;  // [M]
  double *ws;       // [chunks][P]
  int *status;
  int64_t n, P;
  int N, W, M, Kp, N2, n_chunks;
};

__device__ __forceinline__ void split3(float a, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(a);
  const float r = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(FTC_THREADS, 1) rbm_force_tc_kernel(const ForceTcParams p) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const uint32_t raw = smem_addr(smem_dyn);
  unsigned char *base = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  const int nkb = p.Kp / 64;
  unsigned char *sA1 = base;                       // [128 x][Kp]            K-major, nkb x 16 KB
  unsigned char *sB1 = sA1 + nkb * 16384;          // 3 x [128 j][Kp]        K-major
  unsigned char *sA2 = sB1 + 3 * nkb * 16384;      // 3 x [128 x (K)][128 j] MN-major, 2 x 16 KB each
  float *se = reinterpret_cast<float *>(sA2 + 3 * 32768);  // [128] eloc - E
  float *sb = se + 128;                                    // [128] hidden bias of the tile

  const int jt = blockIdx.x, chunk = blockIdx.y;
  const int j0 = jt * 128;
  const int N = p.N, M = p.M, Kp = p.Kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- B1: W of the tile as three BF16 terms; sb: bias --------------------------------
  for (int idx = tid; idx < 128 * Kp; idx += FTC_THREADS) {
    const int jj = idx % 128, i = idx / 128;
    const float w = (j0 + jj < M && i < N) ? p.Wm[(int64_t)i * M + j0 + jj] : 0.f;
    __nv_bfloat16 h, m, l;
    split3(w, h, m, l);
    const uint32_t off = (i / 64) * 16384 + tc::sw128_offset(jj, i % 64);
    *reinterpret_cast<__nv_bfloat16 *>(sB1 + off) = h;
    *reinterpret_cast<__nv_bfloat16 *>(sB1 + nkb * 16384 + off) = m;
    *reinterpret_cast<__nv_bfloat16 *>(sB1 + 2 * nkb * 16384 + off) = l;
  }
  for (int jj = tid; jj < 128; jj += FTC_THREADS) sb[jj] = (j0 + jj < M) ? p.bm[j0 + jj] : 0.f;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tD1 = tmem_base, tD2 = tmem_base + 128, tD3 = tmem_base + 256;
  const double E = p.stats[0];
  const int64_t rows_per_chunk = (p.n + p.n_chunks - 1) / p.n_chunks;
  const int64_t r0 = (int64_t)chunk * rows_per_chunk, r1 = min(p.n, r0 + rows_per_chunk);
  const uint32_t id1 = tc::idesc_bf16_f32(128, 128);
  const uint32_t id2 = tc::idesc_bf16_f32(128, (uint32_t)p.N2, 1, 1);
  uint32_t phase = 0;
  int tiles_since_drain = 0, drains = 0;
  double *out = p.ws + (int64_t)chunk * p.P;

  // Waits for the products committed last; the result is uniform across the block.
  auto wait_mma = [&]() -> bool {
    const bool ok = mbar_wait_bounded(&bar, phase, FTC_POLLS);
    phase ^= 1u;
    const bool any_fail = __syncthreads_or(!ok);
    if (any_fail && tid == 0) {
      atomicOr(p.status, STATUS_TIMEOUT);
      abort_flag = 1;
    }
    tc::fence_after_sync();
    return !any_fail;
  };

  // Adds the FP32 accumulator G (TMEM columns 128 .. 128 + N2) into the FP64 slice
  // (zero_only: writes zeros, for a chunk without rows).
  auto drain = [&](bool zero_only) {
    const int q = warp & 3, h = warp >> 2;
    const int jj = 32 * q + lane, j = j0 + jj;
    for (int c = 0; c < 2; ++c) {
      const int i0 = 64 * h + 32 * c;
      if (i0 >= p.N2) break;  // warp-uniform
      float v[32], w[32];
      if (zero_only) {
        for (int t = 0; t < 32; ++t) v[t] = w[t] = 0.f;
      } else {
        tc::tmem_ld32(tc::tmem_lane_addr(tD2, 32 * q, i0), v);
        tc::tmem_ld32(tc::tmem_lane_addr(tD3, 32 * q, i0), w);
      }
      for (int t = 0; t < 32; ++t) {
        const int i = i0 + t;
        int64_t k = -1;
        if (j < M && i < N) k = N + M + (int64_t)j * N + i;   // W entries
        else if (j < M && i == N) k = N + j;                   // b entries
        else if (j == M && i < N) k = i;                       // a entries
        if (k >= 0) out[k] = (drains ? out[k] : 0.0) + ((double)v[t] + (double)w[t]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    ++drains;
    tiles_since_drain = 0;
  };

  for (int64_t x0 = r0; x0 < r1; x0 += 128) {
    const int nb = (int)(r1 - x0 < 128 ? r1 - x0 : 128);
    // ---- stage the spin tile (row x: +-1 for i < N, +1 at i = N, 0 beyond) and e --------
    if (tid < 128) {
      const int x = tid;
      uint32_t words[4] = {0u, 0u, 0u, 0u};
      if (x < nb)
        for (int w = 0; w < p.W; ++w) words[w] = p.cfg[(x0 + x) * p.W + w];
      for (int c = 0; c < Kp / 8; ++c) {  // 16-byte chunk c holds sites 8c .. 8c + 7
        uint32_t pk[4];
        for (int q2 = 0; q2 < 4; ++q2) {
          float f[2];
          for (int e = 0; e < 2; ++e) {
            const int i = 8 * c + 2 * q2 + e;
            f[e] = (x >= nb) ? 0.f : (i < N ? (((words[i >> 5] >> (i & 31)) & 1u) ? 1.f : -1.f) : (i == N ? 1.f : 0.f));
          }
          pk[q2] = pack2(__float2bfloat16_rn(f[0]), __float2bfloat16_rn(f[1]));
        }
        const uint32_t off = (c / 8) * 16384 + (x >> 3) * 1024 + (x & 7) * 128 + ((((c & 7) ^ (x & 7)) & 7) << 4);
        *reinterpret_cast<uint4 *>(sA1 + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      se[x] = x < nb ? (float)((double)p.eloc[x0 + x] - E) : 0.f;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // ---- GEMM1: theta = spins * W^T (three W terms into one accumulator) ---------------
    if (tid == 0) {
      uint32_t acc = 0;
      for (int s = 0; s < 3; ++s)
        for (int k0 = 0; k0 < Kp; k0 += 16) {
          const uint64_t ad = tc::desc_sw128(smem_addr(sA1 + (k0 / 64) * 16384 + (k0 % 64) * 2));
          const uint64_t bd = tc::desc_sw128(smem_addr(sB1 + s * nkb * 16384 + (k0 / 64) * 16384 + (k0 % 64) * 2));
          tc::mma_bf16(tD1, ad, bd, id1, acc);
          acc = 1;
        }
      tc::mma_commit(&bar);
    }
    if (!wait_mma()) break;
    // ---- epilogue: a = tanh(theta + b) e, three BF16 terms, MN-major rows x ---------------
    {
      const int q = warp & 3, h = warp >> 2;
      const int x = 32 * q + lane;
      const float ex = se[x];
      for (int c = 0; c < 2; ++c) {
        const int jb = 64 * h + 32 * c;  // 32 hidden units jb .. jb + 31
        float v[32];
        tc::tmem_ld32(tc::tmem_lane_addr(tD1, 32 * q, jb), v);
        uint32_t ph[16], pm[16], pl[16];
        for (int t = 0; t < 32; t += 2) {
          __nv_bfloat16 h0, m0, l0, h1, m1, l1;
          for (int u = 0; u < 2; ++u) {
            const int jj = jb + t + u;
            float a = tanhf(v[t + u] + sb[jj]) * ex;
            if (j0 + jj == M) a = ex;
            if (u == 0) split3(a, h0, m0, l0);
            else split3(a, h1, m1, l1);
          }
          ph[t / 2] = pack2(h0, h1);
          pm[t / 2] = pack2(m0, m1);
          pl[t / 2] = pack2(l0, l1);
        }
        // row x, M-elements jb .. jb + 31: 64-element group jb / 64, chunks (jb % 64) / 8 .. + 3
        for (int cc = 0; cc < 4; ++cc) {
          const int chunk16 = ((jb & 63) >> 3) + cc;
          const uint32_t off = (jb >> 6) * 16384 + (x >> 3) * 1024 + (x & 7) * 128 + (((chunk16 ^ (x & 7)) & 7) << 4);
          *reinterpret_cast<uint4 *>(sA2 + off) = make_uint4(ph[4 * cc], ph[4 * cc + 1], ph[4 * cc + 2], ph[4 * cc + 3]);
          *reinterpret_cast<uint4 *>(sA2 + 32768 + off) =
              make_uint4(pm[4 * cc], pm[4 * cc + 1], pm[4 * cc + 2], pm[4 * cc + 3]);
          *reinterpret_cast<uint4 *>(sA2 + 65536 + off) =
              make_uint4(pl[4 * cc], pl[4 * cc + 1], pl[4 * cc + 2], pl[4 * cc + 3]);
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- GEMM2: G += a^T spins (a MN-major over j, spins MN-major over i) ---------------
    if (tid == 0) {
      for (int s = 0; s < 3; ++s)
        for (int k0 = 0; k0 < 128; k0 += 16) {
          const uint64_t ad = tc::desc_sw128(smem_addr(sA2 + s * 32768 + k0 * 128), 16384);
          const uint64_t bd = tc::desc_sw128(smem_addr(sA1 + k0 * 128), 16384);
          const bool first = tiles_since_drain == 0 && k0 == 0 && s < 2;  // s = 1 starts the second accumulator
          tc::mma_bf16(s == 0 ? tD2 : tD3, ad, bd, id2, first ? 0u : 1u);
        }
      tc::mma_commit(&bar);
    }
    if (!wait_mma()) break;
    ++tiles_since_drain;
    if (tiles_since_drain == FTC_DRAIN) drain(false);
  }
  __syncthreads();
  if (!abort_flag) {
    if (tiles_since_drain > 0) drain(false);
    else if (drains == 0) drain(true);
  } else {
    mbar_wait_bounded(&bar, phase, FTC_POLLS);  // let a pending product finish before freeing TMEM
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, 512);
}

}  // namespace

bool rbm_force_tc_supported(const nqs_ctx *c) { return c->N <= 127; }

int rbm_force_tc_chunks(const nqs_ctx *c, int64_t n) {
  const int jt = (c->M + 1 + 127) / 128;
  int64_t ch = std::max<int64_t>(1, c->num_sms / jt);
  ch = std::min<int64_t>(ch, (n + 127) / 128);
  return (int)std::max<int64_t>(1, ch);
}

cudaError_t rbm_force_tc(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                         double *ws, int chunks, cudaStream_t s) {
  ForceTcParams p;
  p.cfg = cfg;
  p.eloc = eloc;
  p.stats = stats;
  p.Wm = c->d_Wm;
  p.bm = c->d_bm;
  p.ws = ws;
  p.status = c->d_status;
  p.n = n;
  p.P = c->P;
  p.N = c->N;
  p.W = c->W;
  p.M = c->M;
  p.Kp = ((c->N + 1 + 63) / 64) * 64;
  p.N2 = ((c->N + 1 + 15) / 16) * 16;
  p.n_chunks = chunks;
  const int jt = (c->M + 1 + 127) / 128;
  const size_t shm = 1024 + (size_t)(p.Kp / 64) * 16384 * 4 + 3 * 32768 + 2 * 128 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(rbm_force_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  rbm_force_tc_kernel<<<dim3(jt, chunks), FTC_THREADS, shm, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nqs
