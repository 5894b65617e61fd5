// Layer GEMM of the dense ansatz on the tensor cores: for rows r of an activation matrix A
// [R x Kpad] (BF16, row-major) and weights B [N x Kpad] (BF16, row-major: B[n][k] = W[n][k]),
//   z[r][n] = sum_k A[r][k] B[n][k]     (tcgen05.mma kind::f16, FP32 accumulation in TMEM)
// followed by one of two epilogues:
//   STORE: out[r][n] = bf16(tanh(z + bias[n]))                      (the next layer's input)
//   DOT:   part[r][range][h] = sum over the range's column chunks of parity h of
//          tanh(z + bias[n]) w[n]                               (last hidden layer -> log psi)
// (dense ansatz: a_l = tanh(W_l a_{l-1} + b_l), log psi = w_out . a_L + b_out).
//
// A CTA owns 128 rows and an N-range of NR <= 512 columns, computed as two MMA parts of
// p0 and p1 columns into one 512-column TMEM accumulator.  Warp roles: warp 0 issues the
// TMA loads of A and B K-blocks (64 wide, 128-byte swizzle) into a ring of stages, warp 1
// allocates TMEM and issues the MMAs (one thread), warps 2-9 run the epilogue: two warps
// per TMEM lane quarter (thread = row = lane), each taking every other 32-column chunk.
// tanh is the MUFU tanh.approx (relative error ~2^-11, below the BF16 rounding of the
// activations).  The CTA loops over row tiles; stage and accumulator hand-offs use
// mbarriers, every wait bounded.
//
// F8 = true is the FP8 sampling copy: A and B in E4M3 (tcgen05.mma kind::f8f6f4, K = 32 per
// instruction), B = W_l * s_l with a per-layer power-of-two scale s_l, so the epilogue takes
// z = acc / s_l; STORE writes E4M3 activations.  A K-block is then 128 elements (still 128
// bytes per row), so the shared-memory tiles and descriptors are those of the BF16 kernel.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace nqs {

bool make_tmap_bf16_2d(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  using Fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                          const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                          CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Fn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<Fn>(p);
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_u8_2d(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  using Fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                          const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                          CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Fn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<Fn>(p);
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols};
  const cuuint32_t box[2] = {128, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

constexpr int GEMM_THREADS = 320;

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr uint32_t GEMM_POLLS = 1u << 24;

struct GemmArgs {
  int R, Kpad, NR, p0, p1, n_ranges, N, mode;
  const float *bias;
  const float *w;
  void *out_act;             // BF16 or (F8) E4M3 [R][ld_out]
  const float *inv_scale;    // F8: 1 / s_l of the layer (device scalar)
  int ld_out;
  float *out_part;
  int *status;
};

// TALL: a CTA owns two row tiles (256 rows) and an N-range of NR <= 256 columns: per K-block
// it loads both A tiles and one B tile and issues one N = NR product per A tile, into TMEM
// columns 0 and 256.  Per K-block that is 64 KB for 256 x 256 outputs instead of 80 KB for
// 128 x 512, i.e. 25 % more products per byte delivered to the SM.  The epilogue warp pair
// of a lane quarter then takes one tile each, over all of the range's columns.
template <int STAGES, bool F8, bool TALL>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    dense_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB0,
                      const __grid_constant__ CUtensorMap mB1, const GemmArgs g) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t full[STAGES], empty[STAGES], tfull, tempty;
  __shared__ float s_bias[512], s_w[512];  // the range's bias and (DOT) w_out, read once
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const uint32_t raw = smem_addr(smem_dyn);
  unsigned char *base = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t a_bytes = TALL ? 32768u : 16384u, b_bytes = (uint32_t)g.NR * 128u, stage_bytes = a_bytes + b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, 8);
    fence_mbar_init();
    abort_flag = 0;
    prefetch_tmap(&mA);
    prefetch_tmap(&mB0);
    if (g.p1) prefetch_tmap(&mB1);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  for (int c = tid; c < g.NR; c += GEMM_THREADS) {
    const int n = blockIdx.y * g.NR + c;
    s_bias[c] = n < g.N ? g.bias[n] : 0.f;
    s_w[c] = (g.mode == 1 && n < g.N) ? g.w[n] : 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  // bounded wait that also gives up once another role has aborted
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    for (uint32_t it = 0; it < GEMM_POLLS; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if (abort_flag) return false;
    }
    abort_flag = 1;
    atomicOr(g.status, STATUS_TIMEOUT);
    return false;
  };

  const int n_tiles = (g.R + 127) / 128;
  const int n_steps = TALL ? (n_tiles + 1) / 2 : n_tiles;  // a step is one (TALL: two) row tile(s)
  constexpr int KB = F8 ? 128 : 64;  // elements per 128-byte K-block
  const int kb_n = g.Kpad / KB;
  const int range = blockIdx.y;
  const int nbase = range * g.NR;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      uint32_t it = 0;
      for (int step = blockIdx.x; step < n_steps && !abort_flag; step += gridDim.x)
        for (int kb = 0; kb < kb_n; ++kb, ++it) {
          const int s = it % STAGES;
          if (!wait(&empty[s], ((it / STAGES) & 1u) ^ 1u)) break;
          unsigned char *st = base + s * stage_bytes;
          mbar_expect_tx(&full[s], stage_bytes);
          if constexpr (TALL) {  // the second tile may lie past R: TMA fills those rows with zeros
            tma_load_2d(st, &mA, kb * KB, 2 * step * 128, &full[s]);
            tma_load_2d(st + 16384, &mA, kb * KB, (2 * step + 1) * 128, &full[s]);
          } else {
            tma_load_2d(st, &mA, kb * KB, step * 128, &full[s]);
          }
          tma_load_2d(st + a_bytes, &mB0, kb * KB, nbase, &full[s]);
          if (g.p1) tma_load_2d(st + a_bytes + g.p0 * 128, &mB1, kb * KB, nbase + g.p0, &full[s]);
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id0 = F8 ? tc::idesc_e4m3_f32(128, (uint32_t)(TALL ? g.NR : g.p0))
                              : tc::idesc_bf16_f32(128, (uint32_t)(TALL ? g.NR : g.p0));
      const uint32_t n1 = (uint32_t)(g.p1 ? g.p1 : 16);
      const uint32_t id1 = F8 ? tc::idesc_e4m3_f32(128, n1) : tc::idesc_bf16_f32(128, n1);
      uint32_t it = 0, t = 0;
      for (int step = blockIdx.x; step < n_steps && !abort_flag; step += gridDim.x, ++t) {
        if (!wait(&tempty, (t & 1u) ^ 1u)) break;
        tc::fence_after_sync();
        bool ok = true;
        for (int kb = 0; kb < kb_n; ++kb, ++it) {
          const int s = it % STAGES;
          if (!wait(&full[s], (it / STAGES) & 1u)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          unsigned char *st = base + s * stage_bytes;
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::desc_sw128(smem_addr(st + kk * 32));
            const uint64_t b0 = tc::desc_sw128(smem_addr(st + a_bytes + kk * 32));
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            if constexpr (TALL) {  // B (both boxes, NR rows) against each A tile
              const uint64_t ad1 = tc::desc_sw128(smem_addr(st + 16384 + kk * 32));
              if constexpr (F8) {
                tc::mma_f8(tmem, ad, b0, id0, acc);
                tc::mma_f8(tmem + 256u, ad1, b0, id0, acc);
              } else {
                tc::mma_bf16(tmem, ad, b0, id0, acc);
                tc::mma_bf16(tmem + 256u, ad1, b0, id0, acc);
              }
              continue;
            }
            if constexpr (F8) tc::mma_f8(tmem, ad, b0, id0, acc);
            else tc::mma_bf16(tmem, ad, b0, id0, acc);
            if (g.p1) {
              const uint64_t b1 = tc::desc_sw128(smem_addr(st + a_bytes + g.p0 * 128 + kk * 32));
              if constexpr (F8) tc::mma_f8(tmem + (uint32_t)g.p0, ad, b1, id1, acc);
              else tc::mma_bf16(tmem + (uint32_t)g.p0, ad, b1, id1, acc);
            }
          }
          tc::mma_commit(&empty[s]);  // stage free once these products are done
        }
        if (!ok) break;
        tc::mma_commit(&tfull);  // accumulator ready
      }
    }
  } else {  // ---- epilogue warps 2..9: row = TMEM lane, every other 32-column chunk
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int row_in_tile = 32 * q + lane;
    const float sc = F8 ? *g.inv_scale : 1.f;
    uint32_t t = 0;
    // TALL: this warp takes tile 2 step + half (accumulator at column 256 half), every chunk;
    // otherwise tile step, every other 32-column chunk from 32 half
    const int c_first = TALL ? 0 : 32 * half, c_step = TALL ? 32 : 64;
    const uint32_t acc_col = TALL ? 256u * (uint32_t)half : 0u;
    for (int step = blockIdx.x; step < n_steps; step += gridDim.x, ++t) {
      if (!wait(&tfull, t & 1u)) break;
      tc::fence_after_sync();
      const int r = (TALL ? 2 * step + half : step) * 128 + row_in_tile;
      float dot = 0.f;
      for (int c0 = c_first; c0 < g.NR; c0 += c_step) {
        float v[32];
        tc::tmem_ld32(tc::tmem_lane_addr(tmem, 32 * q, acc_col + c0), v);
        if (r < g.R) {
          if (g.mode == 0) {
            float a[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int n = nbase + c0 + e;  // columns of this CTA's range only
              a[e] = (n < g.N && c0 + e < g.NR) ? tanh_fast(fmaf(v[e], sc, s_bias[c0 + e])) : 0.f;
            }
            const int n0 = nbase + c0;
            if constexpr (F8) {  // 32 E4M3 values: two 16-byte stores
              uint32_t pk[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a[4 * u], a[4 * u + 1]), __NV_SATFINITE, __NV_E4M3);
                const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(a[4 * u + 2], a[4 * u + 3]), __NV_SATFINITE, __NV_E4M3);
                pk[u] = lo | (hi << 16);
              }
              uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(g.out_act) + (int64_t)r * g.ld_out + n0);
              const int nv = min(2, (min(g.N - n0, g.NR - c0) + 15) / 16);
              for (int u = 0; u < nv; ++u) dst[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
            } else {
              uint32_t pk[16];
#pragma unroll
              for (int e = 0; e < 32; e += 2) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a[e], a[e + 1]);
                pk[e / 2] = *reinterpret_cast<const uint32_t *>(&h);
              }
              uint4 *dst =
                  reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(g.out_act) + (int64_t)r * g.ld_out + n0);
              const int nv = min(4, (min(g.N - n0, g.NR - c0) + 7) / 8);
              for (int u = 0; u < nv; ++u) dst[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int n = nbase + c0 + e;
              if (n < g.N && c0 + e < g.NR) dot = fmaf(tanh_fast(fmaf(v[e], sc, s_bias[c0 + e])), s_w[c0 + e], dot);
            }
          }
        }
      }
      if (g.mode == 1 && r < g.R) {
        if constexpr (TALL) {  // the whole range's dot in one warp: slot 0, slot 1 zero
          g.out_part[((int64_t)r * g.n_ranges + range) * 2] = dot;
          g.out_part[((int64_t)r * g.n_ranges + range) * 2 + 1] = 0.f;
        } else {
          g.out_part[((int64_t)r * g.n_ranges + range) * 2 + half] = dot;
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty)) : "memory");
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (abort_flag && tid == 0) {  // let products or copies in flight land before TMEM/smem are released
    for (int s = 0; s < STAGES; ++s) mbar_wait_bounded(&empty[s], 0, 1u << 16);
  }
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

// Host side of one layer product.  Weight maps (box rows p0 / p1) are passed in; the
// activation map is encoded here (its address and row count change per call).
cudaError_t dense_gemm(const nqs_ctx *c, const void *A, int R, int Kpad, const CUtensorMap &mB0,
                       const CUtensorMap &mB1, int N, int NR, int p0, int p1, int mode, const float *bias,
                       const float *w, void *out_act, int ld_out, float *out_part, cudaStream_t s,
                       const float *inv_scale, bool tall) {
  if (R <= 0) return cudaSuccess;
  if (tall && NR > 256) return cudaErrorInvalidValue;
  const bool f8 = inv_scale != nullptr;
  CUtensorMap mA;
  if (!(f8 ? make_tmap_u8_2d(&mA, A, (uint64_t)R, (uint64_t)Kpad, 128)
           : make_tmap_bf16_2d(&mA, A, (uint64_t)R, (uint64_t)Kpad, 128)))
    return cudaErrorInvalidValue;
  GemmArgs g;
  g.R = R;
  g.Kpad = Kpad;
  g.NR = NR;
  g.p0 = p0;
  g.p1 = p1;
  g.n_ranges = (N + NR - 1) / NR;
  g.N = N;
  g.mode = mode;
  g.bias = bias;
  g.w = w;
  g.out_act = out_act;
  g.inv_scale = inv_scale;
  g.ld_out = ld_out;
  g.out_part = out_part;
  g.status = c->d_status;
  const size_t stage = (tall ? 32768 : 16384) + (size_t)NR * 128;
  const int stages = (int)std::min<size_t>(4, (size_t)(c->smem_optin - 2048 - 4096) / stage);  // - static bias / w_out
  const size_t shm = 1024 + stages * stage;
  const int n_steps = tall ? (R + 255) / 256 : (R + 127) / 128;
  const int gx = std::max(1, std::min(n_steps, c->num_sms / g.n_ranges));
  const dim3 grid(gx, g.n_ranges);
  cudaError_t e;
#define NQS_LAUNCH(S)                                                                                        \
  {                                                                                                          \
    auto k = tall ? (f8 ? dense_gemm_kernel<S, true, true> : dense_gemm_kernel<S, false, true>)            \
                  : (f8 ? dense_gemm_kernel<S, true, false> : dense_gemm_kernel<S, false, false>);          \
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)) != cudaSuccess) \
      return e;                                                                                              \
    k<<<grid, GEMM_THREADS, shm, s>>>(mA, mB0, mB1, g);                                                      \
    return cudaGetLastError();                                                                               \
  }
  if (stages >= 4) NQS_LAUNCH(4)
  if (stages == 3) NQS_LAUNCH(3)
  if (stages == 2) NQS_LAUNCH(2)
#undef NQS_LAUNCH
  return cudaErrorInvalidConfiguration;
}

}  // namespace nqs
