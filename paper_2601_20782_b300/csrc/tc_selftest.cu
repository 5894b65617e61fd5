// nqs_selftest_tc_gemm: checks the tensor-core building block (swizzled operand
// tiles written by threads, tcgen05.mma kind::f16, TMEM accumulator, tcgen05.ld)
// on one 128 x N x K product, D = A B^T.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "tc.cuh"

namespace nqs {
namespace {

// flags bit 0: A is given as [K x 128] and staged MN-major; bit 1: B is given as [K x N]
// and staged MN-major.  Otherwise A [128 x K], B [N x K], staged K-major.
__global__ void __launch_bounds__(128) tc_gemm_selftest_kernel(const uint16_t *__restrict__ A,
                                                               const uint16_t *__restrict__ B, float *D, int N,
                                                               int K, int flags, int *status) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const uint32_t raw = smem_addr(smem_dyn);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  unsigned char *base = smem_dyn + pad;
  const int nkb = K / 64;
  const bool a_mn = flags & 1, b_mn = flags & 2;
  const int nnb = (N + 63) / 64;                 // 64-wide N groups of an MN-major B
  unsigned char *sA = base;                      // 128 x K elements either way: 16 KB per 64 of K or of M
  unsigned char *sB = base + nkb * 128 * 128;
  for (int idx = threadIdx.x; idx < 128 * K; idx += blockDim.x) {
    if (!a_mn) {
      const int r = idx / K, k = idx % K;
      *reinterpret_cast<uint16_t *>(sA + (k / 64) * 16384 + tc::sw128_offset(r, k % 64)) = A[idx];
    } else {  // A given [K x 128]: K-row k holds M elements; 64-element M groups K*128 bytes apart
      const int k = idx / 128, m = idx % 128;
      *reinterpret_cast<uint16_t *>(sA + (m / 64) * (K * 128) + tc::sw128_offset(k, m % 64)) = A[idx];
    }
  }
  for (int idx = threadIdx.x; idx < N * K; idx += blockDim.x) {
    if (!b_mn) {
      const int r = idx / K, k = idx % K;
      *reinterpret_cast<uint16_t *>(sB + (k / 64) * (N * 128) + tc::sw128_offset(r, k % 64)) = B[idx];
    } else {  // B given [K x N]
      const int k = idx / N, n = idx % N;
      *reinterpret_cast<uint16_t *>(sB + (n / 64) * (K * 128) + tc::sw128_offset(k, n % 64)) = B[idx];
    }
  }
  (void)nnb;
  tc::fence_proxy_async_smem();
  uint32_t ncols = 32;
  while (ncols < (uint32_t)N) ncols <<= 1;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)N, a_mn ? 1u : 0u, b_mn ? 1u : 0u);
    uint32_t acc = 0;
    for (int k0 = 0; k0 < K; k0 += 16) {
      // K-major: K-block k0/64, +32 bytes per 16 of K inside it.  MN-major: 16 K-rows = 2048 bytes.
      const uint64_t ad = a_mn ? tc::desc_sw128(smem_addr(sA + k0 * 128), K * 128)
                               : tc::desc_sw128(smem_addr(sA + (k0 / 64) * 16384 + (k0 % 64) * 2));
      const uint64_t bd = b_mn ? tc::desc_sw128(smem_addr(sB + k0 * 128), K * 128)
                               : tc::desc_sw128(smem_addr(sB + (k0 / 64) * (N * 128) + (k0 % 64) * 2));
      tc::mma_bf16(taddr, ad, bd, idesc, acc);
      acc = 1;
    }
    tc::mma_commit(&bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, 1u << 22);
  if (!ok && threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
  tc::fence_after_sync();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tc::tmem_lane_addr(taddr, 32 * warp, c0), v);
      const int row = 32 * warp + lane;
      for (int q = 0; q < 32; ++q)
        if (c0 + q < N) D[row * N + c0 + q] = v[q];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(taddr, ncols);
}

// The shifted-row product of the periodic convolutions (rescnn_tc.cu):
//   D [128 x 16] = sum_t A[base + off_t .. base + off_t + 127] B_t^T,
// A [n_rows x 16] BF16 staged as two 16-byte planes (channels 0-7 and 8-15, one 16-byte row
// per A row), each B_t [16 x 16] as two 8-channel core-matrix columns; no-swizzle descriptors.
// The shared-memory block is 96 KB, so that every address any reading of the two strides
// could produce stays inside it (n_rows <= 256).
constexpr int SHIFT_SMEM = 96 * 1024;
__global__ void __launch_bounds__(128) tc_shift_selftest_kernel(const uint16_t *__restrict__ A, int n_rows,
                                                                const uint16_t *__restrict__ B, int n_taps,
                                                                int4 offs0, int4 offs1, int base, float *D,
                                                                int *status) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  unsigned char *planes = smem_dyn;                   // [2][n_rows][16 B]
  unsigned char *sB = smem_dyn + 2 * n_rows * 16;     // [tap][2][16 rows][16 B]
  for (int i = threadIdx.x; i < SHIFT_SMEM / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(smem_dyn)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int idx = threadIdx.x; idx < n_rows * 16; idx += blockDim.x) {
    const int r = idx / 16, c = idx % 16;
    *reinterpret_cast<uint16_t *>(planes + (c / 8) * n_rows * 16 + r * 16 + (c % 8) * 2) = A[idx];
  }
  for (int idx = threadIdx.x; idx < n_taps * 256; idx += blockDim.x) {
    const int t = idx / 256, n = (idx / 16) % 16, k = idx % 16;
    *reinterpret_cast<uint16_t *>(sB + t * 512 + (k / 8) * 256 + n * 16 + (k % 8) * 2) = B[idx];
  }
  tc::fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&tmem_base, 32);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  if (threadIdx.x == 0) {
    const int offs[8] = {offs0.x, offs0.y, offs0.z, offs0.w, offs1.x, offs1.y, offs1.z, offs1.w};
    for (int t = 0; t < n_taps; ++t) {
      const uint64_t ad = tc::desc_noswz(smem_addr(planes + (base + offs[t]) * 16), n_rows * 16, 128);
      const uint64_t bd = tc::desc_noswz(smem_addr(sB + t * 512), 256, 128);
      tc::mma_bf16(taddr, ad, bd, tc::idesc_bf16_f32(128, 16), t > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, 1u << 22);
  if (!ok && threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
  tc::fence_after_sync();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ok) {
    float v[16];
    tc::tmem_ld16(tc::tmem_lane_addr(taddr, 32 * warp, 0), v);
    for (int q = 0; q < 16; ++q) D[(32 * warp + lane) * 16 + q] = v[q];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(taddr, 32);
}

}  // namespace
}  // namespace nqs

extern "C" nqs_status nqs_selftest_tc_shift(const uint16_t *A, int32_t n_rows, const uint16_t *B, int32_t n_taps,
                                            const int32_t *offs, int32_t base, float *D, int32_t *status,
                                            nqs_stream stream) {
  if (!A || !B || !offs || !D || !status || n_rows < 128 || n_rows > 256 || n_rows % 8 || n_taps < 1 || n_taps > 8)
    return NQS_EINVAL;
  int o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < n_taps; ++t) {
    o[t] = offs[t];
    if (base + o[t] < 0 || base + o[t] + 128 > n_rows) return NQS_EINVAL;
  }
  auto kern = nqs::tc_shift_selftest_kernel;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, nqs::SHIFT_SMEM) != cudaSuccess)
    return NQS_ECUDA;
  kern<<<1, 128, nqs::SHIFT_SMEM, reinterpret_cast<cudaStream_t>(stream)>>>(
      A, n_rows, B, n_taps, make_int4(o[0], o[1], o[2], o[3]), make_int4(o[4], o[5], o[6], o[7]), base, D, status);
  return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ECUDA;
}

extern "C" nqs_status nqs_selftest_tc_gemm(const uint16_t *A, const uint16_t *B, float *D, int32_t N, int32_t K,
                                           int32_t flags, int32_t *status, nqs_stream stream) {
  if (!A || !B || !D || !status || N < 16 || N > 256 || N % 16 || K < 64 || K > 256 || K % 64 || flags < 0 ||
      flags > 3)
    return NQS_EINVAL;
  // K-major B uses nkb tiles of N rows; MN-major B uses ceil(N/64) groups of K rows: take the larger
  const size_t b_bytes = std::max((size_t)(K / 64) * N * 128, (size_t)((N + 63) / 64) * K * 128);
  const size_t shm = 1024 + (size_t)(K / 64) * 128 * 128 + b_bytes;
  auto kern = nqs::tc_gemm_selftest_kernel;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
    return NQS_ECUDA;
  kern<<<1, 128, shm, reinterpret_cast<cudaStream_t>(stream)>>>(A, B, D, N, K, flags, status);
  return cudaGetLastError() == cudaSuccess ? NQS_OK : NQS_ECUDA;
}
