// Device helpers shared by the kernels: Philox4x32-10, warp reductions,
// explicit-rounding PTX wrappers, bounded mbarrier waits and 1D bulk copies.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nqs {

constexpr uint32_t FULL_MASK = 0xffffffffu;
constexpr uint32_t TAG_SWEEP = 0x53574550u;  // "SWEP"
constexpr uint32_t TAG_INIT = 0x494E4954u;   // "INIT"
constexpr float LN2F = 0.693147180559945309f;
constexpr float LOG2EF = 1.442695040888963407f;  // 1 / ln 2

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// products by 0xD2511F53 / 0xCD9E8D57, a swap and an xor with the round key;
// the key is bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Multiply-shift map of a word onto {0..n-1}: (w * n) >> 32.
__device__ __forceinline__ uint32_t index_from_word(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// Butterfly all-reduce over `width` lanes (a power of two dividing 32): every
// lane of a group ends with the bitwise-identical sum, because each stage adds
// the same two operands on both partner lanes.
template <int WIDTH = 32>
__device__ __forceinline__ float group_allsum(float v) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}
template <int WIDTH = 32>
__device__ __forceinline__ double group_allsum(double v) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

// Explicit MUFU forms, so that the result does not depend on global fast-math flags.
__device__ __forceinline__ float lg2_approx(float x) {  // log2; subnormal inputs give -inf
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {  // 2^x
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- mbarrier + 1D bulk copy (TMA) --------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// 1D bulk global->shared copy; dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after max_iter polls (each try_wait suspends for a
// hardware-chosen interval) and reports false; the caller records STATUS_TIMEOUT.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t max_iter) {
  for (uint32_t it = 0; it < max_iter; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

}  // namespace nqs
