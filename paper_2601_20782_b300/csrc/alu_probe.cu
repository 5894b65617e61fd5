// Issue-rate probe of the CUDA-core instructions the RBM kernels are built from.  It has no
// counterpart in the paper: it measures the peak that the sweep's ALU roofline divides by.
//
// Every thread runs PROBE_CHAINS independent dependency chains of one instruction for `iters`
// iterations (enough independent work to hide the pipe latency), then stores a value that
// depends on every chain so that nothing is removed.  The caller times the launch and divides
// threads * iters * PROBE_CHAINS * (operations per instruction) by the time.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int PROBE_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(512) alu_probe_kernel(int64_t iters, float seed, float *sink) {
  float x[PROBE_CHAINS], y[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) {
    x[k] = seed + 1e-3f * (float)(threadIdx.x + k);
    y[k] = 1e-7f * (float)k;
  }
  const float a = 0.9999999f, b = 1e-7f;
  for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
      if constexpr (KIND == NQS_PROBE_FFMA) {  // x = x a + b, one FP32 FMA per lane
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[k]) : "f"(a), "f"(b));
      } else if constexpr (KIND == NQS_PROBE_FFMA2) {  // two FP32 FMAs per lane in one instruction
        asm volatile(
            "{\n .reg .b64 r, m, c;\n mov.b64 r, {%0, %1};\n mov.b64 m, {%2, %2};\n mov.b64 c, {%3, %3};\n"
            " fma.rn.f32x2 r, r, m, c;\n mov.b64 {%0, %1}, r;\n}"
            : "+f"(x[k]), "+f"(y[k])
            : "f"(a), "f"(b));
      } else if constexpr (KIND == NQS_PROBE_FMUL2) {  // two FP32 multiplies per lane
        asm volatile(
            "{\n .reg .b64 r, m;\n mov.b64 r, {%0, %1};\n mov.b64 m, {%2, %2};\n"
            " mul.rn.f32x2 r, r, m;\n mov.b64 {%0, %1}, r;\n}"
            : "+f"(x[k]), "+f"(y[k])
            : "f"(a));
      } else if constexpr (KIND == NQS_PROBE_HFMA2) {  // two F16 FMAs per lane
        uint32_t &h = reinterpret_cast<uint32_t &>(x[k]);
        asm volatile("fma.rn.f16x2 %0, %0, %1, %2;" : "+r"(h) : "r"(0x3BFF3BFFu), "r"(0x00010001u));
      } else if constexpr (KIND == NQS_PROBE_BFMA2) {  // two BF16 FMAs per lane
        uint32_t &h = reinterpret_cast<uint32_t &>(x[k]);
        asm volatile("fma.rn.bf16x2 %0, %0, %1, %2;" : "+r"(h) : "r"(0x3F7F3F7Fu), "r"(0x00010001u));
      } else if constexpr (KIND == NQS_PROBE_LG2) {  // MUFU log2 (with one FP32 add feeding it)
        x[k] += 1.0f;
        float l;
        asm volatile("lg2.approx.f32 %0, %1;" : "=f"(l) : "f"(x[k]));
        y[k] += l;
      } else {  // NQS_PROBE_EX2: MUFU 2^x, chained (2^-x stays in (0.5, 1] for x in [0, 1])
        asm volatile("ex2.approx.f32 %0, %0;" : "+f"(x[k]));
        x[k] = -x[k];
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k] + y[k];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // practically never true; keeps the chains live
}

template <int KIND>
cudaError_t launch_probe(int64_t blocks, int threads, int64_t iters, float *sink, cudaStream_t s) {
  alu_probe_kernel<KIND><<<(unsigned)blocks, threads, 0, s>>>(iters, 0.5f, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" nqs_status nqs_probe_alu(int32_t kind, int64_t blocks, int32_t threads, int64_t iters, float *sink,
                                    nqs_stream stream) {
  if (blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 512 || threads % 32 || iters < 1 || !sink)
    return NQS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (kind) {
    case NQS_PROBE_FFMA: e = launch_probe<NQS_PROBE_FFMA>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_FFMA2: e = launch_probe<NQS_PROBE_FFMA2>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_FMUL2: e = launch_probe<NQS_PROBE_FMUL2>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_HFMA2: e = launch_probe<NQS_PROBE_HFMA2>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_BFMA2: e = launch_probe<NQS_PROBE_BFMA2>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_LG2: e = launch_probe<NQS_PROBE_LG2>(blocks, threads, iters, sink, s); break;
    case NQS_PROBE_EX2: e = launch_probe<NQS_PROBE_EX2>(blocks, threads, iters, sink, s); break;
    default: return NQS_EINVAL;
  }
  return e == cudaSuccess ? NQS_OK : NQS_ECUDA;
}
