// nqs_force_noalloc: the force of nqs_logpsi_grad for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or have torch allocate) at the point where
// they need the force: code that runs inside another framework's memory budget,
// plugins whose host forbids allocation after start-up, or real-time loops that
// must not hit the allocator.  This entry point needs no workspace argument: its
// scratch is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES that every GPU
// loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB of FP64 partial sums
constexpr int MAX_DEVICES = 64;

// The scratch.  In host code this name is only a stand-in for the device symbol, never a
// device address: kernels receive the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) double g_force_scratch[NOALLOC_SCRATCH_BYTES / sizeof(double)];

std::mutex g_mu;
double *g_scratch_addr[MAX_DEVICES] = {};

// Resolves the device address of the scratch on the current device, once per device.
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_force_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" nqs_status nqs_force_noalloc(nqs_ctx *c, const uint32_t *configs, int64_t n, const float *eloc,
                                        const double *stats, double *force, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  auto fail = [&](nqs_status st, const std::string &m) {
    c->err = m;
    return st;
  };
  if (!c->params_set) return fail(NQS_EINVAL, "nqs_force_noalloc: parameters not set");
  if (c->model_kind != NQS_RBM) return fail(NQS_EUNSUPPORTED, "nqs_force_noalloc: RBM contexts only");
  if (n < 0 || !force) return fail(NQS_EINVAL, "nqs_force_noalloc: needs n >= 0 and a non-null force");
  if (n == 0) {  // as nqs_logpsi_grad: the force of no rows is zero
    const cudaError_t z = cudaMemsetAsync(force, 0, (size_t)c->P * sizeof(double),
                                          reinterpret_cast<cudaStream_t>(stream));
    return z == cudaSuccess ? NQS_OK : fail(NQS_ECUDA, std::string("nqs_force_noalloc: ") + cudaGetErrorString(z));
  }
  if (!configs || !eloc || !stats)
    return fail(NQS_EINVAL, "nqs_force_noalloc: needs non-null configs, eloc and stats when n > 0");
  const size_t per_chunk = (size_t)c->P * sizeof(double);
  if (per_chunk > NOALLOC_SCRATCH_BYTES)
    return fail(NQS_EINVAL, "nqs_force_noalloc: the model has more than 4,194,304 parameters, beyond the "
                            "32 MiB built-in scratch; use nqs_logpsi_grad with a workspace");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device)
    return fail(NQS_EINVAL, "nqs_force_noalloc: the context's device must be the current device");
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return fail(NQS_ECUDA, std::string("nqs_force_noalloc: cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
  // The kernel wants about 2 * SMs / ceil(M / 32) chunks of P doubles.  Within the RBM's limits
  // (N <= 256, M <= 1024, so P <= 257 M + 256) that stays below the scratch's capacity of
  // 4,194,304 / P chunks; the clamp only guards a future change of those limits.
  int chunks = nqs::rbm_force_chunks(c, n);
  const int cap = (int)(NOALLOC_SCRATCH_BYTES / per_chunk);
  if (chunks > cap) chunks = cap;
  // Every entry of the chunks used is overwritten before it is read, so nothing left by
  // an earlier call needs clearing.
  e = nqs::rbm_force_into(c, configs, n, eloc, stats, force, scratch, chunks, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : fail(NQS_ECUDA, std::string("nqs_force_noalloc: ") + cudaGetErrorString(e));
}
