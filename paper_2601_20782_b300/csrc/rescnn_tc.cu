// ResCNN (App. H) 16-bit sampling copies on the tensor cores.
#include "rescnn.cuh"

namespace nqs {

bool rescnn_lp_supported(const nqs_ctx *) { return false; }
cudaError_t rescnn_lp_alloc(nqs_ctx *) { return cudaErrorNotSupported; }
void rescnn_lp_free(nqs_ctx *) {}
cudaError_t rescnn_lp_prepare(nqs_ctx *, const double *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t rescnn_lp_logpsi(const nqs_ctx *, const uint32_t *, int64_t, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t rescnn_lp_eval_flips(const nqs_ctx *, const uint32_t *, int64_t, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t rescnn_lp_sweep(const nqs_ctx *, uint32_t *, int64_t, int, int, uint64_t, uint32_t, uint32_t *, float *,
                            int64_t *, uint32_t *, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace nqs
