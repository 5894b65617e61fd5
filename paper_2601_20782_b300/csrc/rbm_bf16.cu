// Sweep and local-energy kernels of the RBM with a BF16 sampling copy (its own
// translation unit so that the per-dtype instantiations compile in parallel).
#include "rbm_core.cuh"

namespace nqs {

cudaError_t rbm_sweep_bf16(const nqs_ctx *c, const rbmk::SweepParams &p, cudaStream_t s) {
  return rbmk::dispatch_l32<rbmk::Runners<__nv_bfloat16>::Sweep>(c->M_pad / 32, c, p, s);
}

cudaError_t rbm_eloc_bf16(const nqs_ctx *c, const rbmk::ElocParams &p, cudaStream_t s) {
  return rbmk::dispatch_l32<rbmk::Runners<__nv_bfloat16>::Eloc>(c->M_pad / 32, c, p, s);
}

}  // namespace nqs
