// Sweep and local-energy kernels of the RBM with a F16 sampling copy (its own
// translation unit so that the per-dtype instantiations compile in parallel).
#include "rbm_core.cuh"

namespace nqs {

cudaError_t rbm_sweep_f16(const nqs_ctx *c, const rbmk::SweepParams &p, cudaStream_t s) {
  return rbmk::dispatch_l32<rbmk::Runners<__half>::Sweep>(c->M_pad / 32, c, p, s);
}

cudaError_t rbm_eloc_f16(const nqs_ctx *c, const rbmk::ElocParams &p, cudaStream_t s) {
  return rbmk::dispatch_l32<rbmk::Runners<__half>::Eloc>(c->M_pad / 32, c, p, s);
}

}  // namespace nqs
