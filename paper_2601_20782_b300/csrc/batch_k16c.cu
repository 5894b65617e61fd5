// Instantiation of the persistent batched sweep kernel (batch_kernel.cuh).
#include "batch_kernel.cuh"

namespace nqs {
namespace batchk {
const void *batch_kernel_f16_capped() {
  return reinterpret_cast<const void *>(rbm_batch_sweep_kernel<__half, BATCH_CAPPED_THREADS>);
}
}  // namespace batchk
}  // namespace nqs
