// Instantiation of the persistent batched sweep kernel (batch_kernel.cuh).
#include "batch_kernel.cuh"

namespace nqs {
namespace batchk {
const void *batch_kernel_f16_wide() { return reinterpret_cast<const void *>(rbm_batch_sweep_kernel<__half, 0>); }
}  // namespace batchk
}  // namespace nqs
