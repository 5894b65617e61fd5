// Shared definitions of the ResCNN kernels (App. H): parameter layout in kernel order and the
// launch arguments.  rescnn.cu holds the FP32 copy on the CUDA cores, rescnn_tc.cu the 16-bit
// copies on the tensor cores.
#pragma once
#include <cstdint>

#include "internal.h"

namespace nqs {
namespace cnn {

constexpr int CF = 16;            // filters
constexpr int MAX_BLOCKS = 8;     // residual blocks
constexpr int CN_THREADS = 512;   // FP32 path: rows (configuration x site) per CTA
constexpr float LN_EPS = 1e-6f;
constexpr float GELU_C = 0.7978845608028654f;  // sqrt(2 / pi)

// per residual block, in floats: gamma, beta, K1 (9 x 16 x 16), b1, K2, b2
constexpr int OFF_G = 0, OFF_BE = CF, OFF_K1 = 2 * CF, OFF_B1 = OFF_K1 + 9 * CF * CF, OFF_K2 = OFF_B1 + CF,
              OFF_B2 = OFF_K2 + 9 * CF * CF, BLOCK_FLOATS = OFF_B2 + CF;

__host__ __device__ constexpr int n_params(int n_blocks) { return 10 * CF + n_blocks * BLOCK_FLOATS + 2 * CF; }

struct CnnArgs {
  const float *cw;  // kernel-order FP32 parameters of the copy
  int N, W, Lx, Ly, n_blocks;
  int G;     // configurations per CTA group
  int rows;  // threads per CTA
  // evaluation modes
  const uint32_t *cfg;
  int64_t n_cfg;
  float *out;
  // sweep
  uint32_t *state;
  int64_t C;
  int n_sweeps, burn_in;
  uint32_t sweep_offset, k0, k1;
  uint32_t *samples;
  float *logpsi;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
};

}  // namespace cnn

// 16-bit (BF16 / F16) copies on the tensor cores (rescnn_tc.cu)
bool rescnn_lp_supported(const nqs_ctx *c);
cudaError_t rescnn_lp_alloc(nqs_ctx *c);
void rescnn_lp_free(nqs_ctx *c);
cudaError_t rescnn_lp_prepare(nqs_ctx *c, const double *params, cudaStream_t s);
cudaError_t rescnn_lp_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
// log psi of the N + 1 local-energy configurations of each of n samples into out [n (N + 1)]
cudaError_t rescnn_lp_eval_flips(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
cudaError_t rescnn_lp_sweep(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int burn_in, uint64_t seed,
                            uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc,
                            uint32_t *acc_bits, float *delta, cudaStream_t s);

}  // namespace nqs
