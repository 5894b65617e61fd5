// Host-side context and the launchers each kernel file exports to the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nqs.h"

struct nqs_ctx {
  int model_kind = NQS_RBM;
  int ham_kind = NQS_TFIM;
  nqs_dtype dtype = NQS_F32;
  int N = 0;  // sites
  int W = 0;  // words per packed configuration
  int Lx = 0, Ly = 1;
  double J1 = 1.0, J2 = 0.0, h = 0.0;
  int marshall = 0;
  int64_t P = 0;  // parameters
  int refresh = 20;
  int chains_per_warp = 0;  // 0: tuner
  int device = 0;
  int num_sms = 0;
  int smem_optin = 0;
  int *d_status = nullptr;    // sticky device status word
  double *d_scratch = nullptr;  // per-block partials of the statistics reduction
  bool params_set = false;

  // Hamiltonian bond list; exchange moves draw a uniform bond from it.
  int n_bonds = 0;
  int2 *d_bonds = nullptr;
  float *d_bondJ = nullptr;

  // RBM sampling copy.  Hidden units are padded to M_pad = L * E (L lanes per
  // chain, E units per lane) with W = b = 0, so padded units contribute nothing.
  int M = 0, M_pad = 0;
  float *d_a = nullptr;     // [N] rounded visible bias
  float *d_b = nullptr;     // [M_pad] rounded hidden bias
  float *d_Wt = nullptr;    // [N][M_pad] rounded weights, site-major (W^T)
  void *d_R = nullptr;      // [N][M_pad] exp(-4 W) in the sampling dtype
  float2 *d_aK = nullptr;   // [N] (a_i, sum_j W_ji)
  // FP32 rounding of the master for the local energy (Sec. 4.2: the low-precision copy is
  // used only for sampling).  For an F32 context these alias the tables above.
  float *d_a32 = nullptr, *d_b32 = nullptr, *d_Wt32 = nullptr, *d_R32 = nullptr;
  float2 *d_aK32 = nullptr;
  float *d_Wm = nullptr;    // [N][M] FP32 master weights, site-major (gradients)
  float *d_bm = nullptr;    // [M] FP32 master hidden bias (gradients)

  std::string err;
};

namespace nqs {

constexpr int MPAD_ALIGN = 32;  // M_pad is a multiple of this, so 8, 16 or 32 lanes divide it
constexpr int STATS_MAX_BLOCKS = 1024;
// Sticky device status bits (read by nqs_check_status).
constexpr int STATUS_RANGE = 1;    // a value left the documented range
constexpr int STATUS_TIMEOUT = 2;  // a bounded wait gave up

// rbm.cu
cudaError_t rbm_prepare(nqs_ctx *c, const double *params, cudaStream_t s);
cudaError_t init_chains(const nqs_ctx *c, uint32_t *state, int64_t n, uint64_t seed, cudaStream_t s);
cudaError_t rbm_sweep(const nqs_ctx *c, uint32_t *state, int64_t n_chains, int n_sweeps, int burn_in,
                      uint64_t seed, uint32_t sweep_offset, uint32_t *samples, float *logpsi,
                      int64_t *n_acc, uint32_t *acc_bits, float *delta, cudaStream_t s);
cudaError_t rbm_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
cudaError_t rbm_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s);
size_t rbm_grad_workspace(const nqs_ctx *c, int64_t n);
cudaError_t rbm_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                            const double *stats, double *force, void *ws, cudaStream_t s);
bool rbm_supported(const nqs_ctx *c, std::string *why);
cudaError_t rbm_flip_delta(const nqs_ctx *c, const uint32_t *cfg, const int32_t *sites, int64_t n, float *out,
                           cudaStream_t s);
namespace rbmk {
struct SweepParams;
struct ElocParams;
}  // namespace rbmk
// rbm_f16.cu, rbm_bf16.cu
cudaError_t rbm_sweep_f16(const nqs_ctx *c, const rbmk::SweepParams &p, cudaStream_t s);
cudaError_t rbm_eloc_f16(const nqs_ctx *c, const rbmk::ElocParams &p, cudaStream_t s);
cudaError_t rbm_sweep_bf16(const nqs_ctx *c, const rbmk::SweepParams &p, cudaStream_t s);
cudaError_t rbm_eloc_bf16(const nqs_ctx *c, const rbmk::ElocParams &p, cudaStream_t s);
int rbm_force_chunks(const nqs_ctx *c, int64_t n);
// force_tc.cu
bool rbm_force_tc_supported(const nqs_ctx *c);
int rbm_force_tc_chunks(const nqs_ctx *c, int64_t n);
cudaError_t rbm_force_tc(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                         double *ws, int chunks, cudaStream_t s);
cudaError_t rbm_force_into(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                           double *force, double *scratch, int chunks, cudaStream_t s);

// stats.cu
cudaError_t energy_stats(const nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains,
                         const int64_t *n_acc, int64_t proposals_per_chain, double *out, cudaStream_t s);

}  // namespace nqs
