// Host-side context and the launchers each kernel file exports to the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

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
  int dense_fused = 1;       // dense sampler: the persistent fused kernel where it applies (NQS_OPT_DENSE_FUSED)
  double noise_sigma = 0.0;  // noisy RBM (nqs_set_noise): 0 = off
  int renorm = 1;            // RBM sweep: accepted flips between cache normalisations (set_params)
  float *d_bounds = nullptr; // RBM: [max |W|, max_j (sum_i |W_ji| + |b_j|)] of the sampling copy
  uint64_t noise_key = 0;
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

  // ---- dense ansatz: widths H[0..L-1]; layer l >= 1 is a tensor-core GEMM --------------
  int L = 0;
  std::vector<int> H, Kp;          // Kp[l]: padded input width of layer l (Kp[0] unused)
  float *d_W1t = nullptr;          // [N][H0] FP32 sampling-copy layer-1 weights, site-major
  float *d_W1d = nullptr;          // [n_bonds][H0] W1t[i_b] - W1t[j_b] per bond (fused exchange sampler)
  float *d_b1 = nullptr;           // [H0]
  std::vector<__nv_bfloat16 *> d_Wl;  // layer l >= 1: [H[l]][Kp[l]] BF16 sampling copy
  std::vector<float *> d_bl;       // layer l >= 1: [H[l]] bias (sampling copy, FP32 values)
  float *d_wout = nullptr;         // [H[L-1]]
  float b_out = 0.f;
  std::vector<CUtensorMap> mB0, mB1;  // per layer l >= 1
  std::vector<int> NR, p0, p1;        // per layer l >= 1: columns per CTA and the two MMA parts
  std::vector<CUtensorMap> mBs0, mBs1;  // split configuration (half-width ranges) for small row counts
  std::vector<int> NRs, p0s, p1s;
  float *d_master = nullptr;       // [P] FP32 master parameters (backward)
  // workspace for up to max_rows rows per pass
  int64_t max_rows = 0;
  __nv_bfloat16 *d_act[2] = {nullptr, nullptr};  // activations [max_rows][max Kp]
  float *d_part = nullptr;         // [max_rows][max ranges] DOT partials
  float *d_out = nullptr;          // [max_rows] log psi of the rows
  float *d_z1 = nullptr;           // [max_rows][H0] FP32 layer-1 pre-activations (per sample / chain)
  float *d_z1b = nullptr;          // [max_rows][H0] second buffer of the fused sampler (dense_fused.cu)
  float *d_lp = nullptr;           // [max_rows] log psi per sample / chain
  int32_t *d_prop = nullptr;       // [max_rows] proposed bond (or -1) per chain
  float *d_thr = nullptr;          // [max_rows] log u per chain
  // FP8 sampling copy (dtype NQS_FP8E4M3; the BF16 copy above then serves the local energy):
  // every weight matrix W_l in E4M3 scaled by a per-layer power of two s_l (max |W_l| s_l <= 448),
  // biases and w_out as in the BF16 copy, E4M3 activations between layers.
  std::vector<int> Kp8;             // layer l >= 1: padded input width, a multiple of 128
  std::vector<uint8_t *> d_Wl8;     // layer l >= 1: [H[l]][Kp8[l]] E4M3 of W_l s_l
  std::vector<CUtensorMap> mB0_8, mB1_8, mBs0_8, mBs1_8;
  float *d_W1t8 = nullptr;          // [N][H0] FP32 values of E4M3(W_0 s_0) / s_0, site-major
  float *d_scale8 = nullptr;        // [2 L]: s_l, then 1 / s_l
  unsigned *d_wmax8 = nullptr;      // [L] max |W_l| (FP32 bits)
  uint8_t *d_act8[2] = {nullptr, nullptr};  // E4M3 activations [max_rows][max Kp8]
  float *d_grad_scratch = nullptr; // O rows for the force when the caller gives none
  void *d_force_part = nullptr;    // FP64 force partials [slices][P]
  int grad_chunk = 0;

  // ---- ResCNN (App. H): n_blocks residual blocks of 16 filters -------------------------
  int n_blocks = 0;
  float *d_cw = nullptr;           // [P] FP32 copy in kernel order (rescnn.cu)
  float *d_cw_lp = nullptr;        // [P] FP32 values of the 16-bit copy in kernel order (rescnn_tc.cu)
  uint16_t *d_ctile = nullptr;     // 16-bit convolution B tiles (rescnn_tc.cu)
  float *d_clp = nullptr;          // [cnn_rows] log psi of local-energy configurations
  int64_t cnn_rows = 0;

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
int rbm_renorm_interval(const nqs_ctx *c, float max_w, float max_theta);
cudaError_t init_chains(const nqs_ctx *c, uint32_t *state, int64_t n, uint64_t seed, cudaStream_t s);
cudaError_t rbm_sweep(const nqs_ctx *c, uint32_t *state, int64_t n_chains, int n_sweeps, int burn_in,
                      uint64_t seed, uint32_t sweep_offset, uint32_t *samples, float *logpsi,
                      int64_t *n_acc, uint32_t *acc_bits, float *delta, cudaStream_t s);
cudaError_t rbm_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
cudaError_t rbm_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s);
cudaError_t rbm_local_energy_chains(const nqs_ctx *c, const uint32_t *cfg, int64_t n_chains, int64_t per_chain,
                                    float *eloc, cudaStream_t s);
size_t rbm_grad_workspace(const nqs_ctx *c, int64_t n);
// share = false: force = (1/n) sum_x O(x) (eps(x) - stats[0]); share = true: divided by stats[4]
cudaError_t rbm_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                            const double *stats, double *force, void *ws, cudaStream_t s, bool share = false);
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
// the complex-parameter RBM's force on the same products (force_tc.cu): partial forces per row
// chunk into part [chunks][P], then their fixed-order sum x 1/n into force [P]
int crbm_force_tc_chunks(int M, int num_sms, int64_t n);
cudaError_t crbm_force_tc(const uint32_t *cfg, int64_t n, int N, int W, int M, int M_pad, int64_t P, const float2 *Wt,
                          const float2 *b, const float *eloc_re, const float *eloc_im, const double *stats,
                          double2 *part, int chunks, double2 *force, int *status, cudaStream_t s);
cudaError_t rbm_force_into(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                           double *force, double *scratch, int chunks, cudaStream_t s);

// dense.cu
bool dense_setup(nqs_ctx *c, const nqs_model_desc *m, std::string *why);
void dense_free(nqs_ctx *c);
cudaError_t dense_alloc_rows(nqs_ctx *c, int64_t rows);
cudaError_t dense_alloc_params(nqs_ctx *c);
cudaError_t dense_prepare(nqs_ctx *c, const double *params, cudaStream_t s);
cudaError_t dense_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
cudaError_t dense_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s);
cudaError_t dense_sweep(const nqs_ctx *c, uint32_t *state, int64_t n_chains, int n_sweeps, int burn_in, uint64_t seed,
                        uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc, uint32_t *acc_bits,
                        float *delta, cudaStream_t s);
cudaError_t dense_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                              const double *stats, double *force, cudaStream_t s, bool share = false);
// dense_fused.cu
bool dense_fused_supported(const nqs_ctx *c);
// per-bond differences of the layer-0 weights for the fused exchange sampler (after dense_prepare)
cudaError_t dense_fused_prepare(const nqs_ctx *c, cudaStream_t s);
cudaError_t dense_fused_sweeps(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int t0, int t1,
                               int burn_in, uint64_t seed, uint32_t sweep_offset, uint32_t *samples, float *logpsi,
                               int64_t *n_acc, uint32_t *acc_bits, float *delta, bool add_acc, cudaStream_t s);
// rescnn.cu
bool rescnn_setup(nqs_ctx *c, const nqs_model_desc *m, std::string *why);
cudaError_t rescnn_alloc(nqs_ctx *c);
void rescnn_free(nqs_ctx *c);
cudaError_t rescnn_prepare(nqs_ctx *c, const double *params, cudaStream_t s);
cudaError_t rescnn_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s);
cudaError_t rescnn_local_energy(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, cudaStream_t s);
// O rows (and the force) of the ResCNN from the FP32 copy; n_rows_max: rows of O per launch without O
bool rescnn_grad_supported(const nqs_ctx *c);
cudaError_t rescnn_logpsi_grad(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                               const double *stats, double *force, cudaStream_t s, bool share = false);
// F_k (+)= sum_x O[x][k] (eloc[x] - E) / n over rows of O [rows x P] (fixed-order FP64 sums; the
// context's d_force_part holds the partials); share: divide by stats[4] (multi-rank step)
cudaError_t force_rows(const nqs_ctx *c, const float *O, int64_t rows, const float *eloc, const double *stats,
                       int64_t n_total, bool share, int accumulate, double *force, cudaStream_t s);
cudaError_t rescnn_sweep(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int burn_in, uint64_t seed,
                         uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc, uint32_t *acc_bits,
                         float *delta, cudaStream_t s);
// dense_gemm.cu
bool make_tmap_bf16_2d(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows);
bool make_tmap_u8_2d(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows);
// inv_scale == nullptr: BF16 operands and activations; otherwise E4M3 (FP8 sampling copy) with
// z = acc * (*inv_scale)
cudaError_t dense_gemm(const nqs_ctx *c, const void *A, int R, int Kpad, const CUtensorMap &mB0,
                       const CUtensorMap &mB1, int N, int NR, int p0, int p1, int mode, const float *bias,
                       const float *w, void *out_act, int ld_out, float *out_part, cudaStream_t s,
                       const float *inv_scale = nullptr, bool tall = false);

// minsr.cu
size_t minsr_workspace(const nqs_ctx *c, int64_t n);
cudaError_t minsr(const nqs_ctx *c, const float *O, int64_t n, const float *eloc, const double *stats, double lam,
                  double *dtheta, double *T_out, void *ws, cudaStream_t s);

// stats.cu
// moments == nullptr: out[5] = (E, Var, err, acceptance, n); otherwise the additive moments
// [8] of stats_finalize are written to `moments` and out is unused
cudaError_t energy_stats(const nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains,
                         const int64_t *n_acc, int64_t proposals_per_chain, double *out, cudaStream_t s,
                         double *moments = nullptr);
cudaError_t stats_finalize(const double *moments, double *out, cudaStream_t s);

}  // namespace nqs
