/*
 * nqs.h -- C ABI of the B300 (sm_103a) hot path of neural-quantum-state
 * variational Monte Carlo, after "Neural Quantum States in Mixed Precision"
 * (arXiv 2601.20782).
 *
 * One VMC step (Sec. 2: sample, then gradients; Sec. 4.2: two model copies)
 * maps onto these calls:
 *   nqs_set_params    FP64 master parameters -> sampling copy (Sec. 4.2, Table tab:precision)
 *   nqs_init_chains   random initial spin configurations
 *   nqs_sweep         Metropolis-Hastings sweeps over pi ~ |psi|^2 (Sec. 3.1)
 *   nqs_local_energy  eps(x) = sum_{x'} H(x,x') psi(x')/psi(x)       (App. I, Eq. local_energies)
 *   nqs_logpsi_grad   O_k(x) = d log psi / d theta_k and the force F  (App. I, Eq. forces)
 *   nqs_stats         FP64 energy mean / variance / error, acceptance (Sec. 2, Eq. loss)
 *
 * Conventions shared by every call
 *  - Spins are s_i in {-1,+1}.  A configuration is stored bit-packed in
 *    W = ceil(N/32) uint32 words: bit (i mod 32) of word i/32 is 1 iff s_i = +1.
 *  - Every array argument is a DEVICE pointer owned by the caller unless the
 *    comment says "host".  The library keeps no reference after the call returns.
 *  - Every call is asynchronous on the given stream (NULL = legacy default
 *    stream) unless it says it synchronises.  Calls on one context must not
 *    run concurrently on different streams.
 *  - Return value: NQS_OK, or an error code; nqs_last_error() gives the text.
 *    Arguments are validated on the host before anything is launched; a call
 *    that returns an error has launched nothing.  CUDA launch failures return
 *    NQS_ECUDA.  Device-side range violations (see nqs_set_params) and
 *    exhausted bounded waits set a sticky device status word read by
 *    nqs_check_status().
 *  - Parameter vectors are FP64 and flat:
 *      RBM   : [a (N) | b (M) | W (M x N, row-major, W[j*N + i])]           (App. G)
 *      dense : [W1 (H1 x N) | b1 | W2 (H2 x H1) | b2 | ... | w_out (H_L) | b_out]
 *    and rows of O use the same order.
 */
#ifndef NQS_H
#define NQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nqs_stream; /* identical to cudaStream_t */

typedef enum {
  NQS_OK = 0,
  NQS_EINVAL = 1,       /* bad argument (shape, pointer, range) */
  NQS_ECUDA = 2,        /* a CUDA runtime call failed */
  NQS_ENOMEM = 3,       /* device allocation at create time failed */
  NQS_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
  NQS_EUNSUPPORTED = 5  /* combination not implemented */
} nqs_status;

/* Arithmetic type of the sampling copy (Table tab:precision).  RBM: F32, BF16, F16.
 * Dense ansatz: BF16, or NQS_FP8E4M3, an extension beyond the paper's formats: every
 * weight matrix in E4M3 scaled by a per-layer power of two (max |W_l| s_l <= 448),
 * E4M3 activations between layers, biases and w_out as in the BF16 copy; the sampler
 * and nqs_logpsi run on that copy, nqs_local_energy on the BF16 copy. */
typedef enum { NQS_F32 = 0, NQS_BF16 = 1, NQS_F16 = 2, NQS_FP8E4M3 = 3 } nqs_dtype;

enum { NQS_RBM = 0, NQS_DENSE = 1, NQS_RESCNN = 2 };
enum { NQS_TFIM = 0, NQS_HEISENBERG = 1 };

/* Hamiltonian on a periodic Lx x Ly lattice (Ly == 1: chain of Lx sites; Lx >= 3,
 * Ly == 1 or Ly >= 3).  Site index i = x + Lx*y.
 *  TFIM       (Sec. 4.1, Eq. TFIM): J1 sum_<ij> sz sz + h sum_i sx.  Single-flip moves.
 *  HEISENBERG (App. E): J1 sum_<ij> s.s + J2 sum_<<ij>> s.s (Pauli matrices; J2 on the
 *             diagonal next-nearest bonds).  Exchange moves over a uniform bond;
 *             marshall != 0 multiplies psi by (-1)^(#up spins with x+y even). */
typedef struct {
  int32_t kind;
  int32_t Lx, Ly;
  double J1, J2, h;
  int32_t marshall;
} nqs_ham_desc;

/* Ansatz.  RBM (App. G): n_hidden = M (1 .. 1024); N <= 256 sites; sampling copy F32,
 * BF16 or F16; TFIM only.
 * DENSE: n_layers (2..8) hidden widths in widths[] (host array, copied; multiples of
 * 16), a_1 = log cosh(W1 s + b1), a_l = tanh(W_l a_{l-1} + b_l), log psi = w_out . a_L
 * + b_out; sampling copy BF16 or FP8 E4M3 (layers >= 2 on the tensor cores, FP32
 * accumulation);
 * TFIM (single flips) or HEISENBERG (exchange moves).  nqs_logpsi_grad of a dense
 * context is FP32 from the FP32 rounding of the master and needs no workspace.
 * RESCNN (App. H): n_hidden = 16 filters, n_layers = residual blocks (0 .. 8), widths unused;
 * h(0) = Conv(s), h(l+1) = h(l) + Conv[GELU(Conv(GELU(LN(h(l)))))], log psi = sum over sites
 * and channels of LN(h(n_layers)); 3 x 3 periodic cross-correlations with a bias per output
 * channel, LN over the 16 channels of a site (eps 1e-6, scale and shift per channel), GELU
 * in its tanh form.  Two-dimensional TFIM (Ly >= 3, N <= 512).  Parameter vector
 *   [K0 (16 x 1 x 3 x 3) | b0 | per block: gamma | beta | K1 (16 x 16 x 3 x 3) | b1 | K2 | b2 |
 *    final gamma | final beta]   (K[co][ci][dy][dx]; P = 192 + 4672 n_layers).
 * nqs_logpsi_grad / nqs_force_share of a ResCNN context: FP32 reverse pass on the CUDA cores
 * from the FP32 rounding of the master, one CTA per configuration; needs no workspace;
 * NQS_EUNSUPPORTED when the residual streams of one configuration ((n_layers + 1) N 16 floats
 * beside the parameters) exceed shared memory.
 * Sampling copy F32 (CUDA cores), or BF16 / F16 with the convolutions as tcgen05 products:
 * kernels and the activations entering a convolution in the 16-bit type, biases, LN, the
 * residual stream, accumulation and the final sum in FP32; nqs_logpsi and nqs_local_energy
 * use the context's copy.  nqs_logpsi_grad and the force are not built for it. */
typedef struct {
  int32_t kind;
  int32_t n_hidden;
  int32_t n_layers;
  const int32_t *widths;
} nqs_model_desc;

typedef struct nqs_ctx nqs_ctx;

/* Creates a context on the current CUDA device and allocates its parameter
 * copies and tables (the only allocations the library makes).  Synchronous.
 * NQS_EUNSUPPORTED for model/Hamiltonian/dtype combinations not built. */
nqs_status nqs_create(nqs_ctx **out, const nqs_model_desc *model, const nqs_ham_desc *ham,
                      nqs_dtype sample_dtype);
void nqs_destroy(nqs_ctx *ctx);
/* Text of the last error on ctx (ctx may be NULL: last error of nqs_create). */
const char *nqs_last_error(const nqs_ctx *ctx);

int32_t nqs_n_sites(const nqs_ctx *ctx);           /* N */
int32_t nqs_words_per_config(const nqs_ctx *ctx);  /* W = ceil(N/32) */
int64_t nqs_n_params(const nqs_ctx *ctx);          /* P */
int32_t nqs_n_bonds(const nqs_ctx *ctx);           /* bonds of the Hamiltonian */

/* Tuning knobs.  NQS_OPT_REFRESH: the sweep recomputes its per-chain cache from
 * scratch every this many sweeps (default 20, >= 1).
 * NQS_OPT_CHAINS_PER_WARP: RBM sweep lanes per chain = 32 / value (1, 2 or 4;
 * 0 = chosen by the built-in rule).
 * NQS_OPT_MAX_ROWS: dense contexts only -- rows of one forward pass held in the
 * context's workspace (default 262144); bounds the chains of nqs_sweep and sets the
 * chunk of nqs_logpsi / nqs_local_energy.  Reallocates (synchronous).
 * NQS_OPT_DENSE_FUSED: dense contexts -- 1 (default): nqs_sweep of a BF16 or FP8 copy with
 * two hidden layers no wider than 448 runs the persistent fused sampler (a CTA owns a tile of
 * chains for all sweeps; proposal rows, the layer product on the tensor cores, log psi and
 * the decision in one kernel); 0: the multi-launch sampler (a producer kernel and the layer
 * GEMM per Metropolis step).  Same draws and decision rule; log psi sums in another order. */
enum { NQS_OPT_REFRESH = 0, NQS_OPT_CHAINS_PER_WARP = 1, NQS_OPT_MAX_ROWS = 2, NQS_OPT_DENSE_FUSED = 3 };
nqs_status nqs_set_option(nqs_ctx *ctx, int32_t option, int64_t value);

/* Sec. 4.2 (two-copy scheme): the FP64 master parameters (device, P doubles) are
 * rounded to the sampling dtype and the sampler's tables are rebuilt from the
 * rounded copy.  Range limits of the RBM sampler: |W| <= 20 (F16 tables:
 * |W| <= 2.5); a violation is reported.  Synchronises with the stream. */
nqs_status nqs_set_params(nqs_ctx *ctx, const double *params, nqs_stream stream);

/* Writes n_chains random configurations to state [n_chains x W]: i.i.d. uniform
 * spins for TFIM, a uniformly random zero-magnetisation configuration for
 * HEISENBERG (N even).  Drawn from Philox4x32-10 keyed by seed. */
nqs_status nqs_init_chains(nqs_ctx *ctx, uint32_t *state, int64_t n_chains, uint64_t seed,
                           nqs_stream stream);

/* Optional per-proposal record, for tests and bias studies (any member may be NULL).
 *  accept_bits [n_chains x n_sweeps x W]: bit p of the sweep's word block = proposal p accepted.
 *  delta       [n_chains x n_sweeps x N]: the log psi(y) - log psi(x) the sampler used. */
typedef struct {
  uint32_t *accept_bits;
  float *delta;
} nqs_sweep_trace;

/* Sec. 3.1: n_sweeps sweeps of N Metropolis-Hastings proposals on each chain,
 * accepting y with probability min{1, |psi(y)/psi(x)|^2}, decided as
 * u < exp(2 (log psi(y) - log psi(x))) with u uniform in [0,1) (u = 0 always accepts).
 * Proposal p of sweep t of chain c uses Philox4x32-10 counter
 * (p/2, sweep_offset + t, c, 0x53574550) under key (seed lo, seed hi): words
 * (0,1) for even p, (2,3) for odd p; site = (w * N) >> 32 (TFIM) or
 * bond = (w * n_bonds) >> 32 (HEISENBERG), u = (w' >> 8) * 2^-24.
 *  state     [n_chains x W]      in/out chain configurations.
 *  samples   [(n_sweeps-burn_in) x n_chains x W] or NULL: configuration after each
 *            sweep t >= burn_in, row (t - burn_in) * n_chains + c.
 *  logpsi    [(n_sweeps-burn_in) x n_chains] or NULL: FP32 log psi of those rows.
 *  n_accepted [n_chains] or NULL: accepted proposals of this call, per chain.
 *  trace     host struct or NULL. */
nqs_status nqs_sweep(nqs_ctx *ctx, uint32_t *state, int64_t n_chains, int32_t n_sweeps,
                     int32_t burn_in, uint64_t seed, uint32_t sweep_offset, uint32_t *samples,
                     float *logpsi, int64_t *n_accepted, const nqs_sweep_trace *trace,
                     nqs_stream stream);

/* log psi of n configurations (FP32 output; the sampling copy's parameters).
 * With marshall the value is log|psi|. */
nqs_status nqs_logpsi(nqs_ctx *ctx, const uint32_t *configs, int64_t n, float *out,
                      nqs_stream stream);

/* Sec. 3.1 (increment of a local proposal): out[x] = log psi(y) - log psi(x) for y =
 * configs[x] with site sites[x] flipped, evaluated exactly as nqs_sweep evaluates it for
 * that proposal (the sampling copy's arithmetic: FP32, or BF16/F16 factors with FP32
 * cache).  TFIM (single-flip) contexts.  Comparing two contexts on the same (x, site)
 * gives the reduced-precision error eps(x, y) of the log-density increment (x2).
 * sites: device int32 [n], 0 <= site < N (unchecked on the device). */
nqs_status nqs_flip_delta(nqs_ctx *ctx, const uint32_t *configs, const int32_t *sites, int64_t n, float *out,
                          nqs_stream stream);

/* App. I, Eq. local_energies: eloc[x] = sum_{x' in C(x)} H(x,x') psi(x')/psi(x), in FP32
 * with the FP32 rounding of the master parameters, whatever the context's sampling
 * dtype (Sec. 4.2: the low-precision copy is used only for sampling). */
nqs_status nqs_local_energy(nqs_ctx *ctx, const uint32_t *configs, int64_t n, float *eloc,
                            nqs_stream stream);

/* App. I, Eq. forces.  O [n x P] (FP32, or NULL) receives O_k(x) = d log psi(x)/d theta_k.
 * If force != NULL (FP64 [P]) it receives F_k = (1/n) sum_x O_k(x) (eloc[x] - E)
 * with E = stats[0] (device, as written by nqs_stats); eloc and stats are then
 * required when n > 0 (for n = 0 the force is set to zero).  workspace: device scratch of nqs_logpsi_grad_workspace(ctx, n) bytes
 * (may be NULL when force == NULL).  Gradients use the FP32 rounding of the
 * master parameters, not the sampling copy. */
size_t nqs_logpsi_grad_workspace(const nqs_ctx *ctx, int64_t n);
nqs_status nqs_logpsi_grad(nqs_ctx *ctx, const uint32_t *configs, int64_t n, float *O,
                           const float *eloc, const double *stats, double *force,
                           void *workspace, size_t workspace_bytes, nqs_stream stream);

/* Sec. 2 (Eq. loss) statistics in FP64 over n = K * n_chains sweep-major samples:
 * out[0] = mean of eloc, out[1] = variance (1/n), out[2] = error of the mean from
 * the per-chain means (std with ddof 1 over sqrt(n_chains)), out[3] = acceptance
 * rate sum(n_accepted) / (n_chains * proposals_per_chain) (0 if n_accepted is NULL),
 * out[4] = n.  out: device, 5 doubles. */
nqs_status nqs_stats(nqs_ctx *ctx, const float *eloc, int64_t n, int64_t n_chains,
                     const int64_t *n_accepted, int64_t proposals_per_chain, double *out,
                     nqs_stream stream);

/* Multi-rank step (chains split over processes, one per GPU; no paper passage: the
 * statistics of Sec. 2 Eq. loss and the force of App. I Eq. forces over the pooled samples).
 * nqs_stats_moments writes the additive moments of this rank's samples, moments[8] (device):
 *   [n, sum eloc, sum eloc^2, n_chains, sum_c m_c, sum_c m_c^2, sum n_accepted,
 *    n_chains * proposals_per_chain (0 if n_accepted is NULL)],  m_c the per-chain means.
 * Summing the moments of all ranks (an all-reduce SUM) and passing the sum to
 * nqs_stats_finalize gives out[5] exactly as nqs_stats gives it for all ranks' chains
 * together; with one rank the two calls equal nqs_stats.  Same argument checks as
 * nqs_stats; nqs_stats_finalize needs moments[0] > 0 (unchecked on the device). */
nqs_status nqs_stats_moments(nqs_ctx *ctx, const float *eloc, int64_t n, int64_t n_chains,
                             const int64_t *n_accepted, int64_t proposals_per_chain, double *moments,
                             nqs_stream stream);
nqs_status nqs_stats_finalize(const double *moments, double *out, nqs_stream stream);

/* App. I, Eq. forces, one rank's share: force[k] = (1 / stats[4]) sum_{x < n} O_k(x) (eloc[x] - stats[0])
 * with stats (device, 5 doubles) as nqs_stats_finalize writes them for the pooled samples
 * (global E and total count).  The shares of all ranks sum (all-reduce SUM) to the force of
 * the pooled samples, since every rank centres on the same E.  With one rank and stats
 * from nqs_stats this equals nqs_logpsi_grad's force.  With stats = (0, ., ., ., 1) and
 * eloc = g it is the vector-Jacobian product sum_x g_x O(x) of log psi.  Arguments,
 * workspace and errors as nqs_logpsi_grad with O = NULL; n = 0 sets force to zero. */
nqs_status nqs_force_share(nqs_ctx *ctx, const uint32_t *configs, int64_t n, const float *eloc,
                           const double *stats, double *force, void *workspace, size_t workspace_bytes,
                           nqs_stream stream);

/* No counterpart in the paper.  The force F of nqs_logpsi_grad (same arguments and
 * result, no O rows) for callers that cannot allocate device memory when they need
 * it: code running under another framework's memory budget, plugins whose host
 * forbids allocation after start-up, or loops that must never reach an allocator.
 * It takes no workspace: its scratch is a built-in 32 MiB device array that every
 * GPU loading this library keeps until the process exits, so models with more than
 * 4,194,304 parameters are rejected with NQS_EINVAL.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The context's device must be current.  All calls share
 * the one array, so calls whose kernels overlap on the GPU (different streams, or
 * different contexts on one device) race; serialise them.  n = 0 sets the force to zero
 * and returns NQS_OK, as nqs_logpsi_grad does; n < 0 or a NULL force (or NULL configs,
 * eloc or stats with n > 0) return NQS_EINVAL; dense contexts NQS_EUNSUPPORTED.
 * Allocates nothing. */
nqs_status nqs_force_noalloc(nqs_ctx *ctx, const uint32_t *configs, int64_t n, const float *eloc,
                             const double *stats, double *force, nqs_stream stream);

/* Issue-rate probe (no counterpart in the paper): the peak that the RBM kernels' ALU
 * roofline divides by is measured, not assumed.  Launches `blocks` x `threads` threads
 * (32 <= threads <= 512, a multiple of 32), each running 8 independent dependency chains of
 * one instruction for `iters` iterations:
 *   NQS_PROBE_FFMA   fma.rn.f32      (1 FP32 FMA per lane per instruction)
 *   NQS_PROBE_FFMA2  fma.rn.f32x2    (2 FP32 FMAs per lane)
 *   NQS_PROBE_FMUL2  mul.rn.f32x2    (2 FP32 multiplies per lane)
 *   NQS_PROBE_HFMA2  fma.rn.f16x2    (2 F16 FMAs per lane)
 *   NQS_PROBE_BFMA2  fma.rn.bf16x2   (2 BF16 FMAs per lane)
 *   NQS_PROBE_LG2    lg2.approx.f32  (1 MUFU op per lane, plus one FP32 add feeding it)
 *   NQS_PROBE_EX2    ex2.approx.f32  (1 MUFU op per lane, chained)
 * The caller times the launch on `stream`; instructions = blocks * threads * iters * 8.
 * sink: device float [blocks] (written only in a practically impossible case).  Bad sizes
 * or kind: NQS_EINVAL. */
enum { NQS_PROBE_FFMA = 0, NQS_PROBE_FFMA2 = 1, NQS_PROBE_FMUL2 = 2, NQS_PROBE_HFMA2 = 3, NQS_PROBE_BFMA2 = 4,
       NQS_PROBE_LG2 = 5, NQS_PROBE_EX2 = 6 };
nqs_status nqs_probe_alu(int32_t kind, int64_t blocks, int32_t threads, int64_t iters, float *sink,
                         nqs_stream stream);

/* Self-test of the tensor-core building block used by the contraction kernels (no
 * counterpart in the paper): D [128 x N] FP32 = A [128 x K] * B [N x K]^T in BF16 with FP32
 * accumulation, one CTA.  flags bit 0: A is passed transposed ([K x 128]) and staged
 * MN-major; bit 1: B is passed transposed ([K x N]) and staged MN-major; otherwise both
 * are row-major with K contiguous and staged K-major.  16 <= N <= 256 (multiple of 16),
 * 64 <= K <= 256 (multiple of 64).  *status (device int) gets the timeout bit if the MMA
 * never completed. */
nqs_status nqs_selftest_tc_gemm(const uint16_t *A, const uint16_t *B, float *D, int32_t N, int32_t K,
                                int32_t flags, int32_t *status, nqs_stream stream);

/* Self-test of the shifted-row product the periodic convolutions use (no counterpart in the
 * paper): D [128 x 16] FP32 = sum_{t < n_taps} A[base + offs[t] .. + 127] B_t^T with A
 * [n_rows x 16] and B [n_taps][16 x 16] BF16 (row-major, device), staged without swizzle as
 * two 8-channel planes; offs: host int32 [n_taps].  128 <= n_rows <= 256 (a multiple of 8),
 * 1 <= n_taps <= 8, every shifted window inside [0, n_rows); else NQS_EINVAL.  *status
 * (device int) gets the timeout bit if the product never completed. */
nqs_status nqs_selftest_tc_shift(const uint16_t *A, int32_t n_rows, const uint16_t *B, int32_t n_taps,
                                 const int32_t *offs, int32_t base, float *D, int32_t *status,
                                 nqs_stream stream);

/* nqs_local_energy of the samples nqs_sweep writes: samples [per_chain * n_chains x W],
 * sweep-major (row k * n_chains + c), eloc the same rows.  The values are those of
 * nqs_local_energy up to FP32 rounding: the RBM kernel walks each chain's samples in order
 * and updates its theta = W s + b only for the spins that changed since the chain's previous
 * sample (rebuilt from scratch every NQS_OPT_REFRESH samples), instead of rebuilding it for
 * every sample.  With fewer than 16 chains per SM it evaluates the samples as
 * nqs_local_energy does (one group per chain would leave the GPU idle).  Dense contexts
 * evaluate it as nqs_local_energy. */
nqs_status nqs_local_energy_chains(nqs_ctx *ctx, const uint32_t *samples, int64_t n_chains, int64_t per_chain,
                                   float *eloc, nqs_stream stream);

/* Noisy RBM (Sec. 4.1): from the next nqs_sweep on, the sampler targets |psi~|^2 with
 *   log psi~(x) = log psi(x) + zeta(x) / 2,  zeta(x) ~ N(0, sigma) held fixed per x,
 * so the sampled log-density is perturbed by exactly zeta(x) (standard deviation sigma).
 * zeta(x) = sigma z(x) with z from the configuration itself: Philox4x32-10 chained over the
 * packed words w_0 .. w_{W-1} (zero-padded to a multiple of 4), h = (0x4E4F4953, W, 0, 0),
 * per block of four words h = Philox(h XOR words; key lo, key hi); then Box-Muller on
 * u1 = ((h0 >> 8) + 1) 2^-24, u2 = (h1 >> 8) 2^-24: z = sqrt(-2 ln u1) cos(2 pi u2).
 * Only sampling is perturbed: logpsi outputs, local energies and gradients use psi.
 * sigma = 0 turns the noise off.  FP32 TFIM RBM contexts only (else NQS_EUNSUPPORTED);
 * 0 <= sigma <= 100.  The sampler then runs 32 lanes per chain. */
nqs_status nqs_set_noise(nqs_ctx *ctx, double sigma, uint64_t key);

/* Preconditioned force by the SR solve of App. I in its n x n ("minSR") form, with diagonal
 * shift lambda (App. I uses shifts of 1e-3 and 1e-1):
 *   Obar = (O - mean_x O) / sqrt(n), ebar = (eloc - E) / sqrt(n), E = stats[0],
 *   T = Obar Obar^T,  y = (T + lambda I)^-1 ebar,  dtheta = Obar^T y
 *     = (Obar^T Obar + lambda I)^-1 F  (push-through identity; F the force of nqs_logpsi_grad).
 *  O       [n x P] FP32 rows of nqs_logpsi_grad (P = nqs_n_params), row-major.
 *  eloc    [n] FP32; stats: device, stats[0] = E (nqs_stats over the same n rows).
 *  dtheta  [P] FP64 out.  T_out: [n x n] FP64 out (T without the shift), or NULL.
 *  workspace of nqs_minsr_workspace(ctx, n) bytes (holds the centred rows as three BF16
 *  terms, 6 n P bytes, and the FP64 n x n system).  2 <= n <= 8192, lambda > 0.
 * The Gram matrix runs on the tensor cores with every FP32 value split into three BF16
 * terms (six products, FP32 accumulation over 1024-wide K blocks, FP64 beyond); the
 * Cholesky factorisation and both triangular solves are FP64.  If T + lambda I is not
 * positive definite in FP64 the range bit of the status word is set (nqs_check_status). */
size_t nqs_minsr_workspace(const nqs_ctx *ctx, int64_t n);
nqs_status nqs_minsr(nqs_ctx *ctx, const float *O, int64_t n, const float *eloc, const double *stats, double lambda,
                     double *dtheta, double *T_out, void *workspace, size_t workspace_bytes, nqs_stream stream);

/* Reads and clears the sticky device status word (synchronises the stream).
 * NQS_OK, NQS_EINVAL (a value left the documented range) or NQS_ETIMEOUT. */
nqs_status nqs_check_status(nqs_ctx *ctx, nqs_stream stream);

/* ---- Batched uneven instances ------------------------------------------------------
 * Many independent TFIM problems (each its own context: lattice, N, M, h, sampling copy)
 * sampled by ONE persistent launch over a work list of (instance, block of chains),
 * largest work first.  The paper runs one problem at a time (Sec. 4.1 workloads); each
 * batched chain is the Markov chain nqs_sweep produces for that context with 32 lanes per
 * chain (F16 always; F32 with NQS_OPT_CHAINS_PER_WARP = 1), bit for bit: same proposals
 * (Philox key = the item's seed, sweep counter = sweep_offset + t), same arithmetic, same
 * outputs and layouts.
 *
 * Every item's context must be a TFIM RBM context with its parameters set, on one device,
 * and all items share one sampling dtype, F32 or F16 (else NQS_EINVAL / NQS_EUNSUPPORTED).
 * The batch keeps the item list (pointers included); contexts and buffers must outlive it.
 * A bounded wait that runs out sets the timeout bit of the item's context
 * (nqs_check_status). */
typedef struct nqs_batch nqs_batch;
typedef struct {
  nqs_ctx *ctx;
  uint32_t *state;         /* device [n_chains x W] chain state (nqs_init_chains), updated in place */
  int64_t n_chains;        /* 1 .. 2^32 - 1 */
  uint64_t seed;           /* Philox key of this instance's proposals */
  uint32_t *samples;       /* device [(n_sweeps - burn_in) * n_chains x W] sweep-major, or NULL */
  float *logpsi;           /* device, same rows, or NULL */
  int64_t *n_accepted;     /* device [n_chains], or NULL */
  uint32_t *accept_bits;   /* device [n_chains x n_sweeps x W] decisions as nqs_sweep_trace, or NULL */
  float *eloc;             /* nqs_batch_step: device [(n_sweeps - burn_in) * n_chains] local energies, or NULL */
  double *stats;           /* nqs_batch_step: device [5] as nqs_stats over eloc (needs eloc, n_accepted) */
  float *O;                /* nqs_batch_step: device [n_chains x P] O rows of the last sweep's samples, or NULL */
} nqs_batch_item;

/* Builds the work list for n_sweeps sweeps (burn_in of them not kept) per call.  One CTA
 * per SM; each warp runs one chain of the CTA's current item.  warps_per_cta > 0 fixes the
 * CTA width (F16: the register-capped kernel variant); 0 runs the autotuner: for every
 * kernel variant (F16: registers capped at 128 with up to 16 warps, or the widest case's
 * registers with up to 8 warps; F32: one) and candidate width (4 .. 24 warps, within the
 * variant's register limit) it times one sweep of every instance on scratch copies of the
 * chains with CUDA events on `stream`, and keeps the fastest (synchronises the stream; the
 * chains are not changed).  Allocates the work list and descriptors; the states must be
 * initialised. */
nqs_status nqs_batch_create(nqs_batch **out, const nqs_batch_item *items, int32_t n_items, int32_t n_sweeps,
                            int32_t burn_in, int32_t warps_per_cta, nqs_stream stream);

/* One persistent launch: n_sweeps sweeps of every instance (sweep counters sweep_offset ..
 * sweep_offset + n_sweeps - 1), writing each item's state, samples, logpsi, n_accepted
 * and accept_bits as nqs_sweep does.  Asynchronous. */
nqs_status nqs_batch_sweep(nqs_batch *b, uint32_t sweep_offset, nqs_stream stream);

/* The VMC step of every instance as one CUDA graph (captured on the first call, then
 * replayed): the batched sweep, then per instance the local energies of its samples
 * (nqs_local_energy), their statistics (nqs_stats, acceptance over n_sweeps * N proposals
 * per chain) and the O rows of the last sweep's samples (nqs_logpsi_grad).  Outputs that
 * are NULL in the item are skipped.  Asynchronous. */
nqs_status nqs_batch_step(nqs_batch *b, uint32_t sweep_offset, nqs_stream stream);

typedef struct {
  int32_t warps_per_cta, max_warps_per_cta, ctas;
  int32_t variant;         /* 0: F32; F16 with registers capped at 128 (1) or the widest case's (2) */
  int32_t n_work_items;
  int32_t n_staged;        /* instances whose table is staged in shared memory */
  int64_t stage_bytes;     /* dynamic shared memory per CTA */
  int32_t n_tuned;         /* autotuner candidates timed (<= 16) */
  int32_t tuned_variant[16];
  int32_t tuned_warps[16];
  float tuned_ms[16];      /* one sweep of every instance with that candidate */
} nqs_batch_info_t;
nqs_status nqs_batch_info(const nqs_batch *b, nqs_batch_info_t *info);
const char *nqs_batch_last_error(const nqs_batch *b);
void nqs_batch_destroy(nqs_batch *b);

/* ---- Complex-parameter RBM ------------------------------------------------------------
 * App. G with complex parameters a in C^N, b in C^M, W in C^{M x N}:
 *   log psi(s) = a . s + sum_j log cosh(theta_j),  theta = W s + b.
 * Sec. 2: the sampled density is |psi|^2, so proposals are decided on 2 Re(log psi(y) - log psi(x)).
 * TFIM (Sec. 4.1, single flips) on the periodic lattices of nqs_ham_desc, N <= 256 sites,
 * 1 <= n_hidden <= 512, FP32 arithmetic.  Parameters, O rows and the force are complex and
 * interleaved (re, im), in the real RBM's order [a (N) | b (M) | W (M x N, row-major)].
 * Configurations use the packed layout of the conventions above; arrays are device pointers
 * owned by the caller; calls are asynchronous on `stream` unless stated; errors as above
 * (nqs_crbm_last_error gives the text). */
typedef struct nqs_crbm nqs_crbm;

/* NQS_EUNSUPPORTED for a Hamiltonian other than TFIM, N > 256 or n_hidden > 512.  Synchronous. */
nqs_status nqs_crbm_create(nqs_crbm **out, const nqs_ham_desc *ham, int32_t n_hidden);
void nqs_crbm_destroy(nqs_crbm *c);
const char *nqs_crbm_last_error(const nqs_crbm *c);  /* c may be NULL: last nqs_crbm_create error */
int64_t nqs_crbm_n_params(const nqs_crbm *c);         /* P (complex parameters) */
int32_t nqs_crbm_words_per_config(const nqs_crbm *c); /* W = ceil(N/32) */
/* The sampler rebuilds its per-unit cache from theta every `refresh` sweeps (default 20);
 * nqs_crbm_local_energy_chains rebuilds theta every `refresh` samples of a chain. */
nqs_status nqs_crbm_set_refresh(nqs_crbm *c, int32_t refresh);

/* params: device, P complex values as 2P doubles (re, im).  Rounded to FP32; the sampler's
 * tables are built from the rounded copy.  Range of the sampler: |Re W_ji| <= 1 and
 * sum_i |Re W_ji| + |Re b_j| <= 10 for every j (NQS_EINVAL otherwise; parameters then
 * count as unset).  Synchronises with the stream. */
nqs_status nqs_crbm_set_params(nqs_crbm *c, const double *params, nqs_stream stream);

/* As nqs_init_chains for a TFIM context (i.i.d. uniform spins, Philox4x32-10 keyed by seed). */
nqs_status nqs_crbm_init_chains(nqs_crbm *c, uint32_t *state, int64_t n_chains, uint64_t seed, nqs_stream stream);

/* nqs_sweep's proposals, counters, layouts and decision rule (u < exp(2 Re(log psi(y) -
 * log psi(x))), u = 0 always accepts) with the complex psi.  trace->delta receives
 * Re(log psi(y) - log psi(x)).  There is no log psi output. */
nqs_status nqs_crbm_sweep(nqs_crbm *c, uint32_t *state, int64_t n_chains, int32_t n_sweeps, int32_t burn_in,
                          uint64_t seed, uint32_t sweep_offset, uint32_t *samples, int64_t *n_accepted,
                          const nqs_sweep_trace *trace, nqs_stream stream);

/* out [n x 2] FP32: (Re log psi, Im log psi) with Im the sum of principal arguments (defined
 * modulo 2 pi). */
nqs_status nqs_crbm_logpsi(nqs_crbm *c, const uint32_t *configs, int64_t n, float *out, nqs_stream stream);

/* App. I, Eq. local_energies with complex psi: eloc_re[x] + i eloc_im[x] =
 * J sum_<ij> s_i s_j + h sum_i psi(flip_i x) / psi(x), FP32, two planar arrays [n]. */
nqs_status nqs_crbm_local_energy(nqs_crbm *c, const uint32_t *configs, int64_t n, float *eloc_re, float *eloc_im,
                                 nqs_stream stream);

/* nqs_crbm_local_energy of the samples nqs_crbm_sweep writes: samples [per_chain * n_chains x W],
 * sweep-major (row k * n_chains + c), eloc_re / eloc_im the same rows.  The values are those of
 * nqs_crbm_local_energy up to FP32 rounding: a warp walks each chain's samples in order and
 * adds 2 s'_i W_i to theta = W s + b only for the spins that changed since the chain's
 * previous sample (rebuilt from scratch every nqs_crbm_set_refresh samples).  With fewer than
 * 16 chains per SM it evaluates the samples as nqs_crbm_local_energy does. */
nqs_status nqs_crbm_local_energy_chains(nqs_crbm *c, const uint32_t *samples, int64_t n_chains, int64_t per_chain,
                                        float *eloc_re, float *eloc_im, nqs_stream stream);

/* out: device, 6 doubles.  out[0..4] = nqs_stats over eloc_re (mean, variance, chain-blocked
 * error, acceptance, n); out[5] = mean of eloc_im (zero in expectation: H is Hermitian). */
nqs_status nqs_crbm_stats(nqs_crbm *c, const float *eloc_re, const float *eloc_im, int64_t n, int64_t n_chains,
                          const int64_t *n_accepted, int64_t proposals_per_chain, double *out, nqs_stream stream);

/* App. I, Eq. forces with the conjugated log-derivatives of the holomorphic log psi.
 * O [n x P] complex FP32 interleaved, or NULL: O_a = s, O_b = tanh theta, O_W[j][i] = tanh(theta_j) s_i.
 * force [P] complex FP64 interleaved, or NULL: F_k = (1/n) sum_x conj(O_k(x)) (eps(x) - E) with
 * E = stats[0] + i stats[5] (nqs_crbm_stats); dE/dRe theta_k = 2 Re F_k, dE/dIm theta_k = 2 Im F_k.
 * With N <= 127 the force runs on the tensor cores (theta and the contraction as products of
 * three-term BF16 splits, FP32 accumulation in TMEM, FP64 across row tiles), else on the CUDA
 * cores; either way the partial forces of the row chunks are added in a fixed order, so the
 * result does not depend on timing.  n = 0 sets it to zero. */
nqs_status nqs_crbm_logpsi_grad(nqs_crbm *c, const uint32_t *configs, int64_t n, float *O, const float *eloc_re,
                                const float *eloc_im, const double *stats, double *force, nqs_stream stream);

/* nqs_check_status for the complex RBM's status word. */
nqs_status nqs_crbm_check_status(nqs_crbm *c, nqs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
