// Persistent Metropolis sampler of the dense ansatz with one tensor-core layer (two hidden
// layers: a1 = log cosh(W1 s + b1), a2 = tanh(W2 a1 + b2), log psi = w_out . a2 + b_out; the
// BF16 sampling copy, or the FP8 copy: E4M3 a1 and W2 s2 with z2 = acc / s2, layer 0 on the
// E4M3-rounded W1), for layer widths up to 448.
//
// A CTA owns a tile of R <= 128 chains for all the sweeps of one launch; chains are
// independent, so CTAs never wait on one another.  Each Metropolis step:
//   1. moves: a thread per chain takes the move drawn during the previous step's products and
//      looks up its spins (an exchange of equal spins is the identity, not evaluated);
//   2. proposal rows: a warp per chain writes log cosh(z0 + move delta) (BF16) straight into
//      the A tile in shared memory (128-byte swizzle, K-major), z0 being the chain's FP32
//      layer-0 pre-activations and the delta +-2 times a row of W1t (a flip) or of the
//      per-bond differences W1t[i] - W1t[j] (an exchange; the same FP32 difference the
//      multi-launch sampler forms), so a proposal reads two rows.  z0 has two buffers per
//      chain in global memory (read through L2): the proposal's z0 + delta goes to the other
//      one, and an accepted move only switches the chain's current buffer.  All loads of a
//      warp's rows are issued before their arithmetic, three rows at a time;
//   3. products: one thread issues tcgen05.mma kind::f16 (FP8: kind::f8f6f4) over the A tile and W2 K-blocks that
//      a TMA thread streams through a two-stage ring (W2 does not fit shared memory); K steps
//      wholly beyond the layer-0 width (zero columns of the A tile) are skipped.  Meanwhile a
//      thread per chain draws the next step's move and log u (Philox, the layout of
//      nqs_sweep) into its registers;
//   4. epilogue: the accumulator rows (TMEM) give log psi(y) = b_out + w_out . tanh(z2 + b2);
//   5. decision: accept iff 2 (log psi(y) - log psi(x)) > log u (the identity is accepted);
//      an accepted move updates the spins and log psi and switches z0's buffer.
// Rows of the tile beyond R hold stale or zero values whose outputs are not read.  Every wait
// is bounded; on a timeout the kernel records STATUS_TIMEOUT and stops.  The host rebuilds z0
// and log psi from the spins between launches (every `refresh` sweeps), as the multi-launch
// sampler does.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace nqs {
namespace {

constexpr int FU_THREADS = 320;  // warp 0: TMA, warp 1: MMA issuer + TMEM, warps 2..9: workers
constexpr int FU_WORKERS = 256;
constexpr int FU_STAGES = 2;
constexpr int FU_MAX_K = 448;   // layer-0 width (padded) and layer-1 width limits
constexpr int FU_ROWS = 3;      // proposal rows a warp loads at once
constexpr uint32_t FU_POLLS = 1u << 24;

struct FusedArgs {
  uint32_t *state;
  float *z0;          // [C][H0]: the chains' z0 at launch
  float *z0b;         // [C][H0]: the second buffer
  float *lp;          // [C]
  const float *W1d;   // [n_moves][H0]: W1t rows (flips) or W1t[i_b] - W1t[j_b] (exchanges)
  const float *b2;    // [H1]
  const float *w_out; // [H1]
  const float *inv_scale;  // FP8 copy: 1 / s2 (device scalar)
  float b_out;
  const int2 *bonds;
  int64_t *n_acc;
  uint32_t *acc_bits;
  float *delta;
  uint32_t *samples;
  float *logpsi;
  int *status;
  int64_t C;
  int R;             // chains per tile
  int N, W, H0, Kp1, H1, p0, p1, exchange, n_moves;
  int n_sweeps_total, t0, t1, burn_in, add_acc;
  uint32_t sweep_offset, k0, k1;
};

__device__ __forceinline__ float log_cosh_f(float z) {
  z = fabsf(z);
  return z + __logf(1.f + __expf(-2.f * z)) - 0.69314718055994531f;
}
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void worker_sync() { asm volatile("bar.sync 1, %0;" ::"n"(FU_WORKERS) : "memory"); }
// worker barrier that also ORs a flag over the workers, so that every worker takes the same branch
__device__ __forceinline__ bool worker_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(FU_WORKERS)
      : "memory");
  return r != 0;
}

// Tile row of chain r: chains go round the four TMEM lane quarters (row 32 (r % 4) + r / 4), so
// that every epilogue warp has rows even when a tile holds fewer than 128 chains.
__device__ __forceinline__ uint32_t tile_row(int r) { return 32u * (uint32_t)(r & 3) + (uint32_t)(r >> 2); }

struct FusedSmem {
  float b2[FU_MAX_K], wout[FU_MAX_K];  // layer-1 bias and w_out, staged once
  float part[128][2];
  float lpx[128], gsign[128];
  int2 mv[128];    // move (i, j) of this step (j = -1 for a flip); i = -1: the identity
  int mi[128];     // its index (site or bond), -1: the identity
  int cur[128];    // buffer holding the chain's z0 (0: z0, 1: z0b)
  int nacc[128];
  uint32_t abits[128];
};

// F8: the FP8 copy.  A K-block is then 128 E4M3 elements (still 128 bytes per row), a lane
// writes four activations per K-block (one 32-bit store at the byte offset of BF16 element
// 2 lane), and the products are kind::f8f6f4 (K = 32 per instruction).
template <bool F8>
__global__ void __launch_bounds__(FU_THREADS, 1)
    dense_fused_sweep_kernel(const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
                             const FusedArgs a) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t full[FU_STAGES], empty[FU_STAGES], a_full, acc_full, acc_empty;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ FusedSmem sm;
  const uint32_t raw = smem_addr(smem_dyn);
  unsigned char *base = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  constexpr int KB = F8 ? 128 : 64;  // elements per 128-byte K-block
  const int kb_n = a.Kp1 / KB;
  unsigned char *atile = base;                                   // kb_n x 16 KB
  unsigned char *ring = base + kb_n * 16384;                     // FU_STAGES x H1 x 128 B
  uint32_t *spins = reinterpret_cast<uint32_t *>(ring + FU_STAGES * a.H1 * 128);  // [128][8]
  const uint32_t stage_bytes = (uint32_t)a.H1 * 128u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < FU_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&a_full, 1);
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 1);
    fence_mbar_init();
    abort_flag = 0;
    prefetch_tmap(&mB0);
    if (a.p1) prefetch_tmap(&mB1);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, 512);
    tc::tmem_relinquish();
  }
  // the A tile starts (and its unused rows stay) zero
  for (int i = tid; i < kb_n * 16384 / 16; i += FU_THREADS) reinterpret_cast<uint4 *>(atile)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < FU_MAX_K; i += FU_THREADS) {
    sm.b2[i] = i < a.H1 ? a.b2[i] : 0.f;
    sm.wout[i] = i < a.H1 ? a.w_out[i] : 0.f;
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    for (uint32_t it = 0; it < FU_POLLS; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if (abort_flag) return false;
    }
    abort_flag = 1;
    atomicOr(a.status, STATUS_TIMEOUT);
    return false;
  };

  // draw of step st of tile chain r: the move (i, j) (j = -1 for a flip) and log u; the
  // thread of chain r draws and decides, so both stay in its registers
  auto draw = [&](int st, int64_t c0, int r, float &thr, int2 &nb, int &mi) {
    const int t = a.t0 + st / a.N, p = st % a.N;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(p / 2), a.sweep_offset + (uint32_t)t, (uint32_t)(c0 + r), TAG_SWEEP),
                                  a.k0, a.k1);
    const uint32_t wm = (p & 1) ? w.z : w.x, wu = (p & 1) ? w.w : w.y;
    const int m = (int)index_from_word(wm, (uint32_t)a.n_moves);
    const uint32_t k = wu >> 8;
    thr = k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
    nb = a.exchange ? a.bonds[m] : make_int2(m, -1);
    mi = m;
  };

  const int64_t n_tiles = (a.C + a.R - 1) / a.R;
  const int steps_per_tile = (a.t1 - a.t0) * a.N;
  uint32_t step_g = 0;  // steps this CTA has run (barrier phases)

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer: W2 K-blocks, kb_n per step, two-stage ring
      uint32_t it = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles && !abort_flag; tile += gridDim.x)
        for (int st = 0; st < steps_per_tile + 1 && !abort_flag; ++st)  // + the initial evaluation
          for (int kb = 0; kb < kb_n; ++kb, ++it) {
            const int s = it % FU_STAGES;
            if (!wait(&empty[s], ((it / FU_STAGES) & 1u) ^ 1u)) break;
            unsigned char *dst = ring + s * stage_bytes;
            mbar_expect_tx(&full[s], stage_bytes);
            tma_load_2d(dst, &mB0, kb * KB, 0, &full[s]);
            if (a.p1) tma_load_2d(dst + a.p0 * 128, &mB1, kb * KB, a.p0, &full[s]);
          }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id0 = F8 ? tc::idesc_e4m3_f32(128, (uint32_t)a.p0) : tc::idesc_bf16_f32(128, (uint32_t)a.p0);
      const uint32_t id1 = F8 ? tc::idesc_e4m3_f32(128, (uint32_t)(a.p1 ? a.p1 : 16))
                              : tc::idesc_bf16_f32(128, (uint32_t)(a.p1 ? a.p1 : 16));
      uint32_t it = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles && !abort_flag; tile += gridDim.x)
        for (int st = 0; st < steps_per_tile + 1 && !abort_flag; ++st, ++step_g) {
          if (!wait(&a_full, step_g & 1u) || !wait(&acc_empty, (step_g & 1u) ^ 1u)) break;
          tc::fence_after_sync();
          bool ok = true;
          for (int kb = 0; kb < kb_n; ++kb, ++it) {
            const int s = it % FU_STAGES;
            if (!wait(&full[s], (it / FU_STAGES) & 1u)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            unsigned char *bs = ring + s * stage_bytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // K steps wholly beyond the layer-0 width multiply the A tile's zero columns: skipped
              if (kb * KB + kk * (KB / 4) >= a.H0) break;
              const uint64_t ad = tc::desc_sw128(smem_addr(atile + kb * 16384 + kk * 32));
              const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
              if constexpr (F8) {
                tc::mma_f8(tmem, ad, tc::desc_sw128(smem_addr(bs + kk * 32)), id0, acc);
                if (a.p1) tc::mma_f8(tmem + (uint32_t)a.p0, ad, tc::desc_sw128(smem_addr(bs + a.p0 * 128 + kk * 32)), id1, acc);
              } else {
                tc::mma_bf16(tmem, ad, tc::desc_sw128(smem_addr(bs + kk * 32)), id0, acc);
                if (a.p1) tc::mma_bf16(tmem + (uint32_t)a.p0, ad, tc::desc_sw128(smem_addr(bs + a.p0 * 128 + kk * 32)), id1, acc);
              }
            }
            tc::mma_commit(&empty[s]);
          }
          if (!ok) break;
          tc::mma_commit(&acc_full);
        }
    }
  } else {  // ---- workers
    const int wt = tid - 64, wk = wt >> 5;  // worker thread 0..255, worker warp 0..7
    const int q = warp & 3, half = wk >> 2;  // TMEM lane quarter (warp w reads lanes 32 (w % 4) ..), column half
    const float sc = F8 ? *a.inv_scale : 1.f;  // FP8: z2 = acc / s2
    bool stop = false;
    float thr = 0.f, thr_next = 0.f;  // log u of this step and of the next (thread of chain wt)
    int2 nb_next = make_int2(0, -1);   // the next step's drawn move
    int mi_next = 0;                   // and its index
    for (int64_t tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x) {
      const int64_t c0 = tile * a.R;
      const int Rv = (int)std::min<int64_t>(a.R, a.C - c0);
      for (int e = wt; e < Rv * a.W; e += FU_WORKERS) spins[(e / a.W) * 8 + e % a.W] = a.state[(c0 + e / a.W) * a.W + e % a.W];
      for (int r = wt; r < 128; r += FU_WORKERS) {
        sm.lpx[r] = r < Rv ? a.lp[c0 + r] : 0.f;
        sm.nacc[r] = 0;
        sm.abits[r] = 0u;
        sm.mv[r] = make_int2(-1, -1);
        sm.gsign[r] = 0.f;
        sm.cur[r] = 0;
      }
      worker_sync();
      // step -1 evaluates the current configurations (log psi(x) as this kernel computes it);
      // steps 0 .. steps_per_tile - 1 are the proposals
      for (int st = -1; st < steps_per_tile; ++st, ++step_g) {
        const int t = a.t0 + (st < 0 ? 0 : st / a.N), p = st < 0 ? 0 : st % a.N;
        // 1. moves (thread per chain): the move drawn during the previous step's products; the
        //    chain's spins decide whether an exchange moves anything and the sign of the change
        if (st >= 0 && wt < Rv) {
          const int r = wt;
          const int2 nb = nb_next;
          thr = thr_next;
          const uint32_t *sw = spins + r * 8;
          const int si = (sw[nb.x >> 5] >> (nb.x & 31)) & 1u;
          const bool moved = nb.y < 0 || si != (int)((sw[nb.y >> 5] >> (nb.y & 31)) & 1u);
          sm.mv[r] = moved ? nb : make_int2(-1, -1);
          sm.mi[r] = moved ? mi_next : -1;
          sm.gsign[r] = si ? -2.f : 2.f;
        }
        worker_sync();
        // 2. proposal rows into the A tile (warp per chain, FU_ROWS rows at a time, every load of
        //    those rows issued before their arithmetic); step -1 writes the unmoved rows
        if constexpr (F8) {
          for (int r0 = wk; r0 < Rv; r0 += 8 * FU_ROWS) {
            float4 z[FU_ROWS][4], d[FU_ROWS][4];
            float g[FU_ROWS];
            bool live[FU_ROWS];
#pragma unroll
            for (int u = 0; u < FU_ROWS; ++u) {
              const int r = r0 + 8 * u;
              live[u] = r < Rv && !(st >= 0 && sm.mv[r].x < 0);  // the identity is not evaluated
              const int mi = live[u] && st >= 0 ? sm.mi[r] : -1;
              g[u] = live[u] ? sm.gsign[r] : 0.f;
              const float *zr = (sm.cur[live[u] ? r : r0] ? a.z0b : a.z0) + (c0 + (live[u] ? r : r0)) * a.H0;
              const float *dr = a.W1d + (int64_t)(mi < 0 ? 0 : mi) * a.H0;
#pragma unroll
              for (int kb = 0; kb < 4; ++kb) {
                const int k = kb * 128 + 4 * lane;
                const bool in = live[u] && kb < kb_n && k < a.H0;
                z[u][kb] = in ? *reinterpret_cast<const float4 *>(zr + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                d[u][kb] = in && mi >= 0 ? *reinterpret_cast<const float4 *>(dr + k) : make_float4(0.f, 0.f, 0.f, 0.f);
              }
            }
#pragma unroll
            for (int u = 0; u < FU_ROWS; ++u) {
              if (!live[u]) continue;
              const int r = r0 + 8 * u;
              const bool moved = st >= 0;
              float *zn = (sm.cur[r] ? a.z0 : a.z0b) + (c0 + r) * a.H0;  // the other buffer
#pragma unroll
              for (int kb = 0; kb < 4; ++kb) {
                if (kb >= kb_n) break;
                const int k = kb * 128 + 4 * lane;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < a.H0) {
                  const float4 zz = make_float4(fmaf(g[u], d[u][kb].x, z[u][kb].x), fmaf(g[u], d[u][kb].y, z[u][kb].y),
                                                fmaf(g[u], d[u][kb].z, z[u][kb].z), fmaf(g[u], d[u][kb].w, z[u][kb].w));
                  if (moved) *reinterpret_cast<float4 *>(zn + k) = zz;
                  v = make_float4(log_cosh_f(zz.x), log_cosh_f(zz.y), log_cosh_f(zz.z), log_cosh_f(zz.w));
                }
                const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v.x, v.y), __NV_SATFINITE, __NV_E4M3);
                const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v.z, v.w), __NV_SATFINITE, __NV_E4M3);
                // elements 4 lane .. 4 lane + 3 of the K-block: the bytes of BF16 element 2 lane
                *reinterpret_cast<uint32_t *>(atile + kb * 16384 + tc::sw128_offset(tile_row(r), (uint32_t)(2 * lane))) =
                    lo | (hi << 16);
              }
            }
          }
        } else {
          for (int r0 = wk; r0 < Rv; r0 += 8 * FU_ROWS) {
            float2 z[FU_ROWS][7], d[FU_ROWS][7];
            float g[FU_ROWS];
            bool live[FU_ROWS];
#pragma unroll
            for (int u = 0; u < FU_ROWS; ++u) {
              const int r = r0 + 8 * u;
              live[u] = r < Rv && !(st >= 0 && sm.mv[r].x < 0);  // the identity is not evaluated
              const int mi = live[u] && st >= 0 ? sm.mi[r] : -1;
              g[u] = live[u] ? sm.gsign[r] : 0.f;
              const float *zr = (sm.cur[live[u] ? r : r0] ? a.z0b : a.z0) + (c0 + (live[u] ? r : r0)) * a.H0;
              const float *dr = a.W1d + (int64_t)(mi < 0 ? 0 : mi) * a.H0;
#pragma unroll
              for (int kb = 0; kb < 7; ++kb) {
                const int k = kb * 64 + 2 * lane;
                const bool in = live[u] && kb < kb_n && k < a.H0;
                z[u][kb] = in ? *reinterpret_cast<const float2 *>(zr + k) : make_float2(0.f, 0.f);
                d[u][kb] = in && mi >= 0 ? *reinterpret_cast<const float2 *>(dr + k) : make_float2(0.f, 0.f);
              }
            }
#pragma unroll
            for (int u = 0; u < FU_ROWS; ++u) {
              if (!live[u]) continue;
              const int r = r0 + 8 * u;
              const bool moved = st >= 0;
              float *zn = (sm.cur[r] ? a.z0 : a.z0b) + (c0 + r) * a.H0;  // the other buffer
#pragma unroll
              for (int kb = 0; kb < 7; ++kb) {
                if (kb >= kb_n) break;
                const int k = kb * 64 + 2 * lane;
                float v0 = 0.f, v1 = 0.f;
                if (k < a.H0) {
                  const float2 zz = make_float2(fmaf(g[u], d[u][kb].x, z[u][kb].x), fmaf(g[u], d[u][kb].y, z[u][kb].y));
                  if (moved) *reinterpret_cast<float2 *>(zn + k) = zz;
                  v0 = log_cosh_f(zz.x);
                  v1 = log_cosh_f(zz.y);
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                *reinterpret_cast<__nv_bfloat162 *>(atile + kb * 16384 +
                                                    tc::sw128_offset(tile_row(r), (uint32_t)(2 * lane))) = h2;
              }
            }
          }
        }
        tc::fence_proxy_async_smem();
        worker_sync();
        if (wt == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&a_full)) : "memory");
        // 2. while the products run: the next step's draws (thread per chain)
        if (st + 1 < steps_per_tile && wt < Rv) draw(st + 1, c0, wt, thr_next, nb_next, mi_next);
        // 3-4. the products, then the epilogue: rows of this warp's lane quarter, its column half
        const bool ok = __all_sync(FULL_MASK, wait(&acc_full, step_g & 1u));  // the TMEM loads are warp-collective
        tc::fence_after_sync();
        // log psi(y) - b_out of chain r is part[r][0] + part[r][1]; the warp pair of lane quarter q
        // takes the 64-column blocks 64 half + 128 j, and every chain's sum runs in one order
        // whichever load serves it: per column residue j = c % 4, the columns in increasing order,
        // then (S0 + S1) + (S2 + S3).  So results do not depend on the tiling.
        if (ok && q < Rv) {
          if (a.R <= 64) {
            // chains in lanes 32 q + i, i = r / 4 < 16: thread t holds the rows i = t / 4 and
            // t / 4 + 8 at columns 4k + t % 4 (16-lane load), so no lane computes an empty row
            const int ia = lane >> 2, cq = lane & 3;
            float da = 0.f, db = 0.f;
            for (int cb = 64 * half; cb < a.H1; cb += 128) {
              float v[32];
              tc::tmem_ld16x128b_x16(tc::tmem_lane_addr(tmem, 32 * q, cb), v);
#pragma unroll
              for (int k = 0; k < 16; ++k) {
                const int c = cb + 4 * k + cq;
                if (c < a.H1) {
                  const float bb = sm.b2[c], w = sm.wout[c];
                  da = fmaf(tanh_approx(F8 ? fmaf(v[2 * k], sc, bb) : v[2 * k] + bb), w, da);
                  db = fmaf(tanh_approx(F8 ? fmaf(v[2 * k + 1], sc, bb) : v[2 * k + 1] + bb), w, db);
                }
              }
            }
            da += __shfl_xor_sync(FULL_MASK, da, 1);
            db += __shfl_xor_sync(FULL_MASK, db, 1);
            da += __shfl_xor_sync(FULL_MASK, da, 2);
            db += __shfl_xor_sync(FULL_MASK, db, 2);
            const int ra = 4 * ia + q, rb = 4 * (ia + 8) + q;
            if (cq == 0 && ra < Rv) sm.part[ra][half] = da;
            if (cq == 0 && rb < Rv) sm.part[rb][half] = db;
          } else {
            const int rq = 4 * lane + q;  // chain of this thread's TMEM row 32 q + lane
            float s4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int cb = 64 * half; cb < a.H1; cb += 128) {
#pragma unroll
              for (int sub = 0; sub < 2; ++sub) {
                float v[32];
                tc::tmem_ld32(tc::tmem_lane_addr(tmem, 32 * q, cb + 32 * sub), v);
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  const int c = cb + 32 * sub + e;
                  if (c < a.H1)
                    s4[e & 3] = fmaf(tanh_approx(F8 ? fmaf(v[e], sc, sm.b2[c]) : v[e] + sm.b2[c]), sm.wout[c], s4[e & 3]);
                }
              }
            }
            if (rq < Rv) sm.part[rq][half] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
          }
        }
        tc::fence_before_sync();
        stop = worker_sync_or(!ok || abort_flag);
        if (stop) break;
        if (wt == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acc_empty)) : "memory");
        // 5. decision (thread per chain)
        if (wt < Rv) {
          const int r = wt;
          const float lpy = a.b_out + sm.part[r][0] + sm.part[r][1];
          if (st < 0) {
            sm.lpx[r] = lpy;
          } else {
            const int2 mv = sm.mv[r];
            bool acc = true;
            float dlt = 0.f;
            if (mv.x >= 0) {
              dlt = lpy - sm.lpx[r];
              acc = 2.f * dlt > thr;
            }
            if (acc) {
              sm.nacc[r] += 1;
              if (mv.x >= 0) {
                uint32_t *sw = spins + r * 8;
                sw[mv.x >> 5] ^= 1u << (mv.x & 31);
                if (mv.y >= 0) sw[mv.y >> 5] ^= 1u << (mv.y & 31);
                sm.lpx[r] = lpy;
                sm.cur[r] ^= 1;  // z0 + delta, written by the proposal, becomes the chain's z0
              }
            }
            const int64_t c = c0 + r;
            if (a.acc_bits) {
              sm.abits[r] |= (acc ? 1u : 0u) << (p & 31);
              if ((p & 31) == 31 || p == a.N - 1) {
                a.acc_bits[(c * a.n_sweeps_total + t) * a.W + (p >> 5)] = sm.abits[r];
                sm.abits[r] = 0u;
              }
            }
            if (a.delta) a.delta[(c * a.n_sweeps_total + t) * a.N + p] = dlt;
          }
        }
        worker_sync();
        // samples after a completed sweep
        if (st >= 0 && p == a.N - 1 && t >= a.burn_in) {
          const int64_t row0 = (int64_t)(t - a.burn_in) * a.C + c0;
          for (int e = wt; e < Rv * a.W; e += FU_WORKERS)
            if (a.samples) a.samples[(row0 + e / a.W) * a.W + e % a.W] = spins[(e / a.W) * 8 + e % a.W];
          if (a.logpsi)
            for (int r = wt; r < Rv; r += FU_WORKERS) a.logpsi[row0 + r] = sm.lpx[r];
        }
        worker_sync();
      }
      if (stop) break;
      for (int e = wt; e < Rv * a.W; e += FU_WORKERS) a.state[(c0 + e / a.W) * a.W + e % a.W] = spins[(e / a.W) * 8 + e % a.W];
      for (int r = wt; r < Rv; r += FU_WORKERS) {
        a.lp[c0 + r] = sm.lpx[r];
        if (a.n_acc) a.n_acc[c0 + r] = (a.add_acc ? a.n_acc[c0 + r] : 0) + sm.nacc[r];
      }
      worker_sync();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (abort_flag && tid == 0) {  // let products or copies in flight land before TMEM and smem are released
    for (int s = 0; s < FU_STAGES; ++s) mbar_wait_bounded(&empty[s], 0, 1u << 16);
    mbar_wait_bounded(&acc_full, 0, 1u << 16);
  }
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// A tile (K-blocks of 64 BF16 or 128 E4M3 elements), the W2 ring and the spins
size_t fused_smem(const nqs_ctx *c) {
  const size_t kb_n = c->dtype == NQS_FP8E4M3 ? (size_t)c->Kp8[1] / 128 : (size_t)c->Kp[1] / 64;
  return 1024 + kb_n * 16384 + 2 * (size_t)c->H[1] * 128 + 128 * 8 * 4;
}

}  // namespace

__global__ void dense_bond_diff_kernel(const float *__restrict__ W1t, const int2 *__restrict__ bonds, int n_bonds,
                                       int H0, float *W1d) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)n_bonds * H0;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / H0), k = (int)(q % H0);
    const int2 bd = bonds[b];
    W1d[q] = W1t[(int64_t)bd.x * H0 + k] - W1t[(int64_t)bd.y * H0 + k];
  }
}

bool dense_fused_supported(const nqs_ctx *c) {
  if (c->model_kind != NQS_DENSE || (c->dtype != NQS_BF16 && c->dtype != NQS_FP8E4M3) || c->L != 2) return false;
  if (c->dtype == NQS_FP8E4M3 && (c->H[0] % 4 != 0 || c->Kp8[1] > 512)) return false;  // float4 rows, 4 K-blocks
  const int H1 = c->H[1];
  const int p1 = H1 > 256 ? H1 - 256 : 0;
  return c->Kp[1] <= FU_MAX_K && H1 <= FU_MAX_K && H1 % 16 == 0 && p1 % 16 == 0 && c->W <= 8 &&
         fused_smem(c) + sizeof(FusedSmem) + 256 <= (size_t)c->smem_optin;
}

cudaError_t dense_fused_prepare(const nqs_ctx *c, cudaStream_t s) {
  const int64_t n = (int64_t)c->n_bonds * c->H[0];
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
  // the differences of the sampling copy's layer-0 rows (E4M3-rounded for the FP8 copy)
  dense_bond_diff_kernel<<<grid, 256, 0, s>>>(c->dtype == NQS_FP8E4M3 ? c->d_W1t8 : c->d_W1t, c->d_bonds, c->n_bonds,
                                              c->H[0], c->d_W1d);
  return cudaGetLastError();
}

// Sweeps [t0, t1) of the fused sampler; z0 and lp hold the chains' current layer-0
// pre-activations and log psi (rebuilt by the caller).
cudaError_t dense_fused_sweeps(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int t0, int t1,
                               int burn_in, uint64_t seed, uint32_t sweep_offset, uint32_t *samples, float *logpsi,
                               int64_t *n_acc, uint32_t *acc_bits, float *delta, bool add_acc, cudaStream_t s) {
  FusedArgs a;
  a.state = state;
  a.z0 = c->d_z1;
  a.z0b = c->d_z1b;
  a.lp = c->d_lp;
  const bool f8 = c->dtype == NQS_FP8E4M3;
  a.W1d = c->ham_kind == NQS_HEISENBERG ? c->d_W1d : (f8 ? c->d_W1t8 : c->d_W1t);
  a.inv_scale = f8 ? c->d_scale8 + c->L + 1 : nullptr;
  if (!a.W1d) return cudaErrorInvalidValue;
  a.b2 = c->d_bl[1];
  a.w_out = c->d_wout;
  a.b_out = c->b_out;
  a.bonds = c->d_bonds;
  a.n_acc = n_acc;
  a.acc_bits = acc_bits;
  a.delta = delta;
  a.samples = samples;
  a.logpsi = logpsi;
  a.status = c->d_status;
  a.C = C;
  a.N = c->N;
  a.W = c->W;
  a.H0 = c->H[0];
  a.Kp1 = f8 ? c->Kp8[1] : c->Kp[1];
  a.H1 = c->H[1];
  a.p0 = std::min(256, a.H1);
  a.p1 = a.H1 - a.p0;
  a.exchange = c->ham_kind == NQS_HEISENBERG;
  a.n_moves = a.exchange ? c->n_bonds : c->N;
  a.n_sweeps_total = n_sweeps;
  a.t0 = t0;
  a.t1 = t1;
  a.burn_in = burn_in;
  a.add_acc = add_acc ? 1 : 0;
  a.sweep_offset = sweep_offset;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.R = (int)std::min<int64_t>(128, (C + c->num_sms - 1) / c->num_sms);
  CUtensorMap mB0, mB1;
  auto tmap = [&](CUtensorMap *m, uint32_t box_rows) {
    return f8 ? make_tmap_u8_2d(m, c->d_Wl8[1], (uint64_t)a.H1, (uint64_t)a.Kp1, box_rows)
              : make_tmap_bf16_2d(m, c->d_Wl[1], (uint64_t)a.H1, (uint64_t)a.Kp1, box_rows);
  };
  if (!tmap(&mB0, (uint32_t)a.p0)) return cudaErrorInvalidValue;
  if (a.p1 && !tmap(&mB1, (uint32_t)a.p1)) return cudaErrorInvalidValue;
  if (!a.p1) mB1 = mB0;
  const size_t shm = fused_smem(c);
  auto k = f8 ? dense_fused_sweep_kernel<true> : dense_fused_sweep_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (C + a.R - 1) / a.R;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_tiles, c->num_sms));
  k<<<grid, FU_THREADS, shm, s>>>(mB0, mB1, a);
  return cudaGetLastError();
}

}  // namespace nqs
