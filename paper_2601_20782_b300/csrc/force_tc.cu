// Force of the RBM (App. I, Eq. forces) on the tensor cores:
//     F_k = (1/n) sum_x O_k(x) (eloc(x) - E),  O_a = s, O_b = tanh(theta), O_W[j, i] = tanh(theta_j) s_i.
//
// Block (jt, chunk) owns hidden units j0 = 64 jt .. j0 + 63 and one chunk of rows; per tile
// of 128 rows (samples x) it runs two tcgen05 products with FP32 accumulation in TMEM:
//   GEMM1  theta_s[x, j] = sum_i s[x, i] W_s[j, i]      M = 128 rows, N = 3 x 64, K = 128 sites
//          A = spins (exact in BF16), B = the three BF16 terms W_s of W (hi, mid, lo) stacked
//          along N, so that one product per K step gives the three partial thetas, summed
//          in the epilogue as (hi + mid) + lo
//   GEMM2  G[i, j]  += sum_x s[x, i] a[x, j]           M = 128 sites, K = 128 rows
//          a = tanh(theta + b) (eloc - E) as three BF16 terms; a_hi and a_mid side by side
//          (N = 128) into the accumulator pair (hi, lo), then a_lo (N = 64) into lo
// Column i = N of the spin tile is a constant +1 whose W column holds the hidden bias, so GEMM1
// gives theta = W s + b and G[N, j] = sum_x a[x, j] gives the b-entries; the extra hidden unit
// j = M carries a = eloc - E, so G[i, M] gives the a-entries.  The spin tile is the K-major A of GEMM1 and, read MN-major, the A of GEMM2.
// The hi term of a accumulates apart from the mid + lo terms, so that the small terms are not
// rounded away against the large running sum.
//
// The block is warp-specialised so that staging, the tensor core and the epilogue overlap:
//   warp 16 (one thread) issues GEMM1 of tile t, then GEMM2 of tile t - 1;
//   warps 0-15 (workers) read theta from TMEM (lanes 32 (w % 4) .., units 16 (w / 4) ..), form
//                        the three a-terms in registers, store them once GEMM2 of the previous
//                        tile has read its terms, then stage their own row's part of the spin
//                        tile two tiles ahead (one byte of spins per 16-byte chunk through a
//                        256-entry table of BF16 +-1), and every DRAIN tiles add the accumulators
//                        into the block's FP64 slice of the workspace (rows chunk * P ...), which
//                        force_reduce_kernel then sums over chunks in a fixed order.
// Buffers: three spin tiles and one set of a-terms in shared memory; theta and two accumulator
// pairs (one drained while the other accumulates) in TMEM; mbarriers hand each buffer between the
// roles.  Every wait is bounded: a wait that gives up records STATUS_TIMEOUT and every role
// leaves its loop.
//
// The complex-parameter RBM (CPLX) runs the same products with 32 complex hidden units per
// block: the 64 columns of a term are Re of units j0 .. j0 + 31, then Im of the same units, so
// GEMM1 gives Re theta and Im theta (spins are real), and the a-terms hold
//     a = conj(tanh theta) (eloc - E)    (Re in columns 0-31, Im in 32-63; eloc and E complex),
// so GEMM2 gives the real and imaginary parts of sum_x s_i conj(O_k) (eloc - E) (App. I, Eq.
// forces with complex O_k); the partial forces go to a [chunks][P] array of complex entries.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace nqs {
namespace {

constexpr int FTC_WORKERS = 16;                  // warps 0-15: epilogue + spin tiles; warp 16: MMA
constexpr int FTC_THREADS = 32 * (FTC_WORKERS + 1);
constexpr int FTC_NW = 32 * FTC_WORKERS;         // worker threads
constexpr int FTC_HT = 64;       // hidden units per block
constexpr int FTC_NS = 3;        // spin tiles in flight
constexpr int FTC_DRAIN = 16;    // tiles per FP32 accumulation period before the FP64 drain
constexpr uint32_t FTC_POLLS = 1u << 24;
constexpr int FTC_KP = 128;      // padded site extent (N + 1 <= 128)
constexpr uint32_t SPIN_BYTES = 128 * FTC_KP * 2;        // one spin tile: 2 K-blocks of 16 KB
constexpr uint32_t WKB_BYTES = 3 * FTC_HT * 128;         // one K-block of the stacked W terms
constexpr uint32_t ATERM_BYTES = 128 * FTC_HT * 2;       // one a term: 128 rows x 128 bytes
constexpr size_t FTC_SMEM = 1024 + 2 * WKB_BYTES + FTC_NS * SPIN_BYTES + 3 * ATERM_BYTES + 256 * 16;
// TMEM columns: theta_hi, theta_mid, theta_lo at 0, 64, 128; accumulator pair d at 256 + 128 d
// (hi, then lo 64 columns later)
constexpr uint32_t TM_G = 256;

struct ForceTcParams {
  const uint32_t *cfg;
  const float *eloc;
  const float *eloc_im;  // CPLX: Im eloc (E = stats[0] + i stats[5])
  const double *stats;
  const float *Wm;  // [N][M] FP32 master, site-major
  const float *bm;  // [M]
  const float2 *Wc; // CPLX: [N][M_pad] complex weights, site-major
  const float2 *bc; // CPLX: [M_pad] complex hidden bias
  double *ws;       // [chunks][P] (CPLX: complex entries, Re then Im)
  int *status;
  int64_t n, P;
  int N, W, M, M_pad, n_chunks;
};

__device__ __forceinline__ void split3(float a, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(a);
  const float r = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Paired FP32 arithmetic (fma.rn.f32x2 / mul.rn.f32x2): two operations per instruction, each
// rounded as its scalar counterpart.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// The three BF16 terms of the pair a (a.x in the low half): the same split as split3, two values
// per conversion; the residuals a - hi and r - mid are exact.
__device__ __forceinline__ void split3_pair(float2 a, uint32_t &h, uint32_t &m, uint32_t &l) {
  h = bf2_bits(__floats2bfloat162_rn(a.x, a.y));
  const float2 r = ffma2(make_float2(bf_lo(h), bf_hi(h)), f2(-1.f), a);
  m = bf2_bits(__floats2bfloat162_rn(r.x, r.y));
  const float2 r2 = ffma2(make_float2(bf_lo(m), bf_hi(m)), f2(-1.f), r);
  l = bf2_bits(__floats2bfloat162_rn(r2.x, r2.y));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tanh of the epilogue for a pair, from two textbook forms selected without a branch: the odd
// Taylor series y (1 - y^2/3 + 2 y^4/15 - ...) through y^15 for |y| < 0.55 (truncation below
// 4.1e-8 relative), and sign(y) (1 - 2 / (e^{2|y|} + 1)) beyond, with e^{2|y|} by ex2.approx and
// the reciprocal by rcp.approx (a few ulp; e^{2|y|} = inf gives exactly 1).
__device__ __forceinline__ float2 tanh_epi2(float2 y) {
  const float2 y2 = fmul2(y, y);
  float2 p = f2(-929569.f / 638512875.f);
  p = ffma2(p, y2, f2(21844.f / 6081075.f));
  p = ffma2(p, y2, f2(-1382.f / 155925.f));
  p = ffma2(p, y2, f2(62.f / 2835.f));
  p = ffma2(p, y2, f2(-17.f / 315.f));
  p = ffma2(p, y2, f2(2.f / 15.f));
  p = ffma2(p, y2, f2(-1.f / 3.f));
  p = ffma2(p, y2, f2(1.f));
  const float2 poly = fmul2(y, p);
  const float2 t = make_float2(fabsf(y.x), fabsf(y.y));
  const float2 g = fmul2(t, f2(2.8853900817779268f));
  const float2 e1 = ffma2(make_float2(ex2_approx(g.x), ex2_approx(g.y)), f2(1.f), f2(1.f));
  const float2 q = ffma2(f2(-2.f), make_float2(rcp_approx(e1.x), rcp_approx(e1.y)), f2(1.f));
  return make_float2(t.x < 0.55f ? poly.x : copysignf(q.x, y.x), t.y < 0.55f ? poly.y : copysignf(q.y, y.y));
}

// tanh(x + iy) = (sinh x cosh x + i sin y cos y) / (sinh^2 x + cos^2 y): the denominator is
// |cosh(x + iy)|^2 as a sum of squares, so there is no cancellation near the zeros of cosh.
__device__ __forceinline__ float2 tanh_cplx(float x, float y) {
  float sy, cy;
  sincosf(y, &sy, &cy);
  const float shx = sinhf(x), chx = coshf(x);
  const float inv = 1.f / fmaf(shx, shx, cy * cy);
  return make_float2(shx * chx * inv, sy * cy * inv);
}

// 8 consecutive FP32 columns of the warp's 32 TMEM lanes (lane rule of tc::tmem_ld32)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// byte offset of the 16-byte chunk c of row r in a 128-byte-swizzled tile of 128-byte rows
__device__ __forceinline__ uint32_t sw_chunk(uint32_t r, uint32_t c) {
  return (r >> 3) * 1024u + (r & 7u) * 128u + (((c ^ r) & 7u) << 4);
}

template <bool CPLX>
__global__ void __launch_bounds__(FTC_THREADS, 1) rbm_force_tc_kernel(const ForceTcParams p) {
  constexpr int UB = CPLX ? FTC_HT / 2 : FTC_HT;  // hidden units per block
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t spin_full[FTC_NS], spin_free[FTC_NS], theta_full, theta_empty, a_full, a_free, g_full[2],
      g_empty[2], fin_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const uint32_t raw = smem_addr(smem_dyn);
  unsigned char *base = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  unsigned char *sW = base;                           // K-major [192 = 3 terms x 64 j][128 i]
  unsigned char *sS = sW + 2 * WKB_BYTES;             // FTC_NS spin tiles, K-major [128 x][128 i]
  unsigned char *sA = sS + FTC_NS * SPIN_BYTES;       // 3 a terms, MN-major [128 x][64 j]
  uint4 *lut = reinterpret_cast<uint4 *>(sA + 3 * ATERM_BYTES);  // byte of 8 spins -> 8 BF16 (+-1)

  const int jt = blockIdx.x, chunk = blockIdx.y;
  const int j0 = jt * UB;
  const int N = p.N, M = p.M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- W of the block as three stacked BF16 terms; bias; barriers; TMEM -----------------
  for (int idx = tid; idx < FTC_HT * FTC_KP; idx += FTC_THREADS) {
    const int jj = idx % FTC_HT, i = idx / FTC_HT;
    // column N multiplies the constant +1 spin: the hidden bias enters theta through GEMM1
    float w;
    if (CPLX) {  // column jj: Re (jj < 32) or Im of unit j0 + jj % 32
      const int j = j0 + jj % UB;
      const float2 wc = j < M ? (i < N ? p.Wc[(int64_t)i * p.M_pad + j] : (i == N ? p.bc[j] : make_float2(0.f, 0.f)))
                              : make_float2(0.f, 0.f);
      w = jj < UB ? wc.x : wc.y;
    } else {
      w = j0 + jj < M ? (i < N ? p.Wm[(int64_t)i * M + j0 + jj] : (i == N ? p.bm[j0 + jj] : 0.f)) : 0.f;
    }
    __nv_bfloat16 h, m, l;
    split3(w, h, m, l);
    unsigned char *kb = sW + (i / 64) * WKB_BYTES;
    *reinterpret_cast<__nv_bfloat16 *>(kb + tc::sw128_offset(jj, i % 64)) = h;
    *reinterpret_cast<__nv_bfloat16 *>(kb + tc::sw128_offset(FTC_HT + jj, i % 64)) = m;
    *reinterpret_cast<__nv_bfloat16 *>(kb + tc::sw128_offset(2 * FTC_HT + jj, i % 64)) = l;
  }
  for (int v = tid; v < 256; v += FTC_THREADS) {  // bit k of v set: spin 8c + k up (+1 = 0x3F80)
    uint32_t w4[4];
    for (int q = 0; q < 4; ++q)
      w4[q] = (((v >> (2 * q)) & 1) ? 0x3F80u : 0xBF80u) | ((((v >> (2 * q + 1)) & 1) ? 0x3F80u : 0xBF80u) << 16);
    lut[v] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
  if (tid == 0) {
    for (int b = 0; b < FTC_NS; ++b) {
      mbar_init(&spin_full[b], FTC_NW);
      mbar_init(&spin_free[b], 1);
    }
    mbar_init(&theta_full, 1);
    mbar_init(&theta_empty, FTC_NW);
    mbar_init(&a_full, FTC_NW);
    mbar_init(&a_free, 1);
    for (int d = 0; d < 2; ++d) {
      mbar_init(&g_full[d], 1);
      mbar_init(&g_empty[d], FTC_NW);
    }
    mbar_init(&fin_bar, 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == FTC_WORKERS) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tm = tmem_base;
  const int64_t rows_per_chunk = (p.n + p.n_chunks - 1) / p.n_chunks;
  const int64_t r0 = (int64_t)chunk * rows_per_chunk, r1 = min(p.n, r0 + rows_per_chunk);
  const int T = r1 > r0 ? (int)((r1 - r0 + 127) / 128) : 0;
  volatile int *abort_v = &abort_flag;

  // Bounded wait by every thread of the calling role; false once the block aborts.
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    for (uint32_t it = 0; it < FTC_POLLS; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if (*abort_v) return false;
    }
    atomicOr(p.status, STATUS_TIMEOUT);
    *abort_v = 1;
    return false;
  };
  // warp-uniform form (for roles that go on to warp-collective tcgen05.ld)
  auto wait_warp = [&](uint64_t *bar, uint32_t parity) -> bool { return __all_sync(FULL_MASK, wait(bar, parity)); };

  if (warp == FTC_WORKERS) {
    // ================================ MMA issuer ===================================
    if (lane == 0 && T > 0) {
      const uint32_t id1 = tc::idesc_bf16_f32(128, 3 * FTC_HT);
      const uint32_t id2 = tc::idesc_bf16_f32(128, 2 * FTC_HT, 1, 1);
      const uint32_t id3 = tc::idesc_bf16_f32(128, FTC_HT, 1, 1);
      auto gemm2 = [&](int u) -> bool {
        const int sb_ = u % FTC_NS, per = u / FTC_DRAIN, d = per & 1;
        const bool first = u % FTC_DRAIN == 0;
        if (!wait(&a_full, u & 1)) return false;
        if (first && per >= 2 && !wait(&g_empty[d], ((per - 2) >> 1) & 1)) return false;
        tc::fence_after_sync();
        const uint32_t gh = tm + TM_G + 128 * d;
        unsigned char *spins = sS + sb_ * SPIN_BYTES;
        for (int k0 = 0; k0 < 128; k0 += 16) {
          const uint64_t ad = tc::desc_sw128(smem_addr(spins + k0 * 128), 16384);
          // a_hi | a_mid (two 64-unit groups one term apart) -> hi | lo
          tc::mma_bf16(gh, ad, tc::desc_sw128(smem_addr(sA + k0 * 128), ATERM_BYTES), id2, first && k0 == 0 ? 0u : 1u);
          // a_lo -> lo
          tc::mma_bf16(gh + FTC_HT, ad, tc::desc_sw128(smem_addr(sA + 2 * ATERM_BYTES + k0 * 128), ATERM_BYTES), id3, 1u);
        }
        tc::mma_commit(&spin_free[sb_]);
        tc::mma_commit(&a_free);
        if (u % FTC_DRAIN == FTC_DRAIN - 1 || u == T - 1) tc::mma_commit(&g_full[d]);
        return true;
      };
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        const int sb_ = t % FTC_NS;
        ok = wait(&spin_full[sb_], (t / FTC_NS) & 1);
        if (ok && t >= 1) ok = wait(&theta_empty, (t - 1) & 1);
        if (!ok) break;
        tc::fence_after_sync();
        unsigned char *spins = sS + sb_ * SPIN_BYTES;
        for (int k0 = 0; k0 < FTC_KP; k0 += 16) {
          const uint64_t ad = tc::desc_sw128(smem_addr(spins + (k0 / 64) * 16384 + (k0 % 64) * 2));
          const uint64_t bd = tc::desc_sw128(smem_addr(sW + (k0 / 64) * WKB_BYTES + (k0 % 64) * 2));
          tc::mma_bf16(tm, ad, bd, id1, k0 > 0 ? 1u : 0u);
        }
        tc::mma_commit(&theta_full);
        if (t >= 1) ok = gemm2(t - 1);
      }
      if (ok) gemm2(T - 1);
      // every product issued above has completed once fin_bar completes
      tc::mma_commit(&fin_bar);
      mbar_wait_bounded(&fin_bar, 0, FTC_POLLS);
    }
    __syncwarp();
  } else {
    // =========================== workers: epilogue + spin tiles ===========================
    // Warp w: TMEM lanes (rows) 32 q .. 32 q + 31 with q = w % 4, hidden units 16 g .. 16 g + 15
    // and spin chunks 4 g .. 4 g + 3 (sites 32 g .. 32 g + 31: packed word g of the row) with
    // g = w / 4.  A thread stages its own row's four chunks of tile t + 2 after storing the
    // a-terms of tile t.
    const int q = warp & 3, g = warp >> 2;
    const int x = 32 * q + lane;
    const double E = p.stats[0], E_im = CPLX ? p.stats[5] : 0.0;
    const bool has_m = j0 <= M && M < j0 + UB;
    double *out = p.ws + (int64_t)chunk * p.P * (CPLX ? 2 : 1);
    int drains = 0;
    auto load_word = [&](int t) -> uint32_t {
      const int64_t r = r0 + (int64_t)t * 128 + x;
      return (r < r1 && g < p.W) ? p.cfg[r * p.W + g] : 0u;
    };
    // chunks 4 g .. 4 g + 3 of row x of tile t (BF16 +-1; site N is +1, sites beyond it 0)
    auto produce = [&](int t, uint32_t word) {
      unsigned char *spins = sS + (t % FTC_NS) * SPIN_BYTES;
      const bool live = r0 + (int64_t)t * 128 + x < r1;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * g + cc;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (live && 8 * c <= N) {
          v = lut[(word >> (8 * cc)) & 0xFFu];
          if (8 * c + 8 > N) {  // the chunk of site N
            uint32_t *e = &v.x;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int i = 8 * c + k;
              if (i >= N) {
                const uint32_t val = i == N ? 0x3F80u : 0u, sh = 16 * (k & 1);
                e[k >> 1] = (e[k >> 1] & ~(0xFFFFu << sh)) | (val << sh);
              }
            }
          }
        }
        *reinterpret_cast<uint4 *>(spins + (c / 8) * 16384 + sw_chunk(x, c & 7)) = v;
      }
      tc::fence_proxy_async_smem();
      mbar_arrive(&spin_full[t % FTC_NS]);
    };
    // Adds the accumulator pair of period per into the FP64 slice (zero_only: writes zeros).
    auto drain = [&](int per, bool zero_only) -> bool {
      const int d = per & 1;
      float v[16], w[16];
      if (zero_only) {
        for (int t = 0; t < 16; ++t) v[t] = w[t] = 0.f;
      } else {
        if (!wait_warp(&g_full[d], (per >> 1) & 1)) return false;
        tc::fence_after_sync();
        tc::tmem_ld16(tc::tmem_lane_addr(tm + TM_G + 128 * d, 32 * q, 16 * g), v);
        tc::tmem_ld16(tc::tmem_lane_addr(tm + TM_G + 128 * d + FTC_HT, 32 * q, 16 * g), w);
        tc::fence_before_sync();
        mbar_arrive(&g_empty[d]);
      }
      const int i = x;  // TMEM lane = site
      for (int t = 0; t < 16; ++t) {
        // column 16 g + t: unit j0 + 16 g + t (CPLX: Re / Im part of unit j0 + (16 g + t) % 32)
        const int j = CPLX ? j0 + (16 * g + t) % UB : j0 + 16 * g + t;
        int64_t k = -1;
        if (j < M && i < N) k = N + M + (int64_t)j * N + i;  // W entries
        else if (j < M && i == N) k = N + j;                  // b entries
        else if (j == M && i < N) k = i;                      // a entries
        if (CPLX && k >= 0) k = 2 * k + (16 * g + t) / UB;
        if (k >= 0) out[k] = (drains ? out[k] : 0.0) + ((double)v[t] + (double)w[t]);
      }
      ++drains;
      return true;
    };
    auto eval = [&](int t) -> float2 {
      const int64_t r = r0 + (int64_t)t * 128 + x;
      if (r >= r1) return make_float2(0.f, 0.f);
      return make_float2((float)((double)p.eloc[r] - E), CPLX ? (float)((double)p.eloc_im[r] - E_im) : 0.f);
    };
    for (int t0 = 0; t0 < 2 && t0 < T; ++t0) produce(t0, load_word(t0));
    float2 e_next = T > 0 ? eval(0) : make_float2(0.f, 0.f);
    bool ok = true;
    for (int t = 0; t < T && ok; ++t) {
      const float2 ec = e_next;
      const float e = ec.x;
      if (t + 1 < T) e_next = eval(t + 1);
      const uint32_t word2 = t + 2 < T ? load_word(t + 2) : 0u;  // used after this tile's epilogue
      if (!wait_warp(&theta_full, t & 1)) { ok = false; break; }
      tc::fence_after_sync();
      if (CPLX) {
        // units j0 + 8 g .. + 7: Re theta in columns 8 g .., Im theta in 32 + 8 g .. of each term
        float re[8], im[8];
        {
          float h[8], m[8], l[8];
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, 8 * g), h);
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, FTC_HT + 8 * g), m);
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, 2 * FTC_HT + 8 * g), l);
#pragma unroll
          for (int u = 0; u < 8; ++u) re[u] = (h[u] + m[u]) + l[u];
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, UB + 8 * g), h);
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, FTC_HT + UB + 8 * g), m);
          tmem_ld8(tc::tmem_lane_addr(tm, 32 * q, 2 * FTC_HT + UB + 8 * g), l);
#pragma unroll
          for (int u = 0; u < 8; ++u) im[u] = (h[u] + m[u]) + l[u];
        }
        tc::fence_before_sync();
        mbar_arrive(&theta_empty);
        uint32_t rh[4], rm[4], rl[4], ih[4], imd[4], il[4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
          float2 ar, ai;  // a of units 8 g + 2 u2, + 1: Re parts, Im parts
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int u = 2 * u2 + v;
            const float2 th = tanh_cplx(re[u], im[u]);
            // conj(t) e = (t.x e.x + t.y e.y) + i (t.x e.y - t.y e.x); the unit M carries e itself
            float2 av = make_float2(fmaf(th.x, ec.x, th.y * ec.y), fmaf(th.x, ec.y, -th.y * ec.x));
            if (has_m && j0 + 8 * g + u == M) av = ec;
            if (v) {
              ar.y = av.x;
              ai.y = av.y;
            } else {
              ar.x = av.x;
              ai.x = av.y;
            }
          }
          split3_pair(ar, rh[u2], rm[u2], rl[u2]);
          split3_pair(ai, ih[u2], imd[u2], il[u2]);
        }
        if (t >= 1 && !wait_warp(&a_free, (t - 1) & 1)) { ok = false; break; }
        // 16-byte chunk g: Re of units 8 g .. 8 g + 7; chunk 4 + g: their Im
        const uint32_t off_r = sw_chunk(x, g), off_i = sw_chunk(x, 4 + g);
        *reinterpret_cast<uint4 *>(sA + off_r) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<uint4 *>(sA + ATERM_BYTES + off_r) = make_uint4(rm[0], rm[1], rm[2], rm[3]);
        *reinterpret_cast<uint4 *>(sA + 2 * ATERM_BYTES + off_r) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<uint4 *>(sA + off_i) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<uint4 *>(sA + ATERM_BYTES + off_i) = make_uint4(imd[0], imd[1], imd[2], imd[3]);
        *reinterpret_cast<uint4 *>(sA + 2 * ATERM_BYTES + off_i) = make_uint4(il[0], il[1], il[2], il[3]);
      } else {
      float2 th[8];  // theta of units 16 g + 2 u, + 1 (bias included through GEMM1)
      {
        float vh[16], vm[16], vl[16];
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 32 * q, 16 * g), vh);
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 32 * q, FTC_HT + 16 * g), vm);
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 32 * q, 2 * FTC_HT + 16 * g), vl);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float2 hm = ffma2(make_float2(vh[2 * u], vh[2 * u + 1]), f2(1.f), make_float2(vm[2 * u], vm[2 * u + 1]));
          th[u] = ffma2(hm, f2(1.f), make_float2(vl[2 * u], vl[2 * u + 1]));
        }
      }
      tc::fence_before_sync();
      mbar_arrive(&theta_empty);
      uint32_t ph[8], pm[8], pl[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float2 a = fmul2(tanh_epi2(th[u]), f2(e));
        if (has_m) {  // the block holding unit M: a = eloc - E there (a-entries)
          const int j = j0 + 16 * g + 2 * u;
          if (j == M) a.x = e;
          if (j + 1 == M) a.y = e;
        }
        split3_pair(a, ph[u], pm[u], pl[u]);
      }
      // the terms of tile t - 1 have been read by its GEMM2 once a_free completes
      if (t >= 1 && !wait_warp(&a_free, (t - 1) & 1)) { ok = false; break; }
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {  // 16-byte chunk 2 g + cc: units 16 g + 8 cc .. + 7
        const uint32_t off = sw_chunk(x, 2 * g + cc);
        *reinterpret_cast<uint4 *>(sA + off) = make_uint4(ph[4 * cc], ph[4 * cc + 1], ph[4 * cc + 2], ph[4 * cc + 3]);
        *reinterpret_cast<uint4 *>(sA + ATERM_BYTES + off) =
            make_uint4(pm[4 * cc], pm[4 * cc + 1], pm[4 * cc + 2], pm[4 * cc + 3]);
        *reinterpret_cast<uint4 *>(sA + 2 * ATERM_BYTES + off) =
            make_uint4(pl[4 * cc], pl[4 * cc + 1], pl[4 * cc + 2], pl[4 * cc + 3]);
      }
      }
      tc::fence_proxy_async_smem();
      mbar_arrive(&a_full);
      if (t + 2 < T) {  // spin buffer of tile t + 2, last read by GEMM2 of tile t - 1
        if (t >= 1 && !wait(&spin_free[(t + 2) % FTC_NS], ((t - 1) / FTC_NS) & 1)) { ok = false; break; }
        produce(t + 2, word2);
      }
      if (t >= 1 && (t - 1) % FTC_DRAIN == FTC_DRAIN - 1) ok = drain((t - 1) / FTC_DRAIN, false);
    }
    if (ok) {
      if (T > 0) drain((T - 1) / FTC_DRAIN, false);
      else drain(0, true);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == FTC_WORKERS) tc::tmem_dealloc(tmem_base, 512);
}

__global__ void crbm_force_tc_reduce_kernel(const double2 *part, int chunks, int64_t P, double inv_n, double2 *force) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < chunks; ++q) {  // fixed order: the result does not depend on timing
      const double2 v = part[q * P + k];
      s.x += v.x;
      s.y += v.y;
    }
    force[k] = make_double2(s.x * inv_n, s.y * inv_n);
  }
}

}  // namespace

bool rbm_force_tc_supported(const nqs_ctx *c) { return c->N <= 127; }

int rbm_force_tc_chunks(const nqs_ctx *c, int64_t n) {
  const int jt = (c->M + 1 + FTC_HT - 1) / FTC_HT;
  int64_t ch = std::max<int64_t>(1, c->num_sms / jt);
  ch = std::min<int64_t>(ch, (n + 127) / 128);
  return (int)std::max<int64_t>(1, ch);
}

cudaError_t rbm_force_tc(const nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                         double *ws, int chunks, cudaStream_t s) {
  ForceTcParams p;
  p.cfg = cfg;
  p.eloc = eloc;
  p.stats = stats;
  p.Wm = c->d_Wm;
  p.bm = c->d_bm;
  p.eloc_im = nullptr;
  p.Wc = nullptr;
  p.bc = nullptr;
  p.ws = ws;
  p.status = c->d_status;
  p.n = n;
  p.P = c->P;
  p.N = c->N;
  p.W = c->W;
  p.M = c->M;
  p.M_pad = c->M;
  p.n_chunks = chunks;
  const int jt = (c->M + 1 + FTC_HT - 1) / FTC_HT;
  cudaError_t e =
      cudaFuncSetAttribute(rbm_force_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FTC_SMEM);
  if (e != cudaSuccess) return e;
  rbm_force_tc_kernel<false><<<dim3(jt, chunks), FTC_THREADS, FTC_SMEM, s>>>(p);
  return cudaGetLastError();
}

int crbm_force_tc_chunks(int M, int num_sms, int64_t n) {
  const int jt = (M + 1 + FTC_HT / 2 - 1) / (FTC_HT / 2);
  int64_t ch = std::max<int64_t>(1, num_sms / jt);
  ch = std::min<int64_t>(ch, (n + 127) / 128);
  return (int)std::max<int64_t>(1, ch);
}

cudaError_t crbm_force_tc(const uint32_t *cfg, int64_t n, int N, int W, int M, int M_pad, int64_t P, const float2 *Wt,
                          const float2 *b, const float *eloc_re, const float *eloc_im, const double *stats,
                          double2 *part, int chunks, double2 *force, int *status, cudaStream_t s) {
  ForceTcParams p;
  p.cfg = cfg;
  p.eloc = eloc_re;
  p.eloc_im = eloc_im;
  p.stats = stats;
  p.Wm = nullptr;
  p.bm = nullptr;
  p.Wc = Wt;
  p.bc = b;
  p.ws = reinterpret_cast<double *>(part);
  p.status = status;
  p.n = n;
  p.P = P;
  p.N = N;
  p.W = W;
  p.M = M;
  p.M_pad = M_pad;
  p.n_chunks = chunks;
  const int jt = (M + 1 + FTC_HT / 2 - 1) / (FTC_HT / 2);
  cudaError_t e =
      cudaFuncSetAttribute(rbm_force_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FTC_SMEM);
  if (e != cudaSuccess) return e;
  rbm_force_tc_kernel<true><<<dim3(jt, chunks), FTC_THREADS, FTC_SMEM, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  crbm_force_tc_reduce_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 1024)), 256, 0, s>>>(
      part, chunks, P, 1.0 / (double)n, force);
  return cudaGetLastError();
}

}  // namespace nqs
