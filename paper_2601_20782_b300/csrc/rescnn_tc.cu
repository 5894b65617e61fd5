// ResCNN (App. H): the 16-bit (BF16 or F16) sampling copies, convolutions on the tensor cores.
//
// Sampling copy: the convolution kernels (embedding included) rounded to the 16-bit type; the
// activations that enter a tensor-core convolution (phi(LN(h)) and phi(Conv(.))) rounded to
// it; biases, LN parameters, the residual stream h, every accumulation and the final sum in
// FP32 (App. I: reductions in higher precision).  GELU is y sigma(2u) = y / (1 + e^{-2u}),
// u = sqrt(2/pi)(y + 0.044715 y^3), the tanh form rewritten, with ex2.approx / rcp.approx.
//
// Implicit GEMM.  A CTA holds G configurations, each on its lattice padded by a one-site halo
// ((Lx + 2) x (Ly + 2) rows; halo rows hold the periodic images).  The input of a convolution
// is stored as two 16-byte planes (channels 0-7 and 8-15), one 16-byte row per padded site.
// For tap (dy, dx) the A operand of an output tile of 128 rows is the same planes read from a
// row offset (dy - 1)(Lx + 2) + (dx - 1) away: a K-major operand without swizzle whose 8-row
// core matrices are 128 bytes apart (SBO) and whose two K halves are a plane apart (LBO).  One
// tcgen05.mma (M 128, N 16, K 16) per tile and tap accumulates in TMEM (16 FP32 columns per
// tile).  Halo and tail rows compute garbage that is never read.
//
// The residual streams h live in TMEM beside the accumulators (columns 128 + 16 t of tile t),
// so a thread needs few registers and two CTAs share an SM: one CTA's epilogue runs while the
// other's products do.  Warp w reads TMEM lane quarter w % 4 of the tiles t = w / 4 + 4 k, so a
// thread owns the same up to two padded rows through the whole pass.  One thread issues the
// products of a convolution tile by tile, committing each tile to its own mbarrier, so the
// epilogue of a tile starts while the later tiles' products run; every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "rescnn.cuh"
#include "tc.cuh"

namespace nqs {
namespace cnn {
namespace {

constexpr int TC_THREADS = 512;  // 16 warps: four groups of four warps (one per TMEM lane quarter)
constexpr int TC_GROUPS = TC_THREADS / 128;
constexpr int MAX_TILES = 8;     // accumulators in columns 0 .. 127, residual streams in 128 .. 255
constexpr int ROWS_PT = (MAX_TILES + TC_GROUPS - 1) / TC_GROUPS;  // rows owned per thread
constexpr int TILE_BYTES = 512;                                 // one tap: 16 x 16 16-bit values
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t H_COL = 128;  // first TMEM column of the residual streams
constexpr uint32_t TC_WAIT_POLLS = 1u << 22;
constexpr int SMALL_FLOATS = 10 * CF;  // k0 (9 x 16) and b0

template <typename TT>
struct Cvt;
template <>
struct Cvt<__nv_bfloat16> {
  __device__ static uint32_t pack(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
  }
  __host__ __device__ static constexpr uint32_t idesc() { return tc::idesc_bf16_f32(128, 16); }
  __device__ static float round(double v) { return __bfloat162float(__double2bfloat16(v)); }
  __device__ static uint16_t bits(double v) {
    __nv_bfloat16 b = __double2bfloat16(v);
    return *reinterpret_cast<uint16_t *>(&b);
  }
};
template <>
struct Cvt<__half> {
  __device__ static uint32_t pack(float a, float b) {
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
  }
  __host__ __device__ static constexpr uint32_t idesc() { return tc::idesc_f16_f32(128, 16); }
  __device__ static float round(double v) { return __half2float(__double2half(v)); }
  __device__ static uint16_t bits(double v) {
    __half b = __double2half(v);
    return *reinterpret_cast<uint16_t *>(&b);
  }
};

// Master -> (a) the copy's FP32 values in kernel order (kernels rounded to TT) and (b) the B
// tiles: block l, convolution w (0, 1), tap: element (co, ci) at (ci / 8) 128 + co 8 + ci % 8.
template <typename TT>
__global__ void rescnn_prepare_lp_kernel(const double *master, int n_blocks, float *cw, uint16_t *tiles) {
  const int P = n_params(n_blocks);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    int src = k;
    bool kern = false;
    if (k < 9 * CF) {
      const int tap = k / CF, co = k % CF;
      src = co * 9 + tap;
      kern = true;
    } else if (k >= 10 * CF && k < 10 * CF + n_blocks * BLOCK_FLOATS) {
      const int blk = (k - 10 * CF) / BLOCK_FLOATS;
      const int base = 10 * CF + blk * BLOCK_FLOATS;
      const int r = k - base;
      int kb = -1, w = 0;
      if (r >= OFF_K1 && r < OFF_K1 + 9 * CF * CF) kb = OFF_K1;
      if (r >= OFF_K2 && r < OFF_K2 + 9 * CF * CF) kb = OFF_K2, w = 1;
      if (kb >= 0) {
        const int e = r - kb, tap = e / (CF * CF), ci = (e / CF) % CF, co = e % CF;
        src = base + kb + (co * CF + ci) * 9 + tap;
        kern = true;
        tiles[((blk * 2 + w) * 9 + tap) * 256 + (ci / 8) * 128 + co * 8 + ci % 8] = Cvt<TT>::bits(master[src]);
      }
    }
    cw[k] = kern ? Cvt<TT>::round(master[src]) : (float)master[src];
  }
}

__device__ __forceinline__ float gelu_lp(float y) {  // y / (1 + e^{-2u})
  const float u = GELU_C * fmaf(0.044715f * y * y, y, y);
  return y * rcp_approx(1.f + ex2_approx(-2.f * LOG2EF * u));
}

__device__ __forceinline__ void ln16(const float (&v)[CF], const float *g, const float *be, float (&y)[CF]) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) m += v[c];
  m *= 1.f / CF;
  float var = 0.f;
#pragma unroll
  for (int c = 0; c < CF; ++c) {
    const float d = v[c] - m;
    var = fmaf(d, d, var);
  }
  const float rs = rsqrtf(fmaf(var, 1.f / CF, LN_EPS));
#pragma unroll
  for (int c = 0; c < CF; ++c) y[c] = fmaf((v[c] - m) * rs, g[c], be[c]);
}

struct TcGeom {
  int Lx, Ly, Lxp, Rp, N, G, T, GR, plane_rows, n_blocks;
};

struct TcArgs {
  TcGeom gm;
  const float *cw;        // FP32 values of the copy, kernel order
  const uint16_t *tiles;  // [n_blocks][2][9][256]
  int *status;
  int W;
  const uint32_t *cfg;
  int64_t n_cfg;
  float *out;
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

// Shared-memory carve (offsets in bytes from a 128-aligned base); the host uses the same.
struct TcLayout {
  uint32_t planes, tiles, small, blockp, spin, rowsum, chain, halo, total;
  __host__ __device__ static TcLayout make(const TcGeom &g) {
    TcLayout L;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes) {
      const uint32_t r = o;
      o = (o + bytes + 127u) & ~127u;
      return r;
    };
    L.planes = take(2u * g.plane_rows * 16u);
    L.tiles = take((uint32_t)g.n_blocks * 2u * 9u * TILE_BYTES);
    L.small = take(SMALL_FLOATS * 4u);
    L.blockp = take((uint32_t)(g.n_blocks * 4 + 2) * CF * 4u);  // per block g, be, b1, b2; final g, be
    L.spin = take((uint32_t)g.G * g.N * 4u);
    L.rowsum = take((uint32_t)g.T * 128u * 4u);
    L.chain = take((uint32_t)g.G * 40u);  // flip, lp, thr, lpx (4 x 4 B) + Philox block (16 B) + spare
    L.halo = take((uint32_t)g.G * (uint32_t)(g.Rp - g.N) * 4u);  // halo row -> image row pairs
    L.total = o;
    return L;
  }
};

template <typename TT>
struct Cta {
  const TcGeom &gm;
  unsigned char *base;
  TcLayout L;
  uint64_t *bars;  // [MAX_TILES]: products of tile t done
  uint32_t tmem;
  uint32_t phase;

  __device__ unsigned char *planes() const { return base + L.planes; }
  __device__ const float *small() const { return reinterpret_cast<const float *>(base + L.small); }
  __device__ const float *blockp(int l) const { return reinterpret_cast<const float *>(base + L.blockp) + l * 4 * CF; }
  __device__ float *spin() const { return reinterpret_cast<float *>(base + L.spin); }
  __device__ float *rowsum() const { return reinterpret_cast<float *>(base + L.rowsum); }
  __device__ int *flip() const { return reinterpret_cast<int *>(base + L.chain); }
  __device__ float *lp() const { return reinterpret_cast<float *>(base + L.chain) + gm.G; }
  __device__ float *thr() const { return reinterpret_cast<float *>(base + L.chain) + 2 * gm.G; }
  __device__ float *lpx() const { return reinterpret_cast<float *>(base + L.chain) + 3 * gm.G; }
  __device__ uint4 *pw() const {
    return reinterpret_cast<uint4 *>(base + L.chain + ((16u * gm.G + 15u) & ~15u));
  }
  // TMEM addresses of this warp's lane quarter: accumulator and residual stream of tile t
  __device__ uint32_t acc_addr(int t) const {
    return tc::tmem_lane_addr(tmem, 32u * ((threadIdx.x >> 5) & 3u), 16u * (uint32_t)t);
  }
  __device__ uint32_t h_addr(int t) const {
    return tc::tmem_lane_addr(tmem, 32u * ((threadIdx.x >> 5) & 3u), H_COL + 16u * (uint32_t)t);
  }

  // 16-bit activations of one padded row (plane row GR + R)
  __device__ void store_act(int R, const float (&v)[CF]) const {
    uint4 lo, hi;
    lo.x = Cvt<TT>::pack(v[0], v[1]);
    lo.y = Cvt<TT>::pack(v[2], v[3]);
    lo.z = Cvt<TT>::pack(v[4], v[5]);
    lo.w = Cvt<TT>::pack(v[6], v[7]);
    hi.x = Cvt<TT>::pack(v[8], v[9]);
    hi.y = Cvt<TT>::pack(v[10], v[11]);
    hi.z = Cvt<TT>::pack(v[12], v[13]);
    hi.w = Cvt<TT>::pack(v[14], v[15]);
    uint4 *p0 = reinterpret_cast<uint4 *>(planes() + (size_t)(gm.GR + R) * 16u);
    p0[0] = lo;
    p0[gm.plane_rows] = hi;
  }

  // halo rows <- their periodic images (every configuration of the CTA), then make the planes
  // visible to the tensor core.  Returns false if any thread saw a timed-out wait (`bad`).
  __device__ bool fill_halo(bool bad) const {
    tc::fence_before_sync();
    if (__syncthreads_or(bad)) return false;
    uint4 *p = reinterpret_cast<uint4 *>(planes() + (size_t)gm.GR * 16u);
    const uint32_t *pairs = reinterpret_cast<const uint32_t *>(base + L.halo);
    for (int e = threadIdx.x; e < gm.G * (gm.Rp - gm.N); e += blockDim.x) {
      const uint32_t v = pairs[e];
      const int dst = (int)(v >> 16), src = (int)(v & 0xFFFFu);
      p[dst] = p[src];
      p[dst + gm.plane_rows] = p[src + gm.plane_rows];
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    return true;
  }

  // Issues one convolution (block l, w = 0 for K1, 1 for K2), tile by tile, each tile committed
  // to bars[t].  Called by thread 0 after the CTA barrier of fill_halo.  A descriptor's address
  // field counts 16-byte units, so a row offset r is added to it as the integer r.
  __device__ void issue_conv(int l, int w) const {
    tc::fence_after_sync();
    const uint64_t a0 = tc::desc_noswz(smem_addr(planes()), (uint32_t)gm.plane_rows * 16u, 128u);
    const uint64_t b0 = tc::desc_noswz(smem_addr(base + L.tiles) + (uint32_t)((l * 2 + w) * 9) * TILE_BYTES, 256u, 128u);
    const int o0 = gm.GR - gm.Lxp - 1;  // row offset of tap (0, 0) from the tile start
    for (int t = 0; t < gm.T; ++t) {
      const uint32_t d = tmem + 16u * t;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const uint64_t ad = a0 + (uint64_t)(o0 + 128 * t + (tap / 3) * gm.Lxp + tap % 3);
        tc::mma_bf16(d, ad, b0 + (uint64_t)(tap * (TILE_BYTES / 16)), Cvt<TT>::idesc(), tap > 0 ? 1u : 0u);
      }
      tc::mma_commit(&bars[t]);
    }
  }

  // Waits for the products of tile t (this warp's epilogue); false after the poll limit.
  // The result is the same on every lane (the TMEM loads that follow are warp-collective).
  __device__ bool wait_tile(int t, int *status) const {
    const bool ok = __all_sync(FULL_MASK, mbar_wait_bounded(&bars[t], phase, TC_WAIT_POLLS));
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_TIMEOUT);
    tc::fence_after_sync();
    return ok;
  }

  // The planes hold the input of the convolution in flight, and the epilogue writes the next
  // one's input into them: a tile's rows may be overwritten once no product still to finish
  // reads them.  A tile's shifted windows reach Lx + 3 rows (< 128) either side, so only tile
  // t + 1 reads rows of tile t; its barrier (tiles commit in order) covers every earlier tile.
  __device__ bool wait_overwrite(int t, int *status) const {
    if (t + 1 >= gm.T) return true;
    const bool ok = __all_sync(FULL_MASK, mbar_wait_bounded(&bars[t + 1], phase, TC_WAIT_POLLS));
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_TIMEOUT);
    return ok;
  }

  // After a timed-out wait: give every product in flight the poll limit again before TMEM is freed.
  __device__ void drain() const {
    if (threadIdx.x == 0)
      for (int t = 0; t < gm.T; ++t) mbar_wait_bounded(&bars[t], phase, TC_WAIT_POLLS);
    __syncthreads();
  }
};

// Row bookkeeping of one thread: rows R_k = 128 t_k + 32 (warp % 4) + lane, t_k = warp / 4 + 4 k;
// per row one word: configuration << 16 | site for an interior row, NONE otherwise.
struct OwnRows {
  static constexpr uint32_t NONE = 0xFFFFFFFFu;
  uint32_t info[ROWS_PT];
  __device__ static int tile(int k) { return (int)(threadIdx.x >> 7) + TC_GROUPS * k; }
  __device__ static int row(int k) { return 128 * tile(k) + (int)(threadIdx.x & 127u); }
  __device__ bool interior(int k) const { return info[k] != NONE; }
  __device__ int site(int k) const { return (int)(info[k] & 0xFFFFu); }
  __device__ int cfg(int k) const { return (int)(info[k] >> 16); }
  __device__ void init(const TcGeom &gm) {
#pragma unroll
    for (int k = 0; k < ROWS_PT; ++k) {
      const int R = row(k);
      const int g0 = R / gm.Rp, pos = R - g0 * gm.Rp;
      const int py = pos / gm.Lxp, px = pos - py * gm.Lxp;
      const bool in = tile(k) < gm.T && g0 < gm.G && px >= 1 && px <= gm.Lx && py >= 1 && py <= gm.Ly;
      info[k] = in ? ((uint32_t)g0 << 16) | (uint32_t)((px - 1) + gm.Lx * (py - 1)) : NONE;
    }
  }
};

// phi(LN(h)) of one row with the LN parameters at bp (gamma, beta), as 16-bit activations
template <typename TT>
__device__ __forceinline__ void ln_gelu_store(const Cta<TT> &cta, int R, const float (&h)[CF], const float *bp) {
  float y[CF];
  ln16(h, bp, bp + CF, y);
#pragma unroll
  for (int c = 0; c < CF; ++c) y[c] = gelu_lp(y[c]);
  cta.store_act(R, y);
}

// log psi of the CTA's G configurations (spins with flips) into lp(); false on a timed-out
// wait (STATUS_TIMEOUT recorded, products drained).
template <typename TT>
__device__ __forceinline__ bool forward_tc(Cta<TT> &cta, const OwnRows &own, int *status) {
  const TcGeom &gm = cta.gm;
  const float *sp = cta.small();
  // embedding h = b0 + sum_tap k0[tap] s(neighbour) into TMEM, then phi(LN(h)) of block 0
#pragma unroll
  for (int k = 0; k < ROWS_PT; ++k) {
    if (OwnRows::tile(k) >= gm.T) continue;  // uniform per warp
    float h[CF];
#pragma unroll
    for (int c = 0; c < CF; ++c) h[c] = sp[9 * CF + c];
    if (own.interior(k)) {
      const int g = own.cfg(k), x = own.site(k) % gm.Lx, yy = own.site(k) / gm.Lx;
      const int fl = cta.flip()[g];
      const float *s = cta.spin() + g * gm.N;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        int xx = x + tap % 3 - 1, y2 = yy + tap / 3 - 1;
        xx += xx < 0 ? gm.Lx : (xx >= gm.Lx ? -gm.Lx : 0);
        y2 += y2 < 0 ? gm.Ly : (y2 >= gm.Ly ? -gm.Ly : 0);
        const int j = xx + gm.Lx * y2;
        const float sv = j == fl ? -s[j] : s[j];
#pragma unroll
        for (int c = 0; c < CF; ++c) h[c] = fmaf(sp[tap * CF + c], sv, h[c]);
      }
      if (gm.n_blocks > 0) ln_gelu_store(cta, OwnRows::row(k), h, cta.blockp(0));
    }
    tc::tmem_st16(cta.h_addr(OwnRows::tile(k)), h);
  }
  tc::tmem_wait_st();
  bool bad = false;
  for (int l = 0; l < gm.n_blocks; ++l) {
    const float *bp = cta.blockp(l);
    for (int w = 0; w < 2; ++w) {
      if (!cta.fill_halo(bad)) {
        cta.drain();
        return false;
      }
      if (threadIdx.x == 0) cta.issue_conv(l, w);
#pragma unroll
      for (int k = 0; k < ROWS_PT; ++k) {
        const int t = OwnRows::tile(k);
        if (t >= gm.T) continue;
        if (!cta.wait_tile(t, status)) {
          bad = true;
          continue;
        }
        uint32_t ra[CF], rh[CF];
        tc::tmem_ld16_async(cta.acc_addr(t), ra);
        if (w == 1) tc::tmem_ld16_async(cta.h_addr(t), rh);
        tc::tmem_wait_ld();
        float v[CF];
        if (w == 0) {  // c = phi(K1 * a + b1)
#pragma unroll
          for (int c = 0; c < CF; ++c) v[c] = gelu_lp(__uint_as_float(ra[c]) + bp[2 * CF + c]);
          if (!cta.wait_overwrite(t, status)) {  // warp-uniform
            bad = true;
            continue;
          }
          if (own.interior(k)) cta.store_act(OwnRows::row(k), v);
        } else {  // h += K2 * c + b2, then phi(LN(h)) of the next block
#pragma unroll
          for (int c = 0; c < CF; ++c) v[c] = __uint_as_float(rh[c]) + (__uint_as_float(ra[c]) + bp[3 * CF + c]);
          tc::tmem_st16(cta.h_addr(t), v);  // warp-collective: every lane, halo rows included
          if (l + 1 < gm.n_blocks) {
            if (!cta.wait_overwrite(t, status)) {  // warp-uniform
              bad = true;
              continue;
            }
            if (own.interior(k)) ln_gelu_store(cta, OwnRows::row(k), v, cta.blockp(l + 1));
          }
        }
      }
      if (w == 1) tc::tmem_wait_st();
      cta.phase ^= 1u;
    }
  }
  tc::fence_before_sync();
  if (__syncthreads_or(bad)) {
    cta.drain();
    return false;
  }
  tc::fence_after_sync();
  // final LN of the residual streams and the per-row sums
  const float *fp = cta.blockp(gm.n_blocks);
#pragma unroll
  for (int k = 0; k < ROWS_PT; ++k) {
    const int t = OwnRows::tile(k);
    if (t >= gm.T) continue;
    uint32_t rh[CF];
    tc::tmem_ld16_async(cta.h_addr(t), rh);
    tc::tmem_wait_ld();
    if (!own.interior(k)) continue;
    float h[CF], y[CF];
#pragma unroll
    for (int c = 0; c < CF; ++c) h[c] = __uint_as_float(rh[c]);
    ln16(h, fp, fp + CF, y);
    float rs = 0.f;
#pragma unroll
    for (int c = 0; c < CF; ++c) rs += y[c];
    cta.rowsum()[OwnRows::row(k)] = rs;
  }
  tc::fence_before_sync();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int g = warp; g < gm.G; g += blockDim.x >> 5) {
    float s = 0.f;
    for (int i = lane; i < gm.N; i += 32)
      s += cta.rowsum()[g * gm.Rp + (i / gm.Lx + 1) * gm.Lxp + (i % gm.Lx) + 1];
    s = group_allsum<32>(s);
    if (lane == 0) cta.lp()[g] = s;
  }
  __syncthreads();
  return true;
}

// CTA set-up: parameters and tiles into shared memory, planes cleared, barrier and TMEM.
template <typename TT>
__device__ void setup_cta(Cta<TT> &cta, const TcArgs &a, uint32_t *tmem_slot) {
  const TcGeom &gm = a.gm;
  uint4 *pl = reinterpret_cast<uint4 *>(cta.planes());
  for (int i = threadIdx.x; i < 2 * gm.plane_rows; i += blockDim.x) pl[i] = make_uint4(0u, 0u, 0u, 0u);
  const uint4 *tsrc = reinterpret_cast<const uint4 *>(a.tiles);
  uint4 *tdst = reinterpret_cast<uint4 *>(cta.base + cta.L.tiles);
  for (int i = threadIdx.x; i < gm.n_blocks * 2 * 9 * TILE_BYTES / 16; i += blockDim.x) tdst[i] = tsrc[i];
  float *sm = reinterpret_cast<float *>(cta.base + cta.L.small);
  for (int i = threadIdx.x; i < SMALL_FLOATS; i += blockDim.x) sm[i] = a.cw[i];
  float *bp = reinterpret_cast<float *>(cta.base + cta.L.blockp);
  for (int i = threadIdx.x; i < (gm.n_blocks * 4 + 2) * CF; i += blockDim.x) {
    const int l = i / (4 * CF), q = (i / CF) % 4, c = i % CF;
    float v;
    if (l < gm.n_blocks) {
      const int off = q == 0 ? OFF_G : q == 1 ? OFF_BE : q == 2 ? OFF_B1 : OFF_B2;
      v = a.cw[10 * CF + l * BLOCK_FLOATS + off + c];
    } else {
      v = a.cw[10 * CF + gm.n_blocks * BLOCK_FLOATS + q * CF + c];  // final gamma (q = 0), beta (q = 1)
    }
    bp[i] = v;
  }
  // the halo rows of every configuration with their periodic images, (row << 16 | image row)
  // in rows from the first padded row: one thread per configuration, in position order
  uint32_t *pairs = reinterpret_cast<uint32_t *>(cta.base + cta.L.halo);
  for (int g = threadIdx.x; g < gm.G; g += blockDim.x) {
    int q = g * (gm.Rp - gm.N);
    for (int pos = 0; pos < gm.Rp; ++pos) {
      const int py = pos / gm.Lxp, px = pos - py * gm.Lxp;
      if (px >= 1 && px <= gm.Lx && py >= 1 && py <= gm.Ly) continue;
      const int sy = (py - 1 + gm.Ly) % gm.Ly + 1, sx = (px - 1 + gm.Lx) % gm.Lx + 1;
      pairs[q++] = ((uint32_t)(g * gm.Rp + pos) << 16) | (uint32_t)(g * gm.Rp + sy * gm.Lxp + sx);
    }
  }
  if (threadIdx.x == 0) {
    for (int t = 0; t < MAX_TILES; ++t) mbar_init(&cta.bars[t], 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tmem_slot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  cta.tmem = *tmem_slot;
  cta.phase = 0;
}

template <typename TT>
__device__ void teardown_cta(Cta<TT> &cta) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(cta.tmem, TMEM_COLS);
}

__device__ __forceinline__ float log_uniform_tc(uint32_t w) {
  const uint32_t k = w >> 8;
  return k == 0u ? -INFINITY : logf((float)k * 5.9604644775390625e-8f);
}

__device__ __forceinline__ unsigned char *aligned_base(unsigned char *raw) {
  const uint32_t a = smem_addr(raw);
  return raw + (((a + 127u) & ~127u) - a);
}

// MODE 0: log psi of cfg[q]; MODE 1: the N + 1 local-energy configurations of each sample.
template <typename TT, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 2) rescnn_tc_eval_kernel(const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bars[MAX_TILES];
  __shared__ uint32_t tmem_slot;
  const TcGeom &gm = a.gm;
  Cta<TT> cta{gm, aligned_base(smem_raw), TcLayout::make(gm), bars, 0u, 0u};
  setup_cta(cta, a, &tmem_slot);
  OwnRows own;
  own.init(gm);
  const int N = gm.N, G = gm.G;
  const int64_t n_groups = (a.n_cfg + G - 1) / G;
  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t q0 = grp * G;
    const int Gv = (int)std::min<int64_t>(G, a.n_cfg - q0);
    for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
      const int g = e / N, i = e % N;
      const int64_t q = q0 + std::min(g, Gv - 1);
      const int64_t x = MODE == 0 ? q : q / (N + 1);
      cta.spin()[e] = ((a.cfg[x * a.W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x)
      cta.flip()[g] = MODE == 0 ? -1 : (int)((q0 + std::min(g, Gv - 1)) % (N + 1)) - 1;
    __syncthreads();
    if (!forward_tc(cta, own, a.status)) break;
    for (int g = threadIdx.x; g < Gv; g += blockDim.x) a.out[q0 + g] = cta.lp()[g];
    __syncthreads();
  }
  teardown_cta(cta);
}

// Metropolis sweeps with the Philox layout, decision rule and traces of the FP32 path.
template <typename TT>
__global__ void __launch_bounds__(TC_THREADS, 2) rescnn_tc_sweep_kernel(const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bars[MAX_TILES];
  __shared__ uint32_t tmem_slot;
  const TcGeom &gm = a.gm;
  Cta<TT> cta{gm, aligned_base(smem_raw), TcLayout::make(gm), bars, 0u, 0u};
  setup_cta(cta, a, &tmem_slot);
  OwnRows own;
  own.init(gm);
  const int N = gm.N, G = gm.G, W = a.W;
  const int64_t n_groups = (a.C + G - 1) / G;
  bool alive = true;
  for (int64_t grp = blockIdx.x; grp < n_groups && alive; grp += gridDim.x) {
    const int64_t c0 = grp * G;
    const int Gv = (int)std::min<int64_t>(G, a.C - c0);
    for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
      const int g = e / N, i = e % N;
      const int64_t c = c0 + std::min(g, Gv - 1);
      cta.spin()[e] = ((a.state[c * W + (i >> 5)] >> (i & 31)) & 1u) ? 1.f : -1.f;
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) cta.flip()[g] = -1;
    __syncthreads();
    if (!forward_tc(cta, own, a.status)) break;
    for (int g = threadIdx.x; g < G; g += blockDim.x) cta.lpx()[g] = cta.lp()[g];
    int64_t nacc = 0;
    uint32_t abits = 0u;
    for (int t = 0; t < a.n_sweeps && alive; ++t) {
      const uint32_t sweep_id = a.sweep_offset + (uint32_t)t;
      for (int p = 0; p < N; ++p) {
        if (threadIdx.x < G) {
          const int g = threadIdx.x;
          const int64_t c = c0 + std::min(g, Gv - 1);
          if ((p & 1) == 0)
            cta.pw()[g] = philox4x32_10(make_uint4((uint32_t)(p / 2), sweep_id, (uint32_t)c, TAG_SWEEP), a.k0, a.k1);
          const uint4 w4 = cta.pw()[g];
          cta.flip()[g] = (int)index_from_word((p & 1) ? w4.z : w4.x, (uint32_t)N);
          cta.thr()[g] = log_uniform_tc((p & 1) ? w4.w : w4.y);
        }
        __syncthreads();
        if (!forward_tc(cta, own, a.status)) {
          alive = false;
          break;
        }
        if (threadIdx.x < Gv) {
          const int g = threadIdx.x;
          const int64_t c = c0 + g;
          const float dlt = cta.lp()[g] - cta.lpx()[g];
          const bool acc = 2.f * dlt > cta.thr()[g];
          if (acc) {
            const int site = cta.flip()[g];
            cta.spin()[g * N + site] = -cta.spin()[g * N + site];
            cta.lpx()[g] = cta.lp()[g];
            ++nacc;
          }
          if (a.acc_bits) {
            abits |= (acc ? 1u : 0u) << (p & 31);
            if ((p & 31) == 31 || p == N - 1) {
              a.acc_bits[(c * a.n_sweeps + t) * W + (p >> 5)] = abits;
              abits = 0u;
            }
          }
          if (a.delta) a.delta[(c * a.n_sweeps + t) * N + p] = dlt;
        }
        __syncthreads();
      }
      if (alive && t >= a.burn_in) {
        const int64_t row0 = (int64_t)(t - a.burn_in) * a.C;
        for (int e = threadIdx.x; e < Gv * W; e += blockDim.x) {
          const int g = e / W, wi = e % W;
          uint32_t word = 0u;
          for (int b = 0; b < 32 && 32 * wi + b < N; ++b)
            if (cta.spin()[g * N + 32 * wi + b] > 0.f) word |= 1u << b;
          if (a.samples) a.samples[(row0 + c0 + g) * W + wi] = word;
        }
        if (a.logpsi)
          for (int g = threadIdx.x; g < Gv; g += blockDim.x) a.logpsi[row0 + c0 + g] = cta.lpx()[g];
      }
    }
    if (!alive) break;
    __syncthreads();
    for (int e = threadIdx.x; e < Gv * W; e += blockDim.x) {
      const int g = e / W, wi = e % W;
      uint32_t word = 0u;
      for (int b = 0; b < 32 && 32 * wi + b < N; ++b)
        if (cta.spin()[g * N + 32 * wi + b] > 0.f) word |= 1u << b;
      a.state[(c0 + g) * W + wi] = word;
    }
    if (threadIdx.x < Gv && a.n_acc) a.n_acc[c0 + threadIdx.x] = nacc;
    __syncthreads();
  }
  teardown_cta(cta);
}

TcGeom geometry(const nqs_ctx *c) {
  TcGeom g;
  g.Lx = c->Lx;
  g.Ly = c->Ly;
  g.Lxp = c->Lx + 2;
  g.Rp = (c->Lx + 2) * (c->Ly + 2);
  g.N = c->N;
  g.G = std::max(1, (MAX_TILES * 128) / g.Rp);
  while (g.G > 1 && (g.G * g.Rp + 127) / 128 > MAX_TILES) --g.G;
  g.T = (g.G * g.Rp + 127) / 128;
  g.GR = ((g.Lxp + 1 + 7) / 8) * 8;
  g.plane_rows = g.GR + 128 * g.T + g.GR;
  g.n_blocks = c->n_blocks;
  return g;
}

template <typename TT>
TcArgs base_args(const nqs_ctx *c) {
  TcArgs a{};
  a.gm = geometry(c);
  a.cw = c->d_cw_lp;
  a.tiles = c->d_ctile;
  a.status = c->d_status;
  a.W = c->W;
  return a;
}

template <typename K>
cudaError_t launch_tc(const nqs_ctx *c, K kern, const TcArgs &a, int64_t groups, cudaStream_t s) {
  const size_t shm = TcLayout::make(a.gm).total + 128;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(groups, 2 * (int64_t)c->num_sms));  // two CTAs per SM
  kern<<<(unsigned)grid, TC_THREADS, shm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace cnn

bool rescnn_lp_supported(const nqs_ctx *c) {
  if (c->dtype != NQS_BF16 && c->dtype != NQS_F16) return false;
  const cnn::TcGeom g = cnn::geometry(c);
  return g.T <= cnn::MAX_TILES && cnn::TcLayout::make(g).total + 128 <= (uint32_t)c->smem_optin;
}

cudaError_t rescnn_lp_alloc(nqs_ctx *c) {
  cudaError_t e = cudaMalloc(&c->d_cw_lp, (size_t)c->P * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMalloc(&c->d_ctile, (size_t)std::max(c->n_blocks, 1) * 2 * 9 * 256 * sizeof(uint16_t));
}

void rescnn_lp_free(nqs_ctx *c) {
  if (c->d_cw_lp) cudaFree(c->d_cw_lp);
  if (c->d_ctile) cudaFree(c->d_ctile);
  c->d_cw_lp = nullptr;
  c->d_ctile = nullptr;
}

cudaError_t rescnn_lp_prepare(nqs_ctx *c, const double *params, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>((c->P + 255) / 256, 1024);
  if (c->dtype == NQS_F16)
    cnn::rescnn_prepare_lp_kernel<__half><<<blocks, 256, 0, s>>>(params, c->n_blocks, c->d_cw_lp, c->d_ctile);
  else
    cnn::rescnn_prepare_lp_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(params, c->n_blocks, c->d_cw_lp, c->d_ctile);
  return cudaGetLastError();
}

namespace {
template <int MODE>
cudaError_t tc_eval(const nqs_ctx *c, const uint32_t *cfg, int64_t n_cfg, float *out, cudaStream_t s) {
  if (c->dtype == NQS_F16) {
    cnn::TcArgs a = cnn::base_args<__half>(c);
    a.cfg = cfg;
    a.n_cfg = n_cfg;
    a.out = out;
    return cnn::launch_tc(c, cnn::rescnn_tc_eval_kernel<__half, MODE>, a, (n_cfg + a.gm.G - 1) / a.gm.G, s);
  }
  cnn::TcArgs a = cnn::base_args<__nv_bfloat16>(c);
  a.cfg = cfg;
  a.n_cfg = n_cfg;
  a.out = out;
  return cnn::launch_tc(c, cnn::rescnn_tc_eval_kernel<__nv_bfloat16, MODE>, a, (n_cfg + a.gm.G - 1) / a.gm.G, s);
}
}  // namespace

cudaError_t rescnn_lp_logpsi(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  return tc_eval<0>(c, cfg, n, out, s);
}

cudaError_t rescnn_lp_eval_flips(const nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, cudaStream_t s) {
  return tc_eval<1>(c, cfg, n * (c->N + 1), out, s);
}

cudaError_t rescnn_lp_sweep(const nqs_ctx *c, uint32_t *state, int64_t C, int n_sweeps, int burn_in, uint64_t seed,
                            uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_acc,
                            uint32_t *acc_bits, float *delta, cudaStream_t s) {
  auto fill = [&](cnn::TcArgs &a) {
    a.state = state;
    a.C = C;
    a.n_sweeps = n_sweeps;
    a.burn_in = burn_in;
    a.sweep_offset = sweep_offset;
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.samples = samples;
    a.logpsi = logpsi;
    a.n_acc = n_acc;
    a.acc_bits = acc_bits;
    a.delta = delta;
  };
  if (c->dtype == NQS_F16) {
    cnn::TcArgs a = cnn::base_args<__half>(c);
    fill(a);
    return cnn::launch_tc(c, cnn::rescnn_tc_sweep_kernel<__half>, a, (C + a.gm.G - 1) / a.gm.G, s);
  }
  cnn::TcArgs a = cnn::base_args<__nv_bfloat16>(c);
  fill(a);
  return cnn::launch_tc(c, cnn::rescnn_tc_sweep_kernel<__nv_bfloat16>, a, (C + a.gm.G - 1) / a.gm.G, s);
}

}  // namespace nqs
