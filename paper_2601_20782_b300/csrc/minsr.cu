// minSR update (the SR solve of App. I in its S x S form, with diagonal shift lambda):
//
//   Obar = (O - mean_x O) / sqrt(n),  ebar = (eloc - E) / sqrt(n),  T = Obar Obar^T,
//   y = (T + lambda I)^-1 ebar,       dtheta = Obar^T y.
//
// Steps (all on the stream, FP64 wherever the solve's stability depends on it):
//   1. minsr_colmean_kernel   FP64 column means of O (one pass over O).
//   2. minsr_split_kernel     Obar' = O - mean (FP32), split into three BF16 terms
//                             hi + mid + lo (exact to ~2^-24 relative), stored K-block-major,
//                             [Pp/64][3][n_pad][64]: the six boxes of one K block then lie in
//                             3 n_pad 128 contiguous bytes.  (Row-major [3][n_pad][Pp] rows are
//                             2 Pp bytes apart, 4.7 MB at P = 2.4M, where the Gram ran 1.4x
//                             slower from that layout; at P = 0.5M the two timed the same.)
//   3. minsr_gram_kernel      T' = Obar' Obar'^T on the tensor cores: TMA loads of the three
//                             terms of a 128-row tile pair per 64-wide K block, six products
//                             (hh into one TMEM accumulator; hm, mh, hl, lh, mm into a second,
//                             so small terms are not rounded against the running sum), FP32
//                             accumulation for DRAIN K blocks, then FP64 partial sums per
//                             (K part, tile pair).  Upper tile pairs only (T is symmetric).
//   4. minsr_reduce_kernel    T = (1/n) sum over K parts, mirrored, + lambda on the diagonal.
//   5. Cholesky T + lambda I = L L^T in FP64 (blocked: diagonal block, panel, trailing update);
//      minsr_reduce_kernel also writes ebar.
//   6. L z = ebar along with the Cholesky (each diagonal block solves its triangle, each
//      panel updates the later rows); minsr_back_kernel: L^T y = z in 64-row blocks from the
//      last; minsr_ysum_kernel: sum_x y_x.
//   7. minsr_dtheta_kernel    dtheta_k = (sum_x O_xk y_x - mean_k sum_x y_x) / sqrt(n), FP64.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace nqs {
namespace {

constexpr int GRAM_THREADS = 320;  // warp 0 TMA, warp 1 MMA + TMEM, warps 2-9 drain
constexpr int GRAM_STAGES = 2;
constexpr int GRAM_DRAIN = 16;     // K blocks (of 64) accumulated in FP32 between FP64 drains
constexpr uint32_t GRAM_POLLS = 1u << 24;
constexpr int CHOL_NB = 64;

// FP32 sums over chunks of MINSR_CHUNK rows, FP64 across chunks: FP64 arithmetic is a small
// fraction of FP32 throughput on this part, and a 16-term FP32 sum carries at most 16 x 2^-24
// relative error before it reaches the FP64 total.
constexpr int MINSR_CHUNK = 16;

__global__ void minsr_colmean_kernel(const float *__restrict__ O, int64_t n, int64_t P, double *mean_d,
                                     float *mean_f) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t x0 = 0; x0 < n; x0 += MINSR_CHUNK) {
      float c = 0.f;
      const int m = (int)(n - x0 < MINSR_CHUNK ? n - x0 : MINSR_CHUNK);
#pragma unroll 4
      for (int q = 0; q < m; ++q) c += O[(x0 + q) * P + k];
      s += (double)c;
    }
    const double m = s / (double)n;
    mean_d[k] = m;
    mean_f[k] = (float)m;
  }
}

__device__ __forceinline__ void split3_bf16(float a, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(a);
  const float r = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

// S3[k / 64][t][x][k % 64] for x < n_pad, k < Pp (pairs of k per thread); zero outside n x P.
__global__ void minsr_split_kernel(const float *__restrict__ O, int64_t n, int64_t P, int64_t n_pad, int64_t Pp,
                                   const float *__restrict__ mean_f, __nv_bfloat16 *S3) {
  const int64_t half_cols = Pp / 2;
  const int64_t total = n_pad * half_cols;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q / half_cols, k = 2 * (q % half_cols);
    float v[2];
    for (int e = 0; e < 2; ++e) v[e] = (x < n && k + e < P) ? O[x * P + k + e] - mean_f[k + e] : 0.f;
    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
    split3_bf16(v[0], h0, m0, l0);
    split3_bf16(v[1], h1, m1, l1);
    const int64_t tb = n_pad * 64;
    const int64_t o = (k >> 6) * 3 * tb + x * 64 + (k & 63);
    *reinterpret_cast<__nv_bfloat162 *>(S3 + o) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162 *>(S3 + tb + o) = __halves2bfloat162(m0, m1);
    *reinterpret_cast<__nv_bfloat162 *>(S3 + 2 * tb + o) = __halves2bfloat162(l0, l1);
  }
}

// The K-block-major copy of the split terms, S3[kb][t][x][c] (64-wide K blocks, three terms of
// n_pad rows, 128-byte rows), as a 3D tensor map {c, t * n_pad + x, kb} with 128 x 64 boxes.
bool make_tmap_kblocks(CUtensorMap *map, const void *base, uint64_t n_pad, uint64_t kb_total) {
  using Fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                          const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                          CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Fn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<Fn>(p);
  }
  const cuuint64_t dims[3] = {64, 3 * n_pad, kb_total};
  const cuuint64_t strides[2] = {128, 3 * n_pad * 128};
  const cuuint32_t box[3] = {64, 128, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct GramArgs {
  int n_tiles;    // 128-row tiles of n_pad
  int n_pairs;    // upper tile pairs
  int n_parts;    // K parts
  int kb_total;   // K blocks of Pp
  int kb_per_part;
  int n_items;    // n_parts * n_pairs, part-major
  int64_t n_pad;
  double *Tpart;  // [n_parts][n_pad][n_pad]
  int *status;
};

__device__ __forceinline__ void pair_of(int p, int nt, int *ti, int *tj) {
  int i = 0, rem = p;
  while (rem >= nt - i) {
    rem -= nt - i;
    ++i;
  }
  *ti = i;
  *tj = i + rem;
}

__global__ void __launch_bounds__(GRAM_THREADS, 1)
    minsr_gram_kernel(const __grid_constant__ CUtensorMap mS, const GramArgs g) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ uint64_t full[GRAM_STAGES], empty[GRAM_STAGES], tfull[2], tempty[2];  // one pair per accumulator set
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const uint32_t raw = smem_addr(smem_dyn);
  unsigned char *base = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  constexpr uint32_t TILE = 16384u, STAGE = 6 * TILE;  // A terms 0..2, B terms 3..5
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < GRAM_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(&tfull[u], 1);
      mbar_init(&tempty[u], 8);
    }
    fence_mbar_init();
    abort_flag = 0;
    prefetch_tmap(&mS);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    for (uint32_t it = 0; it < GRAM_POLLS; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if (abort_flag) return false;
    }
    abort_flag = 1;
    atomicOr(g.status, STATUS_TIMEOUT);
    return false;
  };
  auto kb_range = [&](int item, int *kb0, int *kb1) {
    const int part = item / g.n_pairs;
    *kb0 = part * g.kb_per_part;
    *kb1 = min(g.kb_total, *kb0 + g.kb_per_part);
  };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      uint32_t it = 0;
      for (int item = blockIdx.x; item < g.n_items && !abort_flag; item += gridDim.x) {
        int ti, tj, kb0, kb1;
        pair_of(item % g.n_pairs, g.n_tiles, &ti, &tj);
        kb_range(item, &kb0, &kb1);
        const bool diag = ti == tj;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % GRAM_STAGES;
          if (!wait(&empty[s], ((it / GRAM_STAGES) & 1u) ^ 1u)) break;
          unsigned char *st = base + s * STAGE;
          mbar_expect_tx(&full[s], diag ? 3 * TILE : 6 * TILE);
          for (int t = 0; t < 3; ++t) {
            tma_load_3d(st + t * TILE, &mS, 0, (int32_t)(t * g.n_pad + ti * 128), kb, &full[s]);
            if (!diag) tma_load_3d(st + (3 + t) * TILE, &mS, 0, (int32_t)(t * g.n_pad + tj * 128), kb, &full[s]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      const uint32_t id = tc::idesc_bf16_f32(128, 128);
      uint32_t it = 0, d = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < g.n_items && ok && !abort_flag; item += gridDim.x) {
        int ti, tj, kb0, kb1;
        pair_of(item % g.n_pairs, g.n_tiles, &ti, &tj);
        kb_range(item, &kb0, &kb1);
        const bool diag = ti == tj;
        for (int c0 = kb0; c0 < kb1 && ok; c0 += GRAM_DRAIN, ++d) {
          // accumulator set u = d & 1, used for the (d >> 1)-th time: its previous drain must be done
          if (!wait(&tempty[d & 1u], ((d >> 1) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t acc_hi = tmem + (d & 1u) * 256u, acc_lo = acc_hi + 128u;
          const int c1 = min(kb1, c0 + GRAM_DRAIN);
          for (int kb = c0; kb < c1; ++kb, ++it) {
            const int s = it % GRAM_STAGES;
            if (!wait(&full[s], (it / GRAM_STAGES) & 1u)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            unsigned char *st = base + s * STAGE;
            unsigned char *sb = diag ? st : st + 3 * TILE;
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t first = (kb == c0 && kk == 0) ? 0u : 1u;
              auto A = [&](int t) { return tc::desc_sw128(smem_addr(st + t * TILE + kk * 32)); };
              auto B = [&](int t) { return tc::desc_sw128(smem_addr(sb + t * TILE + kk * 32)); };
              tc::mma_bf16(acc_hi, A(0), B(0), id, first);  // hi * hi
              tc::mma_bf16(acc_lo, A(0), B(1), id, first);  // hi * mid
              tc::mma_bf16(acc_lo, A(1), B(0), id, 1u);     // mid * hi
              tc::mma_bf16(acc_lo, A(0), B(2), id, 1u);     // hi * lo
              tc::mma_bf16(acc_lo, A(2), B(0), id, 1u);     // lo * hi
              tc::mma_bf16(acc_lo, A(1), B(1), id, 1u);     // mid * mid
            }
            tc::mma_commit(&empty[s]);
          }
          if (ok) tc::mma_commit(&tfull[d & 1u]);
        }
      }
    }
  } else {  // ---- drain warps 2..9: TMEM lane quarter q, column half h
    const int q = warp & 3, h = (warp - 2) >> 2;
    uint32_t d = 0;
    for (int item = blockIdx.x; item < g.n_items; item += gridDim.x) {
      int ti, tj, kb0, kb1;
      pair_of(item % g.n_pairs, g.n_tiles, &ti, &tj);
      kb_range(item, &kb0, &kb1);
      const int part = item / g.n_pairs;
      const int64_t r = (int64_t)ti * 128 + 32 * q + lane;
      double *row = g.Tpart + ((int64_t)part * g.n_pad + r) * g.n_pad + (int64_t)tj * 128 + 64 * h;
      // this thread's 64 FP64 partial sums (row r, columns 64h..64h+63) stay in registers for
      // the whole item and are stored once at its end
      double acc[64];
#pragma unroll
      for (int e = 0; e < 64; ++e) acc[e] = 0.0;
      bool stop = false;
      for (int c0 = kb0; c0 < kb1; c0 += GRAM_DRAIN, ++d) {
        if (!wait(&tfull[d & 1u], (d >> 1) & 1u)) {
          stop = true;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc_hi = tmem + (d & 1u) * 256u, acc_lo = acc_hi + 128u;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int col = 64 * h + 16 * cc;
          float vh[16], vl[16];
          tc::tmem_ld16(tc::tmem_lane_addr(acc_hi, 32 * q, col), vh);
          tc::tmem_ld16(tc::tmem_lane_addr(acc_lo, 32 * q, col), vl);
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[16 * cc + e] += (double)vh[e] + (double)vl[e];
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty[d & 1u])) : "memory");
      }
      if (stop) break;
#pragma unroll
      for (int e = 0; e < 64; e += 2) *reinterpret_cast<double2 *>(row + e) = make_double2(acc[e], acc[e + 1]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (abort_flag && tid == 0) {
    for (int s = 0; s < GRAM_STAGES; ++s) mbar_wait_bounded(&empty[s], 0, 1u << 16);
  }
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// T[x][y] = (1/n) sum_parts Tpart[min(x,y)][max(x,y)] + lam on the diagonal (x <= y lies in an
// upper tile pair or a diagonal tile, the pairs the Gram kernel computed); on the diagonal pass
// also the right-hand side w[x] = ebar_x = (eloc_x - E) / sqrt(n), E = stats[0].
__global__ void minsr_reduce_kernel(const double *__restrict__ Tpart, int n_parts, int64_t n, int64_t n_pad,
                                    double lam, double *T, double *T_out, const float *__restrict__ eloc,
                                    const double *__restrict__ stats, double *w) {
  const double inv_n = 1.0 / (double)n, E = stats[0], rs = 1.0 / sqrt((double)n);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = q / n, y = q % n;
    const int64_t src = x <= y ? x * n_pad + y : y * n_pad + x;  // upper element, mirrored: T exactly symmetric
    double s = 0.0;
    for (int p = 0; p < n_parts; ++p) s += Tpart[(int64_t)p * n_pad * n_pad + src];
    s *= inv_n;
    if (T_out) T_out[q] = s;
    T[q] = s + (x == y ? lam : 0.0);
    if (x == y) w[x] = ((double)eloc[x] - E) * rs;
  }
}

// ---- Cholesky (lower, in place in A [n x n] row-major), FP64 -------------------------------
// The forward substitution L z = w runs along with it: when block [k0, k0 + nb) is factored,
// the earlier panels have already subtracted their part from w over these rows, so the block
// solves its own triangle (chol_diag_kernel) and its panel subtracts L[i][block] z_block from
// w_i for every later row (chol_panel_kernel).  w holds z when the factorisation ends.
//
// Diagonal block [k0, k0 + nb) factored by one CTA in shared memory; then warp 0 solves
// L_d z = w over the block's rows (lane l holds rows l and l + 32).
__global__ void chol_diag_kernel(double *A, int64_t n, int64_t k0, int nb, int *status, double *w) {
  __shared__ double a[CHOL_NB][CHOL_NB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) a[q / nb][q % nb] = A[(k0 + q / nb) * n + k0 + q % nb];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        atomicOr(status, STATUS_RANGE);  // not positive definite in FP64
        d = 1e-300;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    const double inv = 1.0 / a[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] *= inv;
    __syncthreads();
    for (int q = threadIdx.x; q < (nb - j - 1) * (nb - j - 1); q += blockDim.x) {
      const int i = j + 1 + q / (nb - j - 1), k = j + 1 + q % (nb - j - 1);
      if (k <= i) a[i][k] -= a[i][j] * a[k][j];
    }
    __syncthreads();
  }
  __shared__ double rinv[CHOL_NB];  // 1 / L_jj, taken once per row before the sequential solve
  for (int j = threadIdx.x; j < nb; j += blockDim.x) rinv[j] = 1.0 / a[j][j];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    double b0 = l < nb ? w[k0 + l] : 0.0, b1 = l + 32 < nb ? w[k0 + l + 32] : 0.0;
    for (int j = 0; j < nb; ++j) {  // z_j = b_j / L_jj, then b_i -= L_ij z_j for the rows i > j
      const double zj = __shfl_sync(FULL_MASK, j < 32 ? b0 : b1, j & 31) * rinv[j];
      if (l == (j & 31)) (j < 32 ? b0 : b1) = zj;
      if (l > j && l < nb) b0 -= a[l][j] * zj;
      if (l + 32 > j && l + 32 < nb) b1 -= a[l + 32][j] * zj;
    }
    if (l < nb) w[k0 + l] = b0;
    if (l + 32 < nb) w[k0 + l + 32] = b1;
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int i = q / nb, k = q % nb;
    A[(k0 + i) * n + k0 + k] = k <= i ? a[i][k] : 0.0;
  }
}

// Panel rows i >= k0 + nb: L[i][k0 .. k0+nb) = A[i][..] L_d^-T (forward substitution per row),
// then w_i -= L[i][k0 .. k0+nb) z_block (z_block = w[k0 .. k0+nb) from chol_diag_kernel).
__global__ void chol_panel_kernel(double *A, int64_t n, int64_t k0, int nb, double *w) {
  __shared__ double l[CHOL_NB][CHOL_NB + 1];
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) l[q / nb][q % nb] = A[(k0 + q / nb) * n + k0 + q % nb];
  __syncthreads();
  for (int64_t i = k0 + nb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double *row = A + i * n + k0;
    double v[CHOL_NB];
    for (int j = 0; j < nb; ++j) {
      double s = row[j];
      for (int k = 0; k < j; ++k) s -= v[k] * l[j][k];
      v[j] = s / l[j][j];
    }
    double s = 0.0;
    for (int j = 0; j < nb; ++j) {
      row[j] = v[j];
      s += v[j] * w[k0 + j];
    }
    w[i] -= s;
  }
}

// Trailing update of the lower triangle: A[i][k] -= sum_j L[i][j] L[k][j] for i, k >= k1,
// tiles of 64 x 64 (4 x 4 per thread), the two panel slices staged 32 columns at a time.
__global__ void __launch_bounds__(256) chol_update_kernel(double *A, int64_t n, int64_t k0, int nb, int64_t k1) {
  __shared__ double li[64][33], lk[64][33];
  const int64_t m = n - k1;
  const int64_t tiles = (m + 63) / 64;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  for (int64_t t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
    const int64_t bi = t / tiles, bk = t % tiles;
    if (bk > bi) continue;  // lower tiles only (uniform per block)
    const int64_t i0 = k1 + bi * 64, kk0 = k1 + bk * 64;
    double acc[4][4] = {};
    for (int j0 = 0; j0 < nb; j0 += 32) {
      const int jn = min(32, nb - j0);
      __syncthreads();
      for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
        const int r = q / 32, j = q % 32;
        li[r][j] = (i0 + r < n && j < jn) ? A[(i0 + r) * n + k0 + j0 + j] : 0.0;
        lk[r][j] = (kk0 + r < n && j < jn) ? A[(kk0 + r) * n + k0 + j0 + j] : 0.0;
      }
      __syncthreads();
      for (int j = 0; j < jn; ++j) {
        double a[4], b[4];
        for (int u = 0; u < 4; ++u) {
          a[u] = li[ty + 16 * u][j];
          b[u] = lk[tx + 16 * u][j];
        }
        for (int u = 0; u < 4; ++u)
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
      }
    }
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) {
        const int64_t i = i0 + ty + 16 * u, k = kk0 + tx + 16 * v;
        if (i < n && k <= i) A[i * n + k] -= acc[u][v];
      }
  }
}

// Backward substitution L^T y = z over the block J = [j0, j0 + nb), the blocks taken from the
// last: every CTA solves the block's triangle L_JJ^T y_J = w_J from a shared-memory copy of
// L_JJ (warp 0; lane l holds rows l and l + 32), CTA 0 stores y_J, and the CTAs subtract
// sum_{j in J} L[j][i] y_j from w_i for the columns i < j0, 64 columns per CTA (rows of L,
// coalesced in i; the block's rows split over four quarters of the CTA).
__global__ void __launch_bounds__(256) minsr_back_kernel(const double *__restrict__ L, int64_t n, int64_t j0, int nb,
                                                         double *w, double *y) {
  __shared__ double ld[CHOL_NB][CHOL_NB + 1];
  __shared__ double yb[CHOL_NB], inv[CHOL_NB];
  __shared__ double part[4][64];
  const int tid = threadIdx.x;
  for (int q = tid; q < nb * nb; q += blockDim.x) ld[q / nb][q % nb] = L[(j0 + q / nb) * n + j0 + q % nb];
  for (int j = tid; j < nb; j += blockDim.x) inv[j] = 1.0 / L[(j0 + j) * n + j0 + j];
  __syncthreads();
  if (tid < 32) {
    const int l = tid;
    double b0 = l < nb ? w[j0 + l] : 0.0, b1 = l + 32 < nb ? w[j0 + l + 32] : 0.0;
    for (int j = nb - 1; j >= 0; --j) {  // y_j = b_j / L_jj, then b_i -= L_ji y_j for the rows i < j
      const double yj = __shfl_sync(FULL_MASK, j < 32 ? b0 : b1, j & 31) * inv[j];
      if (l == (j & 31)) (j < 32 ? b0 : b1) = yj;
      if (l < j) b0 -= ld[j][l] * yj;
      if (l + 32 < j) b1 -= ld[j][l + 32] * yj;
    }
    yb[l] = b0;
    yb[l + 32] = b1;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int q = tid; q < nb; q += blockDim.x) y[j0 + q] = yb[q];
  const int c = tid & 63, qtr = tid >> 6;
  const int64_t i = (int64_t)blockIdx.x * 64 + c;
  double s = 0.0;
  if (i < j0)
    for (int j = qtr; j < nb; j += 4) s += L[(j0 + j) * n + i] * yb[j];
  part[qtr][c] = s;
  __syncthreads();
  if (qtr == 0 && i < j0) w[i] -= (part[0][c] + part[1][c]) + (part[2][c] + part[3][c]);
}

// ysum = sum_x y_x (one CTA, fixed order).
__global__ void __launch_bounds__(1024) minsr_ysum_kernel(const double *__restrict__ y, int64_t n, double *ysum) {
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double s = 0.0;
  for (int64_t i = tid; i < n; i += blockDim.x) s += y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    *ysum = t;
  }
}

// dtheta_k = (sum_x O_xk y_x - mean_k sum_x y_x) / sqrt(n); the row sums as in
// minsr_colmean_kernel (FP32 within chunks, y rounded to FP32, FP64 across chunks).
__global__ void minsr_dtheta_kernel(const float *__restrict__ O, int64_t n, int64_t P, const double *__restrict__ mean_d,
                                    const double *__restrict__ y, const double *__restrict__ ysum, double *dtheta) {
  extern __shared__ float yf[];  // [n] y in FP32
  for (int64_t x = threadIdx.x; x < n; x += blockDim.x) yf[x] = (float)y[x];
  __syncthreads();
  const double rs = 1.0 / sqrt((double)n), ys = *ysum;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t x0 = 0; x0 < n; x0 += MINSR_CHUNK) {
      float c = 0.f;
      const int m = (int)(n - x0 < MINSR_CHUNK ? n - x0 : MINSR_CHUNK);
#pragma unroll 4
      for (int q = 0; q < m; ++q) c = fmaf(O[(x0 + q) * P + k], yf[x0 + q], c);
      s += (double)c;
    }
    dtheta[k] = (s - mean_d[k] * ys) * rs;
  }
}

struct Layout {
  int64_t n_pad, Pp;
  int n_tiles, n_pairs, n_parts, kb_total, kb_per_part;
  size_t off_mean_d, off_mean_f, off_S3, off_Tpart, off_T, off_z, off_y, off_ys, total;
};

Layout layout_for(const nqs_ctx *c, int64_t n) {
  Layout L;
  L.n_pad = (n + 127) / 128 * 128;
  L.Pp = (c->P + 63) / 64 * 64;
  L.n_tiles = (int)(L.n_pad / 128);
  L.n_pairs = L.n_tiles * (L.n_tiles + 1) / 2;
  L.kb_total = (int)(L.Pp / 64);
  // K parts: enough work items to keep every SM busy with little imbalance in the last round
  int best = 1;
  double best_eff = 0.0;
  for (int parts = 1; parts <= 16 && parts <= L.kb_total; ++parts) {
    const double items = (double)parts * L.n_pairs;
    const double rounds = std::ceil(items / c->num_sms);
    const double eff = items / (rounds * c->num_sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = parts;
    }
  }
  L.kb_per_part = (L.kb_total + best - 1) / best;
  L.n_parts = (L.kb_total + L.kb_per_part - 1) / L.kb_per_part;  // every part non-empty
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  size_t o = 0;
  L.off_mean_d = o;
  o = al(o + (size_t)c->P * 8);
  L.off_mean_f = o;
  o = al(o + (size_t)c->P * 4);
  L.off_S3 = o;
  o = al(o + (size_t)3 * L.n_pad * L.Pp * 2);
  L.off_Tpart = o;
  o = al(o + (size_t)L.n_parts * L.n_pad * L.n_pad * 8);
  L.off_T = o;
  o = al(o + (size_t)n * n * 8);
  L.off_z = o;
  o = al(o + (size_t)n * 8);
  L.off_y = o;
  o = al(o + (size_t)n * 8);
  L.off_ys = o;
  o = al(o + 8);
  L.total = o;
  return L;
}

unsigned grid_n(int64_t work, int per_block, int num_sms) {
  const int64_t b = (work + per_block - 1) / per_block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 32));
}

}  // namespace

size_t minsr_workspace(const nqs_ctx *c, int64_t n) { return layout_for(c, n).total; }

cudaError_t minsr(const nqs_ctx *c, const float *O, int64_t n, const float *eloc, const double *stats, double lam,
                  double *dtheta, double *T_out, void *ws, cudaStream_t s) {
  const Layout L = layout_for(c, n);
  char *w = static_cast<char *>(ws);
  double *mean_d = reinterpret_cast<double *>(w + L.off_mean_d);
  float *mean_f = reinterpret_cast<float *>(w + L.off_mean_f);
  __nv_bfloat16 *S3 = reinterpret_cast<__nv_bfloat16 *>(w + L.off_S3);
  double *Tpart = reinterpret_cast<double *>(w + L.off_Tpart);
  double *T = reinterpret_cast<double *>(w + L.off_T);
  double *z = reinterpret_cast<double *>(w + L.off_z);
  double *y = reinterpret_cast<double *>(w + L.off_y);
  double *ys = reinterpret_cast<double *>(w + L.off_ys);
  cudaError_t e;
  minsr_colmean_kernel<<<grid_n(c->P, 256, c->num_sms), 256, 0, s>>>(O, n, c->P, mean_d, mean_f);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  minsr_split_kernel<<<grid_n(L.n_pad * L.Pp / 2, 256, c->num_sms), 256, 0, s>>>(O, n, c->P, L.n_pad, L.Pp, mean_f,
                                                                                 S3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap mS;
  if (!make_tmap_kblocks(&mS, S3, (uint64_t)L.n_pad, (uint64_t)L.kb_total)) return cudaErrorInvalidValue;
  GramArgs g;
  g.n_tiles = L.n_tiles;
  g.n_pairs = L.n_pairs;
  g.n_parts = L.n_parts;
  g.kb_total = L.kb_total;
  g.kb_per_part = L.kb_per_part;
  g.n_items = L.n_parts * L.n_pairs;
  g.n_pad = L.n_pad;
  g.Tpart = Tpart;
  g.status = c->d_status;
  const size_t shm = 1024 + (size_t)GRAM_STAGES * 6 * 16384;
  if ((e = cudaFuncSetAttribute(minsr_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)) !=
      cudaSuccess)
    return e;
  minsr_gram_kernel<<<std::min(g.n_items, c->num_sms), GRAM_THREADS, shm, s>>>(mS, g);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  minsr_reduce_kernel<<<grid_n(n * n, 256, c->num_sms), 256, 0, s>>>(Tpart, L.n_parts, n, L.n_pad, lam, T, T_out,
                                                                    eloc, stats, z);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int64_t k0 = 0; k0 < n; k0 += CHOL_NB) {
    const int nb = (int)std::min<int64_t>(CHOL_NB, n - k0);
    chol_diag_kernel<<<1, 256, 0, s>>>(T, n, k0, nb, c->d_status, z);
    const int64_t k1 = k0 + nb;
    if (k1 < n) {
      chol_panel_kernel<<<grid_n(n - k1, 128, c->num_sms), 128, 0, s>>>(T, n, k0, nb, z);
      const int64_t tiles = (n - k1 + 63) / 64;
      chol_update_kernel<<<(unsigned)std::min<int64_t>(tiles * tiles, (int64_t)c->num_sms * 8), 256, 0, s>>>(
          T, n, k0, nb, k1);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int64_t j0 = (n - 1) / CHOL_NB * CHOL_NB; j0 >= 0; j0 -= CHOL_NB) {
    const int nb = (int)std::min<int64_t>(CHOL_NB, n - j0);
    minsr_back_kernel<<<(unsigned)std::max<int64_t>(1, (j0 + 63) / 64), 256, 0, s>>>(T, n, j0, nb, z, y);
  }
  minsr_ysum_kernel<<<1, 1024, 0, s>>>(y, n, ys);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  minsr_dtheta_kernel<<<grid_n(c->P, 256, c->num_sms), 256, (size_t)n * sizeof(float), s>>>(O, n, c->P, mean_d, y,
                                                                                            ys, dtheta);
  return cudaGetLastError();
}

}  // namespace nqs
