// FP64 energy statistics (Sec. 2, Eq. loss): mean, variance, chain-blocked error
// of the mean and acceptance rate.  Two deterministic passes: per-block partial
// sums into the context's scratch, then one block adds them in a fixed order.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nqs {
namespace {

constexpr int ST_THREADS = 256;

// Thread per chain c (sweep-major rows k * C + c): sum and sum of squares of its
// K samples and of its chain mean.  Partial per block: [sum, sumsq, sum m_c, sum m_c^2, acc].
__global__ void __launch_bounds__(ST_THREADS) stats_partial_kernel(const float *__restrict__ eloc, int64_t n,
                                                                    int64_t C, const int64_t *__restrict__ n_acc,
                                                                    double *partial) {
  const int64_t K = n / C;
  double s = 0.0, s2 = 0.0, m = 0.0, m2 = 0.0, acc = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)ST_THREADS + threadIdx.x; c < C; c += (int64_t)gridDim.x * ST_THREADS) {
    double cs = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      const double v = eloc[k * C + c];
      cs += v;
      s2 += v * v;
    }
    s += cs;
    const double mc = cs / (double)K;
    m += mc;
    m2 += mc * mc;
    if (n_acc) acc += (double)n_acc[c];
  }
  __shared__ double red[5][ST_THREADS / 32];
  double v[5] = {s, s2, m, m2, acc};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const double w = group_allsum<32>(v[q]);
    if (lane == 0) red[q][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double t = 0.0;
    for (int w = 0; w < ST_THREADS / 32; ++w) t += red[threadIdx.x][w];
    partial[blockIdx.x * 5 + threadIdx.x] = t;
  }
}

// The statistics from the additive moments m = [n, sum eps, sum eps^2, C, sum_c m_c,
// sum_c m_c^2, sum n_acc, C * proposals per chain] (m_c: chain means).  Sums of moments over
// disjoint sets of chains (ranks) give the statistics of the pooled chains.
__device__ void finalize_moments(const double *m, double *out) {
  const double n = m[0], C = m[3];
  const double mean = m[1] / n;
  const double var = fmax(m[2] / n - mean * mean, 0.0);
  double err;
  if (C >= 2.0) {
    const double mm = m[4] / C;
    const double vc = fmax((m[5] - C * mm * mm) / (C - 1.0), 0.0);
    err = sqrt(vc / C);
  } else {
    err = sqrt(var / n);
  }
  out[0] = mean;
  out[1] = var;
  out[2] = err;
  out[3] = m[7] > 0.0 ? m[6] / m[7] : 0.0;
  out[4] = n;
}

// Adds the blocks' partials in a fixed order into the moments; writes them (moments != nullptr)
// or the statistics.
__global__ void stats_final_kernel(const double *partial, int nblocks, int64_t n, int64_t C, int64_t proposals,
                                   int has_acc, double *out, double *moments) {
  if (threadIdx.x != 0) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 5; ++q) v[q] += partial[b * 5 + q];
  const double m[8] = {(double)n, v[0], v[1], (double)C, v[2], v[3], has_acc ? v[4] : 0.0,
                       has_acc ? (double)C * (double)proposals : 0.0};
  if (moments) {
    for (int q = 0; q < 8; ++q) moments[q] = m[q];
  } else {
    finalize_moments(m, out);
  }
}

__global__ void stats_finalize_kernel(const double *moments, double *out) {
  if (threadIdx.x == 0) finalize_moments(moments, out);
}

}  // namespace

cudaError_t energy_stats(const nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains, const int64_t *n_acc,
                         int64_t proposals_per_chain, double *out, cudaStream_t s, double *moments) {
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>({(n_chains + ST_THREADS - 1) / ST_THREADS, (int64_t)c->num_sms * 2, STATS_MAX_BLOCKS}));
  stats_partial_kernel<<<blocks, ST_THREADS, 0, s>>>(eloc, n, n_chains, n_acc, c->d_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stats_final_kernel<<<1, 32, 0, s>>>(c->d_scratch, blocks, n, n_chains, proposals_per_chain, n_acc != nullptr, out,
                                      moments);
  return cudaGetLastError();
}

cudaError_t stats_finalize(const double *moments, double *out, cudaStream_t s) {
  stats_finalize_kernel<<<1, 32, 0, s>>>(moments, out);
  return cudaGetLastError();
}

}  // namespace nqs
