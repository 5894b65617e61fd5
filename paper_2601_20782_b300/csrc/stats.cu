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

__global__ void stats_final_kernel(const double *partial, int nblocks, int64_t n, int64_t C, int64_t proposals,
                                   int has_acc, double *out) {
  if (threadIdx.x != 0) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 5; ++q) v[q] += partial[b * 5 + q];
  const double mean = v[0] / (double)n;
  const double var = fmax(v[1] / (double)n - mean * mean, 0.0);
  double err;
  if (C >= 2) {
    const double mm = v[2] / (double)C;
    const double vc = fmax((v[3] - (double)C * mm * mm) / (double)(C - 1), 0.0);
    err = sqrt(vc / (double)C);
  } else {
    err = sqrt(var / (double)n);
  }
  out[0] = mean;
  out[1] = var;
  out[2] = err;
  out[3] = has_acc ? v[4] / ((double)C * (double)proposals) : 0.0;
  out[4] = (double)n;
}

}  // namespace

cudaError_t energy_stats(const nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains, const int64_t *n_acc,
                         int64_t proposals_per_chain, double *out, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>({(n_chains + ST_THREADS - 1) / ST_THREADS, (int64_t)c->num_sms * 2, STATS_MAX_BLOCKS}));
  stats_partial_kernel<<<blocks, ST_THREADS, 0, s>>>(eloc, n, n_chains, n_acc, c->d_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stats_final_kernel<<<1, 32, 0, s>>>(c->d_scratch, blocks, n, n_chains, proposals_per_chain, n_acc != nullptr, out);
  return cudaGetLastError();
}

}  // namespace nqs
