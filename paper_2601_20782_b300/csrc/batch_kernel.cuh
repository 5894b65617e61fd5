// Persistent batched sweep kernel (work list of (instance, block of chains)); the host
// side and the work-list construction are in batch.cu, the instantiations in batch_k*.cu.
#pragma once
#include <cuda_fp16.h>

#include "internal.h"
#include "rbm_core.cuh"
#include "tc.cuh"

namespace nqs {
namespace batchk {
using namespace rbmk;

struct BatchInst {
  SweepParams p;  // n_sweeps / burn_in / sweep_offset are set per launch from BatchParams
  int E;          // hidden units per lane (M_pad / 32)
  int staged;     // the table fits the CTA's shared-memory stage
  uint32_t table_bytes;
};

struct BatchItem {
  int inst;
  int n;  // chains in this item (<= warps per CTA)
  int64_t c0;
};

struct BatchParams {
  const BatchInst *inst;
  const BatchItem *items;
  unsigned *next;  // work counter, zeroed before each launch
  int n_items;
  int n_sweeps, burn_in;
  uint32_t sweep_offset;
  uint32_t table_cap;  // bytes of the table stage; (a_i, K_i) pairs follow it
};

template <typename TT>
__device__ __forceinline__ void sweep_dispatch(int E, const SweepParams &p, const TT *R, const float2 *saK,
                                               int64_t base, int64_t limit) {
  switch (E) {
#define NQS_BCASE(EE)                                     \
  case EE:                                                \
    sweep_chain<32, EE, false, TT>(p, R, saK, base, limit); \
    break;
    NQS_BCASE(1) NQS_BCASE(2) NQS_BCASE(3) NQS_BCASE(4) NQS_BCASE(5) NQS_BCASE(6) NQS_BCASE(7) NQS_BCASE(8)
    NQS_BCASE(9) NQS_BCASE(10) NQS_BCASE(11) NQS_BCASE(12) NQS_BCASE(13) NQS_BCASE(14) NQS_BCASE(16)
    NQS_BCASE(18) NQS_BCASE(20) NQS_BCASE(24) NQS_BCASE(28) NQS_BCASE(32)
#undef NQS_BCASE
    default:
      break;
  }
}

// MAXT > 0 caps the CTA at MAXT threads, which bounds the registers per thread at
// 65536 / MAXT (the wide cases may then spill); MAXT = 0 leaves the registers to the
// widest case (up to 255, so at most 256 threads).  The autotuner chooses.
template <typename TT, int MAXT>
__global__ void __launch_bounds__(MAXT > 0 ? MAXT : 256, 1) rbm_batch_sweep_kernel(const BatchParams bp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  float2 *saK = reinterpret_cast<float2 *>(smem_raw + bp.table_cap);
  const TT *sR = reinterpret_cast<const TT *>(smem_raw);
  uint32_t phase = 0;
  int staged = -1;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(bp.next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= bp.n_items) break;
    const BatchItem item = bp.items[it];
    const BatchInst &in = bp.inst[item.inst];
    SweepParams p = in.p;
    p.n_sweeps = bp.n_sweeps;
    p.burn_in = bp.burn_in;
    p.sweep_offset = bp.sweep_offset;
    const int in_staged = in.staged;
    if (item.inst != staged) {
      bool ok = true;
      if (in_staged) {
        const uint32_t bytes = in.table_bytes;
        if (threadIdx.x == 0) {
          tc::fence_proxy_async_smem();  // earlier generic reads of the stage before the async writes
          mbar_expect_tx(&bar, bytes);
          for (uint32_t off = 0; off < bytes; off += BULK_CHUNK)
            bulk_g2s(smem_raw + off, static_cast<const char *>(p.R) + off, min(BULK_CHUNK, bytes - off), &bar);
        }
        ok = mbar_wait_bounded(&bar, phase, WAIT_POLLS);
        if (!ok) {
          if (threadIdx.x == 0) atomicOr(p.status, STATUS_TIMEOUT);
          mbar_wait_bounded(&bar, phase, WAIT_POLLS);  // let copies in flight land before leaving
        }
        phase ^= 1u;
      }
      for (int i = threadIdx.x; i < p.N; i += blockDim.x) saK[i] = p.aK[i];
      if (!__syncthreads_and(ok)) return;
      staged = item.inst;
    }
    const TT *R = in_staged ? sR : static_cast<const TT *>(p.R);
    if (warp < item.n) sweep_dispatch<TT>(in.E, p, R, saK, item.c0 + warp, item.c0 + item.n);
    __syncthreads();  // every warp is done with the stage and s_item before the next item
  }
}

// instantiations (batch_k*.cu)
const void *batch_kernel_f32();
const void *batch_kernel_f16_capped();
const void *batch_kernel_f16_wide();
constexpr int BATCH_CAPPED_THREADS = 512;  // registers <= 128

}  // namespace batchk
}  // namespace nqs
