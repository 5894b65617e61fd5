// Batched uneven instances: many independent TFIM problems (their own lattice, N, M, h,
// chain count and Philox key) sampled by ONE persistent launch, then the step
// sweep -> local energy -> statistics -> O rows replayed as a CUDA graph.
//
// Work list.  Every instance's chains are cut into items of `warps` chains (one chain per
// warp, L = 32 lanes); items are ordered by cost (chains x N x M_pad, the proposals' hidden-
// unit work) from the largest down and handed out through an atomic counter, so that CTAs
// that finish early take the remaining small items (longest-processing-time-first with
// dynamic assignment).  A CTA stages the item's table in shared memory when it fits
// (1D bulk copies on one mbarrier whose phase it tracks), keeps it while consecutive items
// belong to the same instance, and otherwise reads it through L2.  Each chain runs the same
// device function as nqs_sweep (sweep_chain), so a batched chain is bit-identical to the
// same chain sampled alone.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <numeric>

#include "batch_kernel.cuh"

namespace nqs {
using batchk::BatchInst;
using batchk::BatchItem;
using batchk::BatchParams;
}  // namespace nqs

// ======================================================================================
struct nqs_batch {
  std::vector<nqs_batch_item> items;
  int n_sweeps = 0, burn_in = 0;
  nqs_dtype dtype = NQS_F32;
  int device = 0, num_sms = 0, smem_optin = 0;
  int warps = 0;       // warps (chains) per CTA
  int variant = 0;     // kernel variant (kernel_for)
  int max_warps = 0;   // register limit of the chosen variant
  int max_warps_v[3] = {0, 0, 0};
  int n_staged = 0;
  uint32_t table_cap = 0, ak_cap = 0;
  std::vector<nqs::BatchInst> inst_h;
  nqs::BatchInst *d_inst = nullptr;
  nqs::BatchItem *d_items = nullptr;
  int n_items = 0;
  unsigned *d_next = nullptr;
  std::vector<float> tune_ms;  // autotuner: time of one sweep per candidate (variant, width)
  std::vector<int> tune_warps, tune_variant;
  // step graph: the capture stream plus BRANCHES streams on which the per-instance work forks
  static constexpr int BRANCHES = 3;
  cudaStream_t cap = nullptr;
  cudaStream_t branch[BRANCHES] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[BRANCHES] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t sweep_node = nullptr;
  nqs::BatchParams graph_params{};
  std::string err;
};

namespace {

nqs_status bfail(nqs_batch *b, nqs_status st, const std::string &m) {
  if (b) b->err = m;
  return st;
}
nqs_status bcuda(nqs_batch *b, cudaError_t e, const char *where) {
  if (b) b->err = std::string(where) + ": " + cudaGetErrorString(e);
  return NQS_ECUDA;
}

// variant 0: FP32; FP16 with registers capped at 128 (1) or those of the widest case (2)
const void *kernel_for(int variant) {
  switch (variant) {
    case 1:
      return nqs::batchk::batch_kernel_f16_capped();
    case 2:
      return nqs::batchk::batch_kernel_f16_wide();
    default:
      return nqs::batchk::batch_kernel_f32();
  }
}

// Work items for `warps` chains per CTA, largest cost first.
cudaError_t build_items(nqs_batch *b, int warps) {
  std::vector<nqs::BatchItem> it;
  std::vector<double> cost;
  for (int k = 0; k < (int)b->items.size(); ++k) {
    const nqs_ctx *c = b->items[k].ctx;
    for (int64_t c0 = 0; c0 < b->items[k].n_chains; c0 += warps) {
      const int n = (int)std::min<int64_t>(warps, b->items[k].n_chains - c0);
      it.push_back({k, n, c0});
      cost.push_back((double)n * c->N * c->M_pad);
    }
  }
  std::vector<size_t> ord(it.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t z) { return cost[a] > cost[z]; });
  std::vector<nqs::BatchItem> sorted(it.size());
  for (size_t q = 0; q < ord.size(); ++q) sorted[q] = it[ord[q]];
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  b->n_items = (int)sorted.size();
  cudaError_t e = cudaMalloc(&b->d_items, std::max<size_t>(1, sorted.size()) * sizeof(nqs::BatchItem));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(b->d_items, sorted.data(), sorted.size() * sizeof(nqs::BatchItem), cudaMemcpyHostToDevice);
}

nqs::BatchParams params_for(const nqs_batch *b, uint32_t sweep_offset, int n_sweeps, int burn_in) {
  nqs::BatchParams p;
  p.inst = b->d_inst;
  p.items = b->d_items;
  p.next = b->d_next;
  p.n_items = b->n_items;
  p.n_sweeps = n_sweeps;
  p.burn_in = burn_in;
  p.sweep_offset = sweep_offset;
  p.table_cap = b->table_cap;
  return p;
}

cudaError_t launch_sweep(const nqs_batch *b, const nqs::BatchParams &p, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const size_t shm = (size_t)b->table_cap + b->ak_cap;
  if ((e = cudaFuncSetAttribute(kernel_for(b->variant), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)) !=
      cudaSuccess)
    return e;
  void *args[] = {const_cast<nqs::BatchParams *>(&p)};
  return cudaLaunchKernel(kernel_for(b->variant), dim3((unsigned)b->num_sms), dim3((unsigned)b->warps * 32), args, shm,
                          s);
}

// The per-instance descriptors with the given outputs (the autotuner passes none).
cudaError_t upload_instances(nqs_batch *b, bool outputs, uint32_t *const *state_override) {
  for (size_t k = 0; k < b->items.size(); ++k) {
    const nqs_batch_item &it = b->items[k];
    nqs::BatchInst &in = b->inst_h[k];
    in.p.state = state_override ? state_override[k] : it.state;
    in.p.samples = outputs ? it.samples : nullptr;
    in.p.logpsi = outputs ? it.logpsi : nullptr;
    in.p.n_acc = outputs ? it.n_accepted : nullptr;
    in.p.acc_bits = outputs ? it.accept_bits : nullptr;
  }
  return cudaMemcpy(b->d_inst, b->inst_h.data(), b->inst_h.size() * sizeof(nqs::BatchInst), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

nqs_status nqs_batch_create(nqs_batch **out, const nqs_batch_item *items, int32_t n_items, int32_t n_sweeps,
                            int32_t burn_in, int32_t warps_per_cta, nqs_stream stream) {
  if (!out || !items || n_items < 1) return NQS_EINVAL;
  *out = nullptr;
  if (n_sweeps < 1 || burn_in < 0 || burn_in > n_sweeps) return NQS_EINVAL;
  auto *b = new nqs_batch;
  b->items.assign(items, items + n_items);
  b->n_sweeps = n_sweeps;
  b->burn_in = burn_in;
  const nqs_ctx *c0 = items[0].ctx;
  if (!c0) {
    delete b;
    return NQS_EINVAL;
  }
  b->dtype = c0->dtype;
  if (b->dtype != NQS_F32 && b->dtype != NQS_F16) {
    delete b;
    return NQS_EUNSUPPORTED;
  }
  uint32_t max_n = 0;
  for (int k = 0; k < n_items; ++k) {
    const nqs_batch_item &it = items[k];
    const nqs_ctx *c = it.ctx;
    if (!c || c->model_kind != NQS_RBM || c->ham_kind != NQS_TFIM || c->dtype != b->dtype || !c->params_set ||
        it.n_chains < 1 || it.n_chains > (int64_t)UINT32_MAX || !it.state || c->device != c0->device) {
      delete b;
      return NQS_EINVAL;
    }
    max_n = std::max<uint32_t>(max_n, (uint32_t)c->N);
  }
  b->device = c0->device;
  b->num_sms = c0->num_sms;
  b->smem_optin = c0->smem_optin;
  b->ak_cap = (max_n * (uint32_t)sizeof(float2) + 15u) & ~15u;
  const size_t tsz = b->dtype == NQS_F16 ? 2 : 4;
  // stage every table that fits next to the (a, K) pairs and the static shared memory
  const uint32_t budget = (uint32_t)std::max(0, b->smem_optin - (int)b->ak_cap - 512) & ~127u;
  b->inst_h.resize(n_items);
  for (int k = 0; k < n_items; ++k) {
    const nqs_ctx *c = items[k].ctx;
    nqs::BatchInst &in = b->inst_h[k];
    std::memset(&in, 0, sizeof(in));
    in.table_bytes = (uint32_t)((size_t)c->N * c->M_pad * tsz);
    in.staged = in.table_bytes <= budget;
    if (in.staged) {
      b->table_cap = std::max(b->table_cap, in.table_bytes);
      ++b->n_staged;
    }
    in.E = c->M_pad / 32;
    in.p.R = c->d_R;
    in.p.aK = c->d_aK;
    in.p.Wt = c->d_Wt;
    in.p.b = c->d_b;
    in.p.delta = nullptr;
    in.p.status = c->d_status;
    in.p.C = items[k].n_chains;
    in.p.N = c->N;
    in.p.W = c->W;
    in.p.M_pad = c->M_pad;
    in.p.refresh = c->refresh;
    in.p.renorm = c->renorm;
    in.p.k0 = (uint32_t)items[k].seed;
    in.p.k1 = (uint32_t)(items[k].seed >> 32);
  }
  b->table_cap = (b->table_cap + 127u) & ~127u;
  const int shm = (int)(b->table_cap + b->ak_cap);
  if (cudaSetDevice(b->device) != cudaSuccess || cudaMalloc(&b->d_next, 16) != cudaSuccess ||
      cudaMalloc(&b->d_inst, n_items * sizeof(nqs::BatchInst)) != cudaSuccess) {
    nqs_batch_destroy(b);
    return NQS_ECUDA;
  }
  const std::vector<int> variants = b->dtype == NQS_F16 ? std::vector<int>{1, 2} : std::vector<int>{0};
  for (int v : variants) {  // CTA width limit of each variant from its register use
    cudaFuncAttributes fa;
    if (cudaFuncSetAttribute(kernel_for(v), cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel_for(v)) != cudaSuccess) {
      nqs_batch_destroy(b);
      return NQS_ECUDA;
    }
    const int regs = (std::max(fa.numRegs, 16) + 7) / 8 * 8;
    b->max_warps_v[v] = std::max(1, std::min(fa.maxThreadsPerBlock / 32, 65536 / (regs * 32)));
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (warps_per_cta > 0) {
    b->variant = variants[0];
    b->warps = std::min(warps_per_cta, b->max_warps_v[b->variant]);
  } else {
    // autotuner: one sweep of every instance per candidate (kernel variant, CTA width), on
    // scratch copies of the chains (no outputs); the fastest candidate is kept
    std::vector<uint32_t *> scratch(n_items, nullptr);
    bool okk = true;
    for (int k = 0; k < n_items && okk; ++k) {
      const size_t bytes = (size_t)items[k].n_chains * items[k].ctx->W * 4;
      okk = cudaMalloc(&scratch[k], bytes) == cudaSuccess &&
            cudaMemcpyAsync(scratch[k], items[k].state, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    okk = okk && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
          upload_instances(b, false, scratch.data()) == cudaSuccess;
    float best = 1e30f;
    int best_w = 0, best_v = variants[0];
    for (int v : variants) {
      for (int w : {4, 6, 8, 12, 16, 24}) {
        if (!okk || w > b->max_warps_v[v]) continue;
        b->variant = v;
        b->warps = w;
        if (build_items(b, w) != cudaSuccess) {
          okk = false;
          break;
        }
        const nqs::BatchParams p = params_for(b, 0x7FFF0000u, 1, 1);
        float ms = 0.f;
        okk = launch_sweep(b, p, s) == cudaSuccess &&  // warm-up (first touch of the tables)
              cudaEventRecord(e0, s) == cudaSuccess && launch_sweep(b, p, s) == cudaSuccess &&
              cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
              cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (!okk) break;
        b->tune_variant.push_back(v);
        b->tune_warps.push_back(w);
        b->tune_ms.push_back(ms);
        if (ms < best) {
          best = ms;
          best_w = w;
          best_v = v;
        }
      }
    }
    cudaStreamSynchronize(s);
    for (auto p : scratch)
      if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!okk || best_w == 0) {
      nqs_batch_destroy(b);
      return NQS_ECUDA;
    }
    b->variant = best_v;
    b->warps = best_w;
  }
  b->max_warps = b->max_warps_v[b->variant];
  if (build_items(b, b->warps) != cudaSuccess || upload_instances(b, true, nullptr) != cudaSuccess) {
    nqs_batch_destroy(b);
    return NQS_ECUDA;
  }
  *out = b;
  return NQS_OK;
}

nqs_status nqs_batch_sweep(nqs_batch *b, uint32_t sweep_offset, nqs_stream stream) {
  if (!b) return NQS_EINVAL;
  if ((uint64_t)sweep_offset + (uint64_t)b->n_sweeps > (1ull << 32))
    return bfail(b, NQS_EINVAL, "sweep counter overflow");
  const nqs::BatchParams p = params_for(b, sweep_offset, b->n_sweeps, b->burn_in);
  cudaError_t e = launch_sweep(b, p, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : bcuda(b, e, "nqs_batch_sweep");
}

// The step graph: sweep (one launch) -> per instance local energies, statistics, O rows.  The
// instances' chains of kernels are independent: they fork over the capture stream and the
// branch streams (instance k on lane k mod (BRANCHES + 1), each instance's kernels in order),
// so that one instance's kernels fill the SMs another's tail leaves idle; the lanes join
// before the graph ends.
static cudaError_t capture_step(nqs_batch *b) {
  cudaError_t e;
  if (!b->cap && (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  for (int j = 0; j < nqs_batch::BRANCHES; ++j)
    if (!b->branch[j] && ((e = cudaStreamCreateWithFlags(&b->branch[j], cudaStreamNonBlocking)) != cudaSuccess ||
                          (e = cudaEventCreateWithFlags(&b->join_ev[j], cudaEventDisableTiming)) != cudaSuccess))
      return e;
  if (!b->fork_ev && (e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  b->graph_params = params_for(b, 0, b->n_sweeps, b->burn_in);
  cudaError_t le = launch_sweep(b, b->graph_params, b->cap);
  if (le == cudaSuccess) le = cudaEventRecord(b->fork_ev, b->cap);
  for (int j = 0; j < nqs_batch::BRANCHES && le == cudaSuccess; ++j) le = cudaStreamWaitEvent(b->branch[j], b->fork_ev, 0);
  const int64_t K = b->n_sweeps - b->burn_in;
  for (size_t k = 0; k < b->items.size() && le == cudaSuccess; ++k) {
    const nqs_batch_item &it = b->items[k];
    const nqs_ctx *c = it.ctx;
    const int64_t S = K * it.n_chains;
    const int lane = (int)(k % (nqs_batch::BRANCHES + 1));
    cudaStream_t st = lane == 0 ? b->cap : b->branch[lane - 1];
    if (it.eloc && it.samples && S > 0) le = nqs::rbm_local_energy(c, it.samples, S, it.eloc, st);
    if (le == cudaSuccess && it.stats && it.eloc && it.samples && S > 0)
      le = nqs::energy_stats(c, it.eloc, S, it.n_chains, it.n_accepted, (int64_t)b->n_sweeps * c->N, it.stats, st);
    if (le == cudaSuccess && it.O && it.samples && K > 0)
      le = nqs::rbm_logpsi_grad(c, it.samples + (size_t)(K - 1) * it.n_chains * c->W, it.n_chains, it.O, nullptr,
                                nullptr, nullptr, nullptr, st);
  }
  for (int j = 0; j < nqs_batch::BRANCHES; ++j) {  // join every lane, also after an error, so the capture can end
    cudaError_t je = cudaEventRecord(b->join_ev[j], b->branch[j]);
    if (je == cudaSuccess) je = cudaStreamWaitEvent(b->cap, b->join_ev[j], 0);
    if (le == cudaSuccess) le = je;
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  b->graph = g;
  size_t n = 0;
  if ((e = cudaGraphGetNodes(g, nullptr, &n)) != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if ((e = cudaGraphGetNodes(g, nodes.data(), &n)) != cudaSuccess) return e;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == kernel_for(b->variant)) b->sweep_node = nd;
  }
  if (!b->sweep_node) return cudaErrorInvalidValue;
  return cudaGraphInstantiate(&b->exec, g, 0);
}

nqs_status nqs_batch_step(nqs_batch *b, uint32_t sweep_offset, nqs_stream stream) {
  if (!b) return NQS_EINVAL;
  if ((uint64_t)sweep_offset + (uint64_t)b->n_sweeps > (1ull << 32))
    return bfail(b, NQS_EINVAL, "sweep counter overflow");
  cudaError_t e;
  if (!b->exec && (e = capture_step(b)) != cudaSuccess) return bcuda(b, e, "nqs_batch_step (capture)");
  if (b->graph_params.sweep_offset != sweep_offset) {
    b->graph_params.sweep_offset = sweep_offset;
    cudaKernelNodeParams kp;
    if ((e = cudaGraphKernelNodeGetParams(b->sweep_node, &kp)) != cudaSuccess) return bcuda(b, e, "nqs_batch_step");
    void *args[] = {&b->graph_params};
    kp.kernelParams = args;
    if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->sweep_node, &kp)) != cudaSuccess)
      return bcuda(b, e, "nqs_batch_step");
  }
  e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : bcuda(b, e, "nqs_batch_step");
}

nqs_status nqs_batch_info(const nqs_batch *b, nqs_batch_info_t *info) {
  if (!b || !info) return NQS_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->warps_per_cta = b->warps;
  info->max_warps_per_cta = b->max_warps;
  info->ctas = b->num_sms;
  info->n_work_items = b->n_items;
  info->n_staged = b->n_staged;
  info->stage_bytes = (int64_t)b->table_cap + b->ak_cap;
  info->variant = b->variant;
  info->n_tuned = (int32_t)std::min<size_t>(b->tune_warps.size(), 16);
  for (int q = 0; q < info->n_tuned; ++q) {
    info->tuned_variant[q] = b->tune_variant[q];
    info->tuned_warps[q] = b->tune_warps[q];
    info->tuned_ms[q] = b->tune_ms[q];
  }
  return NQS_OK;
}

const char *nqs_batch_last_error(const nqs_batch *b) { return b ? b->err.c_str() : "null batch"; }

void nqs_batch_destroy(nqs_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int j = 0; j < nqs_batch::BRANCHES; ++j) {
    if (b->branch[j]) cudaStreamDestroy(b->branch[j]);
    if (b->join_ev[j]) cudaEventDestroy(b->join_ev[j]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_next) cudaFree(b->d_next);
  delete b;
}

}  // extern "C"
