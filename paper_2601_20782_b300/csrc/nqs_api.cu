// C ABI of include/nqs.h: argument validation, context lifetime, dispatch.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

thread_local std::string g_create_error;

nqs_status fail(nqs_ctx *c, nqs_status st, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return st;
}

nqs_status cuda_fail(nqs_ctx *c, cudaError_t e, const char *where) {
  return fail(c, NQS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t dev_alloc(T **p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_all(nqs_ctx *c) {
  void *ptrs[] = {c->d_bounds, c->d_status, c->d_scratch, c->d_bonds, c->d_bondJ, c->d_a, c->d_b,
                  c->d_Wt,     c->d_R,       c->d_aK,    c->d_Wm,    c->d_bm};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->dtype != NQS_F32) {
    void *p32[] = {c->d_a32, c->d_b32, c->d_Wt32, c->d_R32, c->d_aK32};
    for (void *p : p32)
      if (p) cudaFree(p);
  }
}

// Bond lists: nearest neighbours (x+1, y) and (x, y+1); J2 bonds (x+1, y+1) and
// (x+1, y-1) in 2D, (x+2) in 1D.  Each bond listed once (Lx, Ly >= 3).
void build_bonds(const nqs_ctx *c, std::vector<int2> &b, std::vector<float> &J) {
  const int Lx = c->Lx, Ly = c->Ly;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const int i = x + Lx * y;
      b.push_back(make_int2(i, (x + 1) % Lx + Lx * y));
      J.push_back((float)c->J1);
      if (Ly > 1) {
        b.push_back(make_int2(i, x + Lx * ((y + 1) % Ly)));
        J.push_back((float)c->J1);
      }
    }
  if (c->ham_kind == NQS_HEISENBERG && c->J2 != 0.0) {
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        const int i = x + Lx * y;
        if (Ly == 1) {
          b.push_back(make_int2(i, (x + 2) % Lx));
          J.push_back((float)c->J2);
        } else {
          b.push_back(make_int2(i, (x + 1) % Lx + Lx * ((y + 1) % Ly)));
          J.push_back((float)c->J2);
          b.push_back(make_int2(i, (x + 1) % Lx + Lx * ((y - 1 + Ly) % Ly)));
          J.push_back((float)c->J2);
        }
      }
  }
}

bool bad_ptr(const void *p) { return p == nullptr; }

}  // namespace

extern "C" {

const char *nqs_last_error(const nqs_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }
int32_t nqs_n_sites(const nqs_ctx *ctx) { return ctx ? ctx->N : 0; }
int32_t nqs_words_per_config(const nqs_ctx *ctx) { return ctx ? ctx->W : 0; }
int64_t nqs_n_params(const nqs_ctx *ctx) { return ctx ? ctx->P : 0; }
int32_t nqs_n_bonds(const nqs_ctx *ctx) { return ctx ? ctx->n_bonds : 0; }

nqs_status nqs_create(nqs_ctx **out, const nqs_model_desc *model, const nqs_ham_desc *ham, nqs_dtype dtype) {
  if (!out || !model || !ham) return fail(nullptr, NQS_EINVAL, "nqs_create: null argument");
  *out = nullptr;
  if (ham->kind != NQS_TFIM && ham->kind != NQS_HEISENBERG) return fail(nullptr, NQS_EINVAL, "unknown Hamiltonian kind");
  if (ham->Lx < 3 || !(ham->Ly == 1 || ham->Ly >= 3))
    return fail(nullptr, NQS_EINVAL, "periodic lattice needs Lx >= 3 and Ly == 1 or Ly >= 3");
  if (model->kind != NQS_RBM && model->kind != NQS_DENSE && model->kind != NQS_RESCNN)
    return fail(nullptr, NQS_EINVAL, "unknown model kind");
  if ((int)dtype < 0 || (int)dtype > 3) return fail(nullptr, NQS_EINVAL, "unknown dtype");
  const int64_t N64 = (int64_t)ham->Lx * ham->Ly;
  if (N64 > 1024) return fail(nullptr, NQS_EINVAL, "at most 1024 sites");

  nqs_ctx *c = new (std::nothrow) nqs_ctx();
  if (!c) return fail(nullptr, NQS_ENOMEM, "host allocation failed");
  c->model_kind = model->kind;
  c->ham_kind = ham->kind;
  c->dtype = dtype;
  c->Lx = ham->Lx;
  c->Ly = ham->Ly;
  c->N = (int)N64;
  c->W = (c->N + 31) / 32;
  c->J1 = ham->J1;
  c->J2 = ham->J2;
  c->h = ham->h;
  c->marshall = ham->marshall;
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) {
    delete c;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);

  std::string why;
  if (model->kind == NQS_RBM) {
    if (model->n_hidden < 1 || model->n_hidden > 1024) {
      delete c;
      return fail(nullptr, NQS_EINVAL, "RBM needs 1 <= n_hidden <= 1024");
    }
    c->M = model->n_hidden;
    // padding: 32 * E with E one of the instantiated widths
    static const int Es[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 16, 18, 20, 24, 28, 32};
    int need = (c->M + nqs::MPAD_ALIGN - 1) / nqs::MPAD_ALIGN;
    int E = 32;
    for (int v : Es)
      if (v >= need) {
        E = v;
        break;
      }
    c->M_pad = 32 * E;
    c->P = (int64_t)c->N + c->M + (int64_t)c->M * c->N;
    if (!nqs::rbm_supported(c, &why)) {
      delete c;
      return fail(nullptr, NQS_EUNSUPPORTED, why);
    }
  } else if (model->kind == NQS_DENSE) {
    if (!nqs::dense_setup(c, model, &why)) {
      delete c;
      return fail(nullptr, NQS_EUNSUPPORTED, why);
    }
    c->M = 32;  // the RBM tables below are not used by a dense context (kept minimal)
    c->M_pad = 32;
  } else {
    if (!nqs::rescnn_setup(c, model, &why)) {
      delete c;
      return fail(nullptr, NQS_EUNSUPPORTED, why);
    }
    c->M = 32;  // as for the dense ansatz, the RBM tables are not used
    c->M_pad = 32;
  }
  if (ham->kind == NQS_HEISENBERG && (c->N % 2) != 0) {
    delete c;
    return fail(nullptr, NQS_EINVAL, "zero-magnetisation sector needs an even number of sites");
  }

  std::vector<int2> bonds;
  std::vector<float> bJ;
  build_bonds(c, bonds, bJ);
  c->n_bonds = (int)bonds.size();
  const size_t tsz = c->dtype == NQS_F32 ? 4 : 2;
  if ((e = cudaMalloc(&c->d_bounds, 2 * sizeof(float))) != cudaSuccess || (e = dev_alloc(&c->d_status, 1)) != cudaSuccess || (e = dev_alloc(&c->d_scratch, 5 * nqs::STATS_MAX_BLOCKS)) ||
      (e = dev_alloc(&c->d_bonds, bonds.size())) || (e = dev_alloc(&c->d_bondJ, bJ.size())) ||
      (e = dev_alloc(&c->d_a, c->N)) || (e = dev_alloc(&c->d_b, c->M_pad)) ||
      (e = dev_alloc(&c->d_Wt, (size_t)c->N * c->M_pad)) ||
      (e = cudaMalloc(&c->d_R, (size_t)c->N * c->M_pad * tsz)) || (e = dev_alloc(&c->d_aK, c->N + 1)) ||
      (e = dev_alloc(&c->d_Wm, (size_t)c->N * c->M)) || (e = dev_alloc(&c->d_bm, c->M))) {
    free_all(c);
    delete c;
    return fail(nullptr, NQS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  if (c->dtype == NQS_F32) {
    c->d_a32 = c->d_a;
    c->d_b32 = c->d_b;
    c->d_Wt32 = c->d_Wt;
    c->d_R32 = (float *)c->d_R;
    c->d_aK32 = c->d_aK;
  } else if ((e = dev_alloc(&c->d_a32, c->N)) || (e = dev_alloc(&c->d_b32, c->M_pad)) ||
             (e = dev_alloc(&c->d_Wt32, (size_t)c->N * c->M_pad)) ||
             (e = dev_alloc(&c->d_R32, (size_t)c->N * c->M_pad)) || (e = dev_alloc(&c->d_aK32, c->N + 1))) {
    free_all(c);
    delete c;
    return fail(nullptr, NQS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemset(c->d_status, 0, sizeof(int))) ||
      (e = cudaMemcpy(c->d_bonds, bonds.data(), bonds.size() * sizeof(int2), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c->d_bondJ, bJ.data(), bJ.size() * sizeof(float), cudaMemcpyHostToDevice))) {
    free_all(c);
    delete c;
    return cuda_fail(nullptr, e, "nqs_create");
  }
  if (c->model_kind == NQS_DENSE && (e = nqs::dense_alloc_params(c)) != cudaSuccess) {
    nqs::dense_free(c);
    free_all(c);
    delete c;
    return fail(nullptr, NQS_ENOMEM, std::string("dense allocation failed: ") + cudaGetErrorString(e));
  }
  if (c->model_kind == NQS_RESCNN && (e = nqs::rescnn_alloc(c)) != cudaSuccess) {
    nqs::rescnn_free(c);
    free_all(c);
    delete c;
    return fail(nullptr, NQS_ENOMEM, std::string("ResCNN allocation failed: ") + cudaGetErrorString(e));
  }
  *out = c;
  return NQS_OK;
}

void nqs_destroy(nqs_ctx *c) {
  if (!c) return;
  if (c->model_kind == NQS_DENSE) nqs::dense_free(c);
  if (c->model_kind == NQS_RESCNN) nqs::rescnn_free(c);
  free_all(c);
  delete c;
}

nqs_status nqs_set_option(nqs_ctx *c, int32_t option, int64_t value) {
  if (!c) return NQS_EINVAL;
  if (option == NQS_OPT_REFRESH) {
    if (value < 1 || value > (1 << 30)) return fail(c, NQS_EINVAL, "refresh must be >= 1");
    c->refresh = (int)value;
    return NQS_OK;
  }
  if (option == NQS_OPT_MAX_ROWS) {
    if (c->model_kind != NQS_DENSE) return NQS_OK;
    if (value < 128 || value > (int64_t)1 << 24) return fail(c, NQS_EINVAL, "max rows: 128 .. 2^24");
    cudaError_t e = nqs::dense_alloc_rows(c, value);
    return e == cudaSuccess ? NQS_OK : fail(c, NQS_ENOMEM, "dense workspace allocation failed");
  }
  if (option == NQS_OPT_DENSE_FUSED) {
    if (value != 0 && value != 1) return fail(c, NQS_EINVAL, "dense fused sampler: 0 or 1");
    c->dense_fused = (int)value;
    return NQS_OK;
  }
  if (option == NQS_OPT_CHAINS_PER_WARP) {
    if (value != 0 && value != 1 && value != 2 && value != 4) return fail(c, NQS_EINVAL, "chains per warp: 0, 1, 2 or 4");
    c->chains_per_warp = (int)value;
    return NQS_OK;
  }
  return fail(c, NQS_EINVAL, "unknown option");
}

nqs_status nqs_set_params(nqs_ctx *c, const double *params, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (bad_ptr(params)) return fail(c, NQS_EINVAL, "nqs_set_params: null params");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int zero = 0;
  cudaError_t e = cudaMemcpyAsync(c->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "nqs_set_params");
  e = c->model_kind == NQS_DENSE    ? nqs::dense_prepare(c, params, s)
      : c->model_kind == NQS_RESCNN ? nqs::rescnn_prepare(c, params, s)
                                    : nqs::rbm_prepare(c, params, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "nqs_set_params");
  int st = 0;
  float bounds[2] = {0.f, 0.f};
  if ((e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (c->model_kind == NQS_RBM &&
       (e = cudaMemcpyAsync(bounds, c->d_bounds, sizeof(bounds), cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "nqs_set_params");
  if (c->model_kind == NQS_RBM) c->renorm = nqs::rbm_renorm_interval(c, bounds[0], bounds[1]);
  if (st & nqs::STATUS_RANGE) {
    cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
    return fail(c, NQS_EINVAL, c->dtype == NQS_F16 ? "a weight is outside the F16 sampler's range (|W| <= 2.5)"
                                                   : "a weight is outside the sampler's range (|W| <= 20)");
  }
  c->params_set = true;
  return NQS_OK;
}

nqs_status nqs_init_chains(nqs_ctx *c, uint32_t *state, int64_t n, uint64_t seed, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n < 0 || (n > 0 && bad_ptr(state))) return fail(c, NQS_EINVAL, "nqs_init_chains: bad state/n");
  if (n > (int64_t)UINT32_MAX) return fail(c, NQS_EINVAL, "at most 2^32 chains");
  if (n == 0) return NQS_OK;
  cudaError_t e = nqs::init_chains(c, state, n, seed, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_init_chains");
}

nqs_status nqs_sweep(nqs_ctx *c, uint32_t *state, int64_t n_chains, int32_t n_sweeps, int32_t burn_in, uint64_t seed,
                     uint32_t sweep_offset, uint32_t *samples, float *logpsi, int64_t *n_accepted,
                     const nqs_sweep_trace *trace, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_sweep: parameters not set");
  if (n_chains < 0 || n_sweeps < 0 || burn_in < 0) return fail(c, NQS_EINVAL, "nqs_sweep: negative size");
  if (n_chains > (int64_t)UINT32_MAX) return fail(c, NQS_EINVAL, "at most 2^32 chains");
  if ((uint64_t)sweep_offset + (uint64_t)n_sweeps > (1ull << 32)) return fail(c, NQS_EINVAL, "sweep counter overflow");
  if (n_chains == 0 || n_sweeps == 0) return NQS_OK;
  if (bad_ptr(state)) return fail(c, NQS_EINVAL, "nqs_sweep: null state");
  if (c->model_kind == NQS_DENSE && n_chains > c->max_rows)
    return fail(c, NQS_EINVAL, "nqs_sweep: more chains than the dense workspace rows (NQS_OPT_MAX_ROWS)");
  cudaError_t e =
      c->model_kind == NQS_DENSE
          ? nqs::dense_sweep(c, state, n_chains, n_sweeps, burn_in, seed, sweep_offset, samples, logpsi, n_accepted,
                             trace ? trace->accept_bits : nullptr, trace ? trace->delta : nullptr,
                             reinterpret_cast<cudaStream_t>(stream))
      : c->model_kind == NQS_RESCNN
          ? nqs::rescnn_sweep(c, state, n_chains, n_sweeps, burn_in, seed, sweep_offset, samples, logpsi, n_accepted,
                              trace ? trace->accept_bits : nullptr, trace ? trace->delta : nullptr,
                              reinterpret_cast<cudaStream_t>(stream))
          : nqs::rbm_sweep(c, state, n_chains, n_sweeps, burn_in, seed, sweep_offset, samples, logpsi, n_accepted,
                           trace ? trace->accept_bits : nullptr, trace ? trace->delta : nullptr,
                           reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_sweep");
}

nqs_status nqs_logpsi(nqs_ctx *c, const uint32_t *cfg, int64_t n, float *out, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_logpsi: parameters not set");
  if (n < 0 || (n > 0 && (bad_ptr(cfg) || bad_ptr(out)))) return fail(c, NQS_EINVAL, "nqs_logpsi: bad arguments");
  if (n == 0) return NQS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = c->model_kind == NQS_DENSE    ? nqs::dense_logpsi(c, cfg, n, out, s)
                  : c->model_kind == NQS_RESCNN ? nqs::rescnn_logpsi(c, cfg, n, out, s)
                                                : nqs::rbm_logpsi(c, cfg, n, out, s);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_logpsi");
}

nqs_status nqs_local_energy(nqs_ctx *c, const uint32_t *cfg, int64_t n, float *eloc, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_local_energy: parameters not set");
  if (n < 0 || (n > 0 && (bad_ptr(cfg) || bad_ptr(eloc)))) return fail(c, NQS_EINVAL, "nqs_local_energy: bad arguments");
  if (n == 0) return NQS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = c->model_kind == NQS_DENSE    ? nqs::dense_local_energy(c, cfg, n, eloc, s)
                  : c->model_kind == NQS_RESCNN ? nqs::rescnn_local_energy(c, cfg, n, eloc, s)
                                                : nqs::rbm_local_energy(c, cfg, n, eloc, s);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_local_energy");
}

nqs_status nqs_flip_delta(nqs_ctx *c, const uint32_t *cfg, const int32_t *sites, int64_t n, float *out,
                          nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_flip_delta: parameters not set");
  if (c->ham_kind != NQS_TFIM || c->model_kind != NQS_RBM)
    return fail(c, NQS_EUNSUPPORTED, "nqs_flip_delta: RBM single-flip (TFIM) contexts only");
  if (n < 0 || (n > 0 && (bad_ptr(cfg) || bad_ptr(sites) || bad_ptr(out))))
    return fail(c, NQS_EINVAL, "nqs_flip_delta: bad arguments");
  if (n == 0) return NQS_OK;
  cudaError_t e = nqs::rbm_flip_delta(c, cfg, sites, n, out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_flip_delta");
}

size_t nqs_logpsi_grad_workspace(const nqs_ctx *c, int64_t n) {
  if (!c || n <= 0 || c->model_kind != NQS_RBM) return 0;
  return nqs::rbm_grad_workspace(c, n);
}

nqs_status nqs_logpsi_grad(nqs_ctx *c, const uint32_t *cfg, int64_t n, float *O, const float *eloc,
                           const double *stats, double *force, void *ws, size_t ws_bytes, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_logpsi_grad: parameters not set");
  if (c->model_kind == NQS_RESCNN && !nqs::rescnn_grad_supported(c))
    return fail(c, NQS_EUNSUPPORTED, "nqs_logpsi_grad: this ResCNN's residual streams exceed shared memory");
  if (n < 0 || (n > 0 && bad_ptr(cfg))) return fail(c, NQS_EINVAL, "nqs_logpsi_grad: bad arguments");
  if (force && n > 0 && (bad_ptr(eloc) || bad_ptr(stats)))
    return fail(c, NQS_EINVAL, "nqs_logpsi_grad: the force needs eloc and stats");
  if (force && n > 0 && c->model_kind == NQS_RBM && (bad_ptr(ws) || ws_bytes < nqs::rbm_grad_workspace(c, n)))
    return fail(c, NQS_EINVAL, "nqs_logpsi_grad: workspace too small");
  if (n == 0) {
    if (force) {
      cudaError_t e = cudaMemsetAsync(force, 0, (size_t)c->P * sizeof(double), reinterpret_cast<cudaStream_t>(stream));
      if (e != cudaSuccess) return cuda_fail(c, e, "nqs_logpsi_grad");
    }
    return NQS_OK;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = c->model_kind == NQS_DENSE    ? nqs::dense_logpsi_grad(c, cfg, n, O, eloc, stats, force, st)
                  : c->model_kind == NQS_RESCNN ? nqs::rescnn_logpsi_grad(c, cfg, n, O, eloc, stats, force, st)
                                                : nqs::rbm_logpsi_grad(c, cfg, n, O, eloc, stats, force, ws, st);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_logpsi_grad");
}

nqs_status nqs_stats(nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains, const int64_t *n_accepted,
                     int64_t proposals_per_chain, double *out, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n <= 0 || n_chains <= 0 || n % n_chains != 0 || bad_ptr(eloc) || bad_ptr(out))
    return fail(c, NQS_EINVAL, "nqs_stats: need n > 0 a multiple of n_chains and non-null eloc/out");
  if (n_accepted && proposals_per_chain <= 0) return fail(c, NQS_EINVAL, "nqs_stats: proposals_per_chain must be > 0");
  cudaError_t e = nqs::energy_stats(c, eloc, n, n_chains, n_accepted, proposals_per_chain, out,
                                    reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_stats");
}

nqs_status nqs_stats_moments(nqs_ctx *c, const float *eloc, int64_t n, int64_t n_chains, const int64_t *n_accepted,
                             int64_t proposals_per_chain, double *moments, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n <= 0 || n_chains <= 0 || n % n_chains != 0 || bad_ptr(eloc) || bad_ptr(moments))
    return fail(c, NQS_EINVAL, "nqs_stats_moments: need n > 0 a multiple of n_chains and non-null eloc/moments");
  if (n_accepted && proposals_per_chain <= 0)
    return fail(c, NQS_EINVAL, "nqs_stats_moments: proposals_per_chain must be > 0");
  cudaError_t e = nqs::energy_stats(c, eloc, n, n_chains, n_accepted, proposals_per_chain, nullptr,
                                    reinterpret_cast<cudaStream_t>(stream), moments);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_stats_moments");
}

nqs_status nqs_stats_finalize(const double *moments, double *out, nqs_stream stream) {
  if (bad_ptr(moments) || bad_ptr(out)) return NQS_EINVAL;
  cudaError_t e = nqs::stats_finalize(moments, out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(nullptr, e, "nqs_stats_finalize");
}

nqs_status nqs_force_share(nqs_ctx *c, const uint32_t *cfg, int64_t n, const float *eloc, const double *stats,
                           double *force, void *ws, size_t ws_bytes, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_force_share: parameters not set");
  if (c->model_kind == NQS_RESCNN && !nqs::rescnn_grad_supported(c))
    return fail(c, NQS_EUNSUPPORTED, "nqs_force_share: this ResCNN's residual streams exceed shared memory");
  if (n < 0 || bad_ptr(force) || (n > 0 && (bad_ptr(cfg) || bad_ptr(eloc) || bad_ptr(stats))))
    return fail(c, NQS_EINVAL, "nqs_force_share: bad arguments");
  if (n > 0 && c->model_kind == NQS_RBM && (bad_ptr(ws) || ws_bytes < nqs::rbm_grad_workspace(c, n)))
    return fail(c, NQS_EINVAL, "nqs_force_share: workspace too small");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(force, 0, (size_t)c->P * sizeof(double), s);
    return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_force_share");
  }
  cudaError_t e = c->model_kind == NQS_DENSE    ? nqs::dense_logpsi_grad(c, cfg, n, nullptr, eloc, stats, force, s, true)
                  : c->model_kind == NQS_RESCNN ? nqs::rescnn_logpsi_grad(c, cfg, n, nullptr, eloc, stats, force, s, true)
                                                : nqs::rbm_logpsi_grad(c, cfg, n, nullptr, eloc, stats, force, ws, s, true);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_force_share");
}

nqs_status nqs_local_energy_chains(nqs_ctx *c, const uint32_t *samples, int64_t n_chains, int64_t per_chain,
                                   float *eloc, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (!c->params_set) return fail(c, NQS_EINVAL, "nqs_local_energy_chains: parameters not set");
  if (n_chains < 0 || per_chain < 0) return fail(c, NQS_EINVAL, "nqs_local_energy_chains: negative size");
  if (n_chains == 0 || per_chain == 0) return NQS_OK;
  if (bad_ptr(samples) || bad_ptr(eloc)) return fail(c, NQS_EINVAL, "nqs_local_energy_chains: null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = c->model_kind == NQS_DENSE    ? nqs::dense_local_energy(c, samples, n_chains * per_chain, eloc, s)
                  : c->model_kind == NQS_RESCNN ? nqs::rescnn_local_energy(c, samples, n_chains * per_chain, eloc, s)
                                                : nqs::rbm_local_energy_chains(c, samples, n_chains, per_chain, eloc, s);
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_local_energy_chains");
}

nqs_status nqs_set_noise(nqs_ctx *c, double sigma, uint64_t key) {
  if (!c) return NQS_EINVAL;
  if (!(sigma >= 0.0) || sigma > 100.0) return fail(c, NQS_EINVAL, "nqs_set_noise: need 0 <= sigma <= 100");
  if (sigma > 0.0 && (c->model_kind != NQS_RBM || c->ham_kind != NQS_TFIM || c->dtype != NQS_F32))
    return fail(c, NQS_EUNSUPPORTED, "nqs_set_noise: the noisy RBM is built for FP32 TFIM RBM contexts");
  c->noise_sigma = sigma;
  c->noise_key = key;
  return NQS_OK;
}

size_t nqs_minsr_workspace(const nqs_ctx *c, int64_t n) {
  if (!c || n < 2 || n > 8192) return 0;
  return nqs::minsr_workspace(c, n);
}

nqs_status nqs_minsr(nqs_ctx *c, const float *O, int64_t n, const float *eloc, const double *stats, double lambda,
                     double *dtheta, double *T_out, void *workspace, size_t workspace_bytes, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  if (n < 2 || n > 8192) return fail(c, NQS_EINVAL, "nqs_minsr: need 2 <= n <= 8192 samples");
  if (!(lambda > 0.0)) return fail(c, NQS_EINVAL, "nqs_minsr: lambda must be positive");
  if (bad_ptr(O) || bad_ptr(eloc) || bad_ptr(stats) || bad_ptr(dtheta) || bad_ptr(workspace))
    return fail(c, NQS_EINVAL, "nqs_minsr: null argument");
  if (workspace_bytes < nqs::minsr_workspace(c, n)) return fail(c, NQS_EINVAL, "nqs_minsr: workspace too small");
  cudaError_t e = nqs::minsr(c, O, n, eloc, stats, lambda, dtheta, T_out, workspace,
                             reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_minsr");
}

nqs_status nqs_check_status(nqs_ctx *c, nqs_stream stream) {
  if (!c) return NQS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = 0;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess || (e = cudaMemsetAsync(c->d_status, 0, sizeof(int), s)) != cudaSuccess)
    return cuda_fail(c, e, "nqs_check_status");
  if (st & nqs::STATUS_TIMEOUT) return fail(c, NQS_ETIMEOUT, "a bounded device wait ran out");
  if (st & nqs::STATUS_RANGE) return fail(c, NQS_EINVAL, "a value left the documented range");
  return NQS_OK;
}

}  // extern "C"
