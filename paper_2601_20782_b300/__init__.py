"""B300 (sm_103a) hot path of neural-quantum-state VMC: thin Python binding of libnqs.so.

Every call marshals torch CUDA tensors (device pointers) and the current CUDA
stream into the C ABI of include/nqs.h; all arithmetic runs in the library's
kernels.  There is no CPU fallback: importing this package raises if the
library has not been built, and every call raises ``NQSError`` on failure.

Packed configurations are int32 (or uint32) tensors of shape [n, W], W = ceil(N/32),
bit (i mod 32) of word i // 32 set iff s_i = +1.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnqs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2601_20782_b300/build.py` "
                      "(or __graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)

NQS_OK, NQS_EINVAL, NQS_ECUDA, NQS_ENOMEM, NQS_ETIMEOUT, NQS_EUNSUPPORTED = range(6)
DTYPES = {"f32": 0, "bf16": 1, "f16": 2, "fp8": 3}
MODELS = {"rbm": 0, "dense": 1, "rescnn": 2}
HAMS = {"tfim": 0, "heisenberg": 1}
OPT_REFRESH, OPT_CHAINS_PER_WARP, OPT_MAX_ROWS, OPT_DENSE_FUSED = 0, 1, 2, 3


class NQSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nqs error {code}: {msg}")
        self.code = code


class HamDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("J1", ctypes.c_double), ("J2", ctypes.c_double), ("h", ctypes.c_double),
                ("marshall", ctypes.c_int32)]


class ModelDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("widths", ctypes.POINTER(ctypes.c_int32))]


class SweepTrace(ctypes.Structure):
    _fields_ = [("accept_bits", ctypes.c_void_p), ("delta", ctypes.c_void_p)]


class BatchItem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("state", ctypes.c_void_p), ("n_chains", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("samples", ctypes.c_void_p), ("logpsi", ctypes.c_void_p),
                ("n_accepted", ctypes.c_void_p), ("accept_bits", ctypes.c_void_p), ("eloc", ctypes.c_void_p),
                ("stats", ctypes.c_void_p), ("O", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("max_warps_per_cta", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("n_work_items", ctypes.c_int32), ("n_staged", ctypes.c_int32),
                ("stage_bytes", ctypes.c_int64), ("n_tuned", ctypes.c_int32),
                ("tuned_variant", ctypes.c_int32 * 16), ("tuned_warps", ctypes.c_int32 * 16),
                ("tuned_ms", ctypes.c_float * 16)]


_vp, _i32, _i64, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_size_t)
_SIGS = {
    "nqs_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(ModelDesc), ctypes.POINTER(HamDesc), _i32]),
    "nqs_destroy": (None, [_vp]),
    "nqs_last_error": (ctypes.c_char_p, [_vp]),
    "nqs_n_sites": (_i32, [_vp]),
    "nqs_words_per_config": (_i32, [_vp]),
    "nqs_n_params": (_i64, [_vp]),
    "nqs_n_bonds": (_i32, [_vp]),
    "nqs_set_option": (_i32, [_vp, _i32, _i64]),
    "nqs_set_params": (_i32, [_vp, _vp, _vp]),
    "nqs_init_chains": (_i32, [_vp, _vp, _i64, _u64, _vp]),
    "nqs_sweep": (_i32, [_vp, _vp, _i64, _i32, _i32, _u64, _u32, _vp, _vp, _vp, ctypes.POINTER(SweepTrace), _vp]),
    "nqs_logpsi": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "nqs_flip_delta": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "nqs_local_energy": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "nqs_logpsi_grad_workspace": (_sz, [_vp, _i64]),
    "nqs_logpsi_grad": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nqs_stats": (_i32, [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp]),
    "nqs_check_status": (_i32, [_vp, _vp]),
    "nqs_force_noalloc": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "nqs_probe_alu": (_i32, [_i32, _i64, _i32, _i64, _vp, _vp]),
    "nqs_stats_moments": (_i32, [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp]),
    "nqs_stats_finalize": (_i32, [_vp, _vp, _vp]),
    "nqs_force_share": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nqs_selftest_tc_gemm": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "nqs_selftest_tc_shift": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _vp, _vp, _vp]),
    "nqs_set_noise": (_i32, [_vp, ctypes.c_double, _u64]),
    "nqs_local_energy_chains": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp]),
    "nqs_minsr_workspace": (_sz, [_vp, _i64]),
    "nqs_minsr": (_i32, [_vp, _vp, _i64, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _sz, _vp]),
    "nqs_batch_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(BatchItem), _i32, _i32, _i32, _i32, _vp]),
    "nqs_batch_sweep": (_i32, [_vp, _u32, _vp]),
    "nqs_batch_step": (_i32, [_vp, _u32, _vp]),
    "nqs_batch_info": (_i32, [_vp, ctypes.POINTER(BatchInfo)]),
    "nqs_batch_last_error": (ctypes.c_char_p, [_vp]),
    "nqs_batch_destroy": (None, [_vp]),
    "nqs_crbm_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(HamDesc), _i32]),
    "nqs_crbm_destroy": (None, [_vp]),
    "nqs_crbm_last_error": (ctypes.c_char_p, [_vp]),
    "nqs_crbm_n_params": (_i64, [_vp]),
    "nqs_crbm_words_per_config": (_i32, [_vp]),
    "nqs_crbm_set_refresh": (_i32, [_vp, _i32]),
    "nqs_crbm_set_params": (_i32, [_vp, _vp, _vp]),
    "nqs_crbm_init_chains": (_i32, [_vp, _vp, _i64, _u64, _vp]),
    "nqs_crbm_sweep": (_i32, [_vp, _vp, _i64, _i32, _i32, _u64, _u32, _vp, _vp, _vp, _vp]),
    "nqs_crbm_logpsi": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "nqs_crbm_local_energy": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "nqs_crbm_local_energy_chains": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "nqs_crbm_stats": (_i32, [_vp, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp]),
    "nqs_crbm_logpsi_grad": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nqs_crbm_check_status": (_i32, [_vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _ptr(t, dtypes, name, shape=None, allow_none=True):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


_WORD = (torch.int32, torch.uint32)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """One nqs_ctx: a Hamiltonian, an ansatz and the dtype of its sampling copy.

    model="rbm" (n_hidden), "dense" (widths) or "rescnn" (n_hidden = filters, n_blocks)."""

    def __init__(self, ham="tfim", Lx=4, Ly=1, J1=1.0, J2=0.0, h=0.0, marshall=False,
                 model="rbm", n_hidden=0, widths=(), dtype="f32", n_blocks=0):
        self._h = None
        hd = HamDesc(HAMS[ham], Lx, Ly, J1, J2, h, int(bool(marshall)))
        self._widths = (ctypes.c_int32 * max(len(widths), 1))(*widths)
        n_layers = n_blocks if model == "rescnn" else len(widths)
        md = ModelDesc(MODELS[model], n_hidden, n_layers, self._widths)
        out = ctypes.c_void_p()
        st = _lib.nqs_create(ctypes.byref(out), ctypes.byref(md), ctypes.byref(hd), DTYPES[dtype])
        if st != NQS_OK:
            raise NQSError(st, _lib.nqs_last_error(None).decode())
        self._h = out
        self.N = _lib.nqs_n_sites(out)
        self.W = _lib.nqs_words_per_config(out)
        self.P = _lib.nqs_n_params(out)
        self.n_bonds = _lib.nqs_n_bonds(out)
        self.dtype = dtype

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.nqs_destroy(self._h)
            self._h = None

    def _check(self, st):
        if st != NQS_OK:
            raise NQSError(st, _lib.nqs_last_error(self._h).decode())

    def set_option(self, option, value):
        self._check(_lib.nqs_set_option(self._h, option, int(value)))

    def set_params(self, params):
        self._check(_lib.nqs_set_params(self._h, _ptr(params, (torch.float64,), "params", (self.P,), False), _stream()))

    def init_chains(self, state, seed):
        n = state.shape[0]
        self._check(_lib.nqs_init_chains(self._h, _ptr(state, _WORD, "state", (n, self.W), False), n,
                                         int(seed) & (2 ** 64 - 1), _stream()))

    def sweep(self, state, n_sweeps, burn_in, seed, sweep_offset=0, samples=None, logpsi=None,
              n_accepted=None, accept_bits=None, delta=None):
        C = state.shape[0]
        K = max(n_sweeps - burn_in, 0)
        tr = None
        if accept_bits is not None or delta is not None:
            tr = SweepTrace(_ptr(accept_bits, _WORD, "accept_bits", (C, n_sweeps, self.W)),
                            _ptr(delta, (torch.float32,), "delta", (C, n_sweeps, self.N)))
        self._check(_lib.nqs_sweep(
            self._h, _ptr(state, _WORD, "state", (C, self.W), False), C, n_sweeps, burn_in,
            int(seed) & (2 ** 64 - 1), int(sweep_offset),
            _ptr(samples, _WORD, "samples", (K * C, self.W)),
            _ptr(logpsi, (torch.float32,), "logpsi", (K * C,)),
            _ptr(n_accepted, (torch.int64,), "n_accepted", (C,)),
            ctypes.byref(tr) if tr is not None else None, _stream()))

    def logpsi(self, configs, out):
        n = configs.shape[0]
        self._check(_lib.nqs_logpsi(self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
                                    _ptr(out, (torch.float32,), "out", (n,), False), _stream()))

    def flip_delta(self, configs, sites, out):
        """log psi(flip_{sites[x]} configs[x]) - log psi(configs[x]) as the sampler evaluates it."""
        n = configs.shape[0]
        self._check(_lib.nqs_flip_delta(self._h, _ptr(configs, _WORD, "configs", (n, self.W), False),
                                        _ptr(sites, (torch.int32,), "sites", (n,), False), n,
                                        _ptr(out, (torch.float32,), "out", (n,), False), _stream()))

    def local_energy(self, configs, eloc):
        n = configs.shape[0]
        self._check(_lib.nqs_local_energy(self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
                                          _ptr(eloc, (torch.float32,), "eloc", (n,), False), _stream()))

    def logpsi_grad_workspace(self, n):
        return int(_lib.nqs_logpsi_grad_workspace(self._h, n))

    def logpsi_grad(self, configs, O=None, eloc=None, stats=None, force=None, workspace=None):
        n = configs.shape[0]
        ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
        self._check(_lib.nqs_logpsi_grad(
            self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
            _ptr(O, (torch.float32,), "O", (n, self.P)), _ptr(eloc, (torch.float32,), "eloc", (n,)),
            _ptr(stats, (torch.float64,), "stats"), _ptr(force, (torch.float64,), "force", (self.P,)),
            _ptr(workspace, (torch.uint8, torch.float64, torch.float32, torch.int32), "workspace"), ws_bytes,
            _stream()))

    def stats(self, eloc, n_chains, out, n_accepted=None, proposals_per_chain=0):
        n = eloc.shape[0]
        self._check(_lib.nqs_stats(self._h, _ptr(eloc, (torch.float32,), "eloc", (n,), False), n, n_chains,
                                   _ptr(n_accepted, (torch.int64,), "n_accepted", (n_chains,)),
                                   int(proposals_per_chain), _ptr(out, (torch.float64,), "out", (5,), False),
                                   _stream()))

    def stats_moments(self, eloc, n_chains, moments, n_accepted=None, proposals_per_chain=0):
        """nqs_stats_moments: the additive moments [8] of these chains' statistics."""
        n = eloc.shape[0]
        self._check(_lib.nqs_stats_moments(self._h, _ptr(eloc, (torch.float32,), "eloc", (n,), False), n, n_chains,
                                           _ptr(n_accepted, (torch.int64,), "n_accepted", (n_chains,)),
                                           int(proposals_per_chain),
                                           _ptr(moments, (torch.float64,), "moments", (8,), False), _stream()))

    def stats_finalize(self, moments, out):
        """nqs_stats_finalize: statistics [5] from (summed) moments [8]."""
        self._check(_lib.nqs_stats_finalize(_ptr(moments, (torch.float64,), "moments", (8,), False),
                                            _ptr(out, (torch.float64,), "out", (5,), False), _stream()))

    def force_share(self, configs, eloc, stats, force, workspace=None):
        """nqs_force_share: (1 / stats[4]) sum_x O(x) (eloc[x] - stats[0]) over these rows."""
        n = configs.shape[0]
        ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
        self._check(_lib.nqs_force_share(
            self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
            _ptr(eloc, (torch.float32,), "eloc", (n,), n == 0), _ptr(stats, (torch.float64,), "stats", (5,), n == 0),
            _ptr(force, (torch.float64,), "force", (self.P,), False),
            _ptr(workspace, (torch.uint8, torch.float64, torch.float32, torch.int32), "workspace"), ws_bytes,
            _stream()))

    def force_noalloc(self, configs, eloc, stats, force):
        """nqs_force_noalloc: the force without a workspace (built-in device scratch)."""
        n = configs.shape[0]
        self._check(_lib.nqs_force_noalloc(
            self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
            _ptr(eloc, (torch.float32,), "eloc", (n,), False), _ptr(stats, (torch.float64,), "stats", None, False),
            _ptr(force, (torch.float64,), "force", (self.P,), False), _stream()))

    def local_energy_chains(self, samples, n_chains, eloc):
        """nqs_local_energy_chains: eloc of sweep-major samples of n_chains chains."""
        n = samples.shape[0]
        if n % n_chains:
            raise ValueError("samples rows must be a multiple of n_chains")
        self._check(_lib.nqs_local_energy_chains(
            self._h, _ptr(samples, _WORD, "samples", (n, self.W), False), n_chains, n // n_chains,
            _ptr(eloc, (torch.float32,), "eloc", (n,), False), _stream()))

    def set_noise(self, sigma, key=0):
        """Noisy RBM (nqs_set_noise): sample |psi~|^2, log psi~ = log psi + zeta(x)/2."""
        self._check(_lib.nqs_set_noise(self._h, float(sigma), int(key) & (2 ** 64 - 1)))

    def minsr_workspace(self, n):
        return int(_lib.nqs_minsr_workspace(self._h, n))

    def minsr(self, O, eloc, stats, lam, dtheta, T_out=None, workspace=None):
        """dtheta = Obar^T (Obar Obar^T + lam I)^-1 ebar (nqs_minsr); allocates the workspace if none."""
        n = O.shape[0]
        if workspace is None:
            workspace = torch.empty(self.minsr_workspace(n), dtype=torch.uint8, device=O.device)
        self._check(_lib.nqs_minsr(
            self._h, _ptr(O, (torch.float32,), "O", (n, self.P), False), n,
            _ptr(eloc, (torch.float32,), "eloc", (n,), False), _ptr(stats, (torch.float64,), "stats", None, False),
            float(lam), _ptr(dtheta, (torch.float64,), "dtheta", (self.P,), False),
            _ptr(T_out, (torch.float64,), "T_out", (n, n)),
            _ptr(workspace, (torch.uint8,), "workspace", None, False), workspace.numel(), _stream()))

    def check_status(self):
        self._check(_lib.nqs_check_status(self._h, _stream()))


class Batch:
    """nqs_batch: many TFIM RBM instances sampled by one persistent launch.

    items: list of dicts with keys ctx (Context), state (required), seed (required) and the
    optional device tensors samples, logpsi, n_accepted, accept_bits, eloc, stats, O (shapes as
    for Context.sweep / local_energy / stats / logpsi_grad).  warps_per_cta = 0 autotunes."""

    def __init__(self, items, n_sweeps, burn_in, warps_per_cta=0):
        self._h = None
        K = max(n_sweeps - burn_in, 0)
        arr = (BatchItem * len(items))()
        self._keep = items                      # the library keeps the pointers
        for k, it in enumerate(items):
            c = it["ctx"]
            C = it["state"].shape[0]
            arr[k] = BatchItem(
                c._h, _ptr(it["state"], _WORD, "state", (C, c.W), False), C, int(it["seed"]) & (2 ** 64 - 1),
                _ptr(it.get("samples"), _WORD, "samples", (K * C, c.W)),
                _ptr(it.get("logpsi"), (torch.float32,), "logpsi", (K * C,)),
                _ptr(it.get("n_accepted"), (torch.int64,), "n_accepted", (C,)),
                _ptr(it.get("accept_bits"), _WORD, "accept_bits", (C, n_sweeps, c.W)),
                _ptr(it.get("eloc"), (torch.float32,), "eloc", (K * C,)),
                _ptr(it.get("stats"), (torch.float64,), "stats", (5,)),
                _ptr(it.get("O"), (torch.float32,), "O", (C, c.P)))
        out = ctypes.c_void_p()
        st = _lib.nqs_batch_create(ctypes.byref(out), arr, len(items), n_sweeps, burn_in, warps_per_cta, _stream())
        if st != NQS_OK:
            raise NQSError(st, "nqs_batch_create failed")
        self._h = out
        self.n_sweeps, self.burn_in = n_sweeps, burn_in

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.nqs_batch_destroy(self._h)
            self._h = None

    def _check(self, st):
        if st != NQS_OK:
            raise NQSError(st, _lib.nqs_batch_last_error(self._h).decode())

    def sweep(self, sweep_offset=0):
        self._check(_lib.nqs_batch_sweep(self._h, int(sweep_offset), _stream()))

    def step(self, sweep_offset=0):
        self._check(_lib.nqs_batch_step(self._h, int(sweep_offset), _stream()))

    def info(self):
        i = BatchInfo()
        self._check(_lib.nqs_batch_info(self._h, ctypes.byref(i)))
        return {"warps_per_cta": i.warps_per_cta, "max_warps_per_cta": i.max_warps_per_cta, "ctas": i.ctas,
                "variant": i.variant, "n_work_items": i.n_work_items, "n_staged": i.n_staged,
                "stage_bytes": i.stage_bytes,
                "tuned": [(i.tuned_variant[q], i.tuned_warps[q], i.tuned_ms[q]) for q in range(i.n_tuned)]}


class LogPsi(torch.autograd.Function):
    """log psi(configs; params) as a differentiable function of the FP64 parameter vector.

    forward: nqs_set_params(params), then nqs_logpsi(configs) -> FP32 [n].
    backward: d/dparams of sum_x g_x log psi(x) = sum_x g_x O(x), the hand-written backward
    (App. I, Eq. forces) in the library's force kernel: nqs_force_share with eloc = g and
    stats = (0, 0, 0, 0, 1) (no centring, divisor 1).  No O rows are materialised.  The derivative is
    that of the FP32 rounding of the master parameters; the forward of a 16-bit context is its
    sampling copy's log psi.

    Use: LogPsi.apply(ctx, params, configs) with params a CUDA float64 tensor [P] that
    requires grad, configs packed [n, W]."""

    @staticmethod
    def forward(fctx, nctx, params, configs):
        n = configs.shape[0]
        nctx.set_params(params.detach().contiguous())
        out = torch.empty(n, dtype=torch.float32, device=configs.device)
        nctx.logpsi(configs, out)
        fctx.nctx = nctx
        fctx.save_for_backward(configs)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        (configs,) = fctx.saved_tensors
        nctx = fctx.nctx
        n = configs.shape[0]
        g = grad_out.detach().to(torch.float32).contiguous()
        stats = torch.tensor([0.0, 0.0, 0.0, 0.0, 1.0], dtype=torch.float64, device=configs.device)
        vjp = torch.empty(nctx.P, dtype=torch.float64, device=configs.device)
        ws = torch.empty(max(nctx.logpsi_grad_workspace(n), 1), dtype=torch.uint8, device=configs.device)
        nctx.force_share(configs, g, stats, vjp, ws)
        return None, vjp, None


PROBE_KINDS = {"ffma": 0, "ffma2": 1, "fmul2": 2, "hfma2": 3, "bfma2": 4, "lg2": 5, "ex2": 6}
# operations per lane per probed instruction
PROBE_OPS = {"ffma": 1, "ffma2": 2, "fmul2": 2, "hfma2": 2, "bfma2": 2, "lg2": 1, "ex2": 1}


def probe_alu(kind, blocks, threads, iters, sink):
    """nqs_probe_alu: launches the issue-rate probe of one instruction on the current stream
    (time it with CUDA events); sink is a CUDA float32 tensor of at least `blocks` elements."""
    if sink.numel() < blocks:
        raise ValueError("sink needs at least `blocks` elements")
    st = _lib.nqs_probe_alu(PROBE_KINDS[kind], blocks, threads, iters, _ptr(sink, (torch.float32,), "sink"),
                            _stream())
    if st != NQS_OK:
        raise NQSError(st, "nqs_probe_alu failed")


def selftest_tc_gemm(A, B, a_transposed=False, b_transposed=False):
    """D = A B^T on the tensor cores (tcgen05).  A [128 x K] (or [K x 128] when a_transposed),
    B [N x K] (or [K x N] when b_transposed), BF16 CUDA tensors."""
    K = A.shape[0] if a_transposed else A.shape[1]
    N = B.shape[1] if b_transposed else B.shape[0]
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = _lib.nqs_selftest_tc_gemm(_ptr(A, (torch.bfloat16,), "A", (K, 128) if a_transposed else (128, K), False),
                                   _ptr(B, (torch.bfloat16,), "B", (K, N) if b_transposed else (N, K), False),
                                   _ptr(D, (torch.float32,), "D"), N, K,
                                   int(a_transposed) | (int(b_transposed) << 1),
                                   _ptr(status, (torch.int32,), "status"), _stream())
    if st != NQS_OK:
        raise NQSError(st, "nqs_selftest_tc_gemm failed")
    return D, status


def selftest_tc_shift(A, B, offs, base):
    """D [128 x 16] = sum_t A[base + offs[t] : base + offs[t] + 128] @ B[t]^T on the tensor cores
    (no-swizzle operand planes).  A [n_rows x 16], B [n_taps x 16 x 16] BF16 CUDA tensors."""
    n_rows, n_taps = A.shape[0], B.shape[0]
    D = torch.empty((128, 16), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    o = (ctypes.c_int32 * max(n_taps, 1))(*offs)
    st = _lib.nqs_selftest_tc_shift(_ptr(A, (torch.bfloat16,), "A", (n_rows, 16), False), n_rows,
                                    _ptr(B, (torch.bfloat16,), "B", (n_taps, 16, 16), False), n_taps, o, base,
                                    _ptr(D, (torch.float32,), "D"), _ptr(status, (torch.int32,), "status"), _stream())
    if st != NQS_OK:
        raise NQSError(st, "nqs_selftest_tc_shift failed")
    return D, status


def pack_spins(s):
    """[n, N] +-1 tensor (any device) -> [n, W] int32 packed words (same device)."""
    n, N = s.shape
    W = (N + 31) // 32
    bits = (s > 0).to(torch.int64)
    pad = torch.zeros((n, W * 32 - N), dtype=torch.int64, device=s.device)
    bits = torch.cat([bits, pad], dim=1).view(n, W, 32)
    words = (bits << torch.arange(32, device=s.device, dtype=torch.int64)).sum(dim=2)
    return torch.where(words >= 2 ** 31, words - 2 ** 32, words).to(torch.int32)


def unpack_spins(words, N):
    """[n, W] packed words -> [n, N] int8 +-1 (same device)."""
    w = words.to(torch.int64) & 0xFFFFFFFF
    bits = (w.unsqueeze(2) >> torch.arange(32, device=w.device, dtype=torch.int64)) & 1
    return (bits.view(words.shape[0], -1)[:, :N] * 2 - 1).to(torch.int8)


class ComplexContext:
    """One nqs_crbm: the complex-parameter RBM (App. G, complex a, b, W) on a TFIM.

    Parameters and the force are complex128 tensors [P], O rows complex64 [n, P], log psi
    complex64 [n]; local energies are two float32 tensors (real and imaginary parts)."""

    def __init__(self, Lx=4, Ly=1, J1=1.0, h=0.0, n_hidden=4):
        self._h = None
        hd = HamDesc(HAMS["tfim"], Lx, Ly, J1, 0.0, h, 0)
        out = ctypes.c_void_p()
        st = _lib.nqs_crbm_create(ctypes.byref(out), ctypes.byref(hd), n_hidden)
        if st != NQS_OK:
            raise NQSError(st, _lib.nqs_crbm_last_error(None).decode())
        self._h = out
        self.N = Lx * Ly
        self.M = n_hidden
        self.W = _lib.nqs_crbm_words_per_config(out)
        self.P = _lib.nqs_crbm_n_params(out)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.nqs_crbm_destroy(self._h)
            self._h = None

    def _check(self, st):
        if st != NQS_OK:
            raise NQSError(st, _lib.nqs_crbm_last_error(self._h).decode())

    def set_refresh(self, refresh):
        self._check(_lib.nqs_crbm_set_refresh(self._h, int(refresh)))

    def set_params(self, params):
        self._check(_lib.nqs_crbm_set_params(self._h, _ptr(params, (torch.complex128,), "params", (self.P,), False),
                                             _stream()))

    def init_chains(self, state, seed):
        n = state.shape[0]
        self._check(_lib.nqs_crbm_init_chains(self._h, _ptr(state, _WORD, "state", (n, self.W), False), n,
                                              int(seed) & (2 ** 64 - 1), _stream()))

    def sweep(self, state, n_sweeps, burn_in, seed, sweep_offset=0, samples=None, n_accepted=None,
              accept_bits=None, delta=None):
        C = state.shape[0]
        K = max(n_sweeps - burn_in, 0)
        tr = None
        if accept_bits is not None or delta is not None:
            tr = SweepTrace(_ptr(accept_bits, _WORD, "accept_bits", (C, n_sweeps, self.W)),
                            _ptr(delta, (torch.float32,), "delta", (C, n_sweeps, self.N)))
        self._check(_lib.nqs_crbm_sweep(
            self._h, _ptr(state, _WORD, "state", (C, self.W), False), C, n_sweeps, burn_in,
            int(seed) & (2 ** 64 - 1), int(sweep_offset), _ptr(samples, _WORD, "samples", (K * C, self.W)),
            _ptr(n_accepted, (torch.int64,), "n_accepted", (C,)), ctypes.byref(tr) if tr is not None else None,
            _stream()))

    def logpsi(self, configs, out):
        n = configs.shape[0]
        self._check(_lib.nqs_crbm_logpsi(self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
                                         _ptr(out, (torch.complex64,), "out", (n,), False), _stream()))

    def local_energy(self, configs, eloc_re, eloc_im):
        n = configs.shape[0]
        self._check(_lib.nqs_crbm_local_energy(
            self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
            _ptr(eloc_re, (torch.float32,), "eloc_re", (n,), False),
            _ptr(eloc_im, (torch.float32,), "eloc_im", (n,), False), _stream()))

    def local_energy_chains(self, samples, n_chains, eloc_re, eloc_im):
        """nqs_crbm_local_energy_chains: eloc of sweep-major samples of n_chains chains."""
        n = samples.shape[0]
        if n % n_chains:
            raise ValueError("samples rows must be a multiple of n_chains")
        self._check(_lib.nqs_crbm_local_energy_chains(
            self._h, _ptr(samples, _WORD, "samples", (n, self.W), False), n_chains, n // n_chains,
            _ptr(eloc_re, (torch.float32,), "eloc_re", (n,), False),
            _ptr(eloc_im, (torch.float32,), "eloc_im", (n,), False), _stream()))

    def stats(self, eloc_re, eloc_im, n_chains, out, n_accepted=None, proposals_per_chain=0):
        n = eloc_re.shape[0]
        self._check(_lib.nqs_crbm_stats(
            self._h, _ptr(eloc_re, (torch.float32,), "eloc_re", (n,), False),
            _ptr(eloc_im, (torch.float32,), "eloc_im", (n,), False), n, n_chains,
            _ptr(n_accepted, (torch.int64,), "n_accepted", (n_chains,)), int(proposals_per_chain),
            _ptr(out, (torch.float64,), "out", (6,), False), _stream()))

    def logpsi_grad(self, configs, O=None, eloc_re=None, eloc_im=None, stats=None, force=None):
        n = configs.shape[0]
        self._check(_lib.nqs_crbm_logpsi_grad(
            self._h, _ptr(configs, _WORD, "configs", (n, self.W), False), n,
            _ptr(O, (torch.complex64,), "O", (n, self.P)), _ptr(eloc_re, (torch.float32,), "eloc_re", (n,)),
            _ptr(eloc_im, (torch.float32,), "eloc_im", (n,)), _ptr(stats, (torch.float64,), "stats", (6,)),
            _ptr(force, (torch.complex128,), "force", (self.P,)), _stream()))

    def check_status(self):
        self._check(_lib.nqs_crbm_check_status(self._h, _stream()))
