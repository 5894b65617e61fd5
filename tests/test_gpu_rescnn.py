"""Parity of the CUDA ResCNN path (App. H) with the FP64 oracle, through the C ABI.

FP32 copy (CUDA cores): log psi within 1e-5 relative; local energies within the bound the
log psi tolerance implies for the ratios psi(x') / psi(x); sweeps replayed in the oracle in
lockstep (bit-exact proposals, samples and accept counts; decisions may differ only within
tau of the threshold); the 4 x 3 sampled energy and histogram against exact enumeration;
O rows (the FP32 reverse pass) against the oracle's gradient, and the force.
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, unpack_np, unpack_accept_bits, to_words_tensor, words_from_tensor
from oracle import exact
from oracle.estimators import local_energy as oracle_eloc
from oracle.hamiltonian import TFIM
from oracle.philox import init_spins_random
from oracle.rescnn import ResCNN
from oracle.sampler import mh_sweeps
from workloads import rescnn_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LOGPSI_RTOL = 1e-5


def make(Lx, Ly, B, seed, h=3.04, dtype="f32"):
    p = nqs()
    ctx = p.Context("tfim", Lx, Ly, J1=1.0, h=h, model="rescnn", n_hidden=16, n_blocks=B, dtype=dtype)
    params = rescnn_params(16, B, seed)
    ctx.set_params(torch.from_numpy(params).cuda())
    return ctx, ResCNN(Lx, Ly, 16, B, params), TFIM(Lx, Ly, 1.0, h)


def rand_configs(n, N, seed):
    return np.random.default_rng(seed).choice([-1, 1], size=(n, N)).astype(np.int8)


@pytest.mark.parametrize("Lx,Ly,B,n", [(4, 4, 4, 517), (10, 10, 4, 131), (6, 5, 2, 77), (3, 7, 1, 40),
                                       (16, 16, 3, 9), (5, 5, 0, 33)])
def test_logpsi_fp32_matches_oracle(Lx, Ly, B, n):
    ctx, model, _ = make(Lx, Ly, B, 100 + Lx * Ly)
    s = rand_configs(n, Lx * Ly, 1)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.logpsi(to_words_tensor(pack_np(s)), out)
    ref = model.logpsi(s)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=LOGPSI_RTOL * np.maximum(1.0, np.abs(ref)).max())


@pytest.mark.parametrize("Lx,Ly,B,n", [(4, 4, 4, 37), (10, 10, 4, 9), (6, 5, 2, 23)])
def test_local_energy_fp32_matches_oracle(Lx, Ly, B, n):
    ctx, model, ham = make(Lx, Ly, B, 7 + Lx)
    s = rand_configs(n, Lx * Ly, 2)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.local_energy(to_words_tensor(pack_np(s)), out)
    ref = oracle_eloc(ham, model.logpsi, s)
    # each ratio psi(x') / psi(x) = exp(dlp) carries at most the two log psi errors
    lp = model.logpsi(s)
    off = ref - ham.diagonal(s)
    tol = 2 * LOGPSI_RTOL * np.abs(lp).max() * np.abs(off) + 1e-5 * np.abs(ref) + 1e-5
    assert np.all(np.abs(out.cpu().numpy() - ref) <= tol)


def _lockstep(Lx, Ly, B, C, T, burn, seed=5, tau=1e-3):
    ctx, model, _ = make(Lx, Ly, B, 41, h=1.0)
    N = Lx * Ly
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=seed + 1)
    s0 = unpack_np(words_from_tensor(state), N)
    np.testing.assert_array_equal(s0, init_spins_random(seed + 1, np.arange(C), N))
    K = T - burn
    samples = torch.zeros((K * C, ctx.W), dtype=torch.int32, device="cuda")
    logpsi = torch.zeros(K * C, dtype=torch.float32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    bits = torch.zeros((C, T, ctx.W), dtype=torch.int32, device="cuda")
    delta = torch.zeros((C, T, N), dtype=torch.float32, device="cuda")
    ctx.sweep(state, T, burn, seed, 3, samples, logpsi, nacc, accept_bits=bits, delta=delta)
    torch.cuda.synchronize()
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    ref = mh_sweeps(model.logpsi, s0, np.arange(C), seed, T, burn, sweep_offset=3, replay_accepts=acc, tau=tau,
                    record_deltas=True)
    np.testing.assert_array_equal(unpack_np(words_from_tensor(state), N), ref["spins"])
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), N), ref["samples"])
    np.testing.assert_array_equal(nacc.cpu().numpy(), acc.sum(axis=(1, 2)))
    lp_ref = ref["logpsi"]
    np.testing.assert_allclose(logpsi.cpu().numpy(), lp_ref, rtol=0,
                               atol=LOGPSI_RTOL * np.maximum(1.0, np.abs(lp_ref)).max())
    d = delta.cpu().numpy()
    np.testing.assert_allclose(d, ref["deltas"], rtol=0, atol=2 * LOGPSI_RTOL * np.abs(lp_ref).max())
    return ref, acc


def test_sweep_lockstep_4x4_ragged_groups():
    # 70 chains over groups of 32: two full groups and a ragged one
    ref, acc = _lockstep(4, 4, 4, 70, 3, 1)
    assert 0.05 < acc.mean() < 0.95


def test_sweep_lockstep_10x10():
    ref, acc = _lockstep(10, 10, 2, 7, 1, 0)
    assert acc.mean() > 0.02


def test_sampled_energy_4x3_matches_enumeration():
    Lx, Ly, B = 4, 3, 2
    ctx, model, ham = make(Lx, Ly, B, 77, h=1.0)
    N = Lx * Ly
    S = exact.all_configs(N)
    pi = exact.exact_pi(model.logpsi, N)
    E_exact = pi @ oracle_eloc(ham, model.logpsi, S)
    C, T, burn = 4096, 40, 10
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=9)
    samples = torch.zeros(((T - burn) * C, ctx.W), dtype=torch.int32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    ctx.sweep(state, T, burn, 123, 0, samples, None, nacc)
    eloc = torch.empty((T - burn) * C, dtype=torch.float32, device="cuda")
    ctx.local_energy(samples, eloc)
    stats = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.stats(eloc, C, stats, nacc, T * N)
    E, var, err, acc_rate, n = stats.cpu().numpy()
    assert abs(E - E_exact) < 5 * err, (E, E_exact, err)
    # the sampled histogram against the exact distribution, at the i.i.d. noise floor
    idx = exact.config_index(unpack_np(words_from_tensor(samples[-C:]), N))
    hist = np.bincount(idx, minlength=pi.size) / C
    tv = 0.5 * np.abs(hist - pi).sum()
    floor = np.mean([0.5 * np.abs(np.bincount(np.random.default_rng(k).choice(pi.size, C, p=pi),
                                              minlength=pi.size) / C - pi).sum() for k in range(4)])
    assert tv < 1.2 * floor + 0.01, (tv, floor)


def test_rescnn_rejections():
    p = nqs()
    with pytest.raises(p.NQSError):
        p.Context("tfim", 16, 1, h=1.0, model="rescnn", n_hidden=16, n_blocks=2)     # 1D
    with pytest.raises(p.NQSError):
        p.Context("tfim", 4, 4, h=1.0, model="rescnn", n_hidden=8, n_blocks=2)      # filters
    with pytest.raises(p.NQSError):
        p.Context("heisenberg", 4, 4, J1=1.0, model="rescnn", n_hidden=16, n_blocks=2)
    # O rows need one configuration's residual streams in shared memory: 512 sites x 9 streams do not fit
    big = p.Context("tfim", 16, 32, h=1.0, model="rescnn", n_hidden=16, n_blocks=8)
    big.set_params(torch.from_numpy(rescnn_params(16, 8, 3)).cuda())
    cfg = to_words_tensor(pack_np(rand_configs(2, 512, 3)))
    with pytest.raises(p.NQSError):
        big.logpsi_grad(cfg, torch.zeros((2, big.P), dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("Lx,Ly,B,n", [(4, 4, 2, 19), (10, 10, 4, 7), (5, 3, 0, 11), (6, 5, 1, 9), (16, 16, 4, 3)])
def test_grad_fp32_matches_oracle(Lx, Ly, B, n):
    """O_k = d log psi / d theta_k (nqs_logpsi_grad of a ResCNN context, the FP32 reverse pass)
    against the oracle's layer-by-layer gradient (pinned by central differences), every
    parameter group (embedding, the blocks' LN, both kernels and biases, the final LN)
    within 1e-4 of the row's largest entry."""
    ctx, model, _ = make(Lx, Ly, B, 41 + Lx)
    s = rand_configs(n, Lx * Ly, 5)
    O = torch.zeros((n, ctx.P), dtype=torch.float32, device="cuda")
    ctx.logpsi_grad(to_words_tensor(pack_np(s)), O)
    ctx.check_status()
    got = O.cpu().numpy().astype(np.float64)
    ref = model.grad(s)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-4 * scale + 1e-5 * np.abs(ref)), (err / scale).max()


@pytest.mark.parametrize("n", [64, 5000])
def test_force_fp32_matches_oracle(n):
    """F_k = mean(O_k (eps - E)) of a ResCNN context, with caller O rows and without (the
    library's chunked scratch: 5000 rows are two chunks), against the oracle's force of its
    own O rows."""
    from oracle.estimators import force as oracle_force
    ctx, model, _ = make(4, 4, 1, 61)
    s = rand_configs(n, 16, 6)
    cfg = to_words_tensor(pack_np(s))
    eps = np.random.default_rng(7).normal(-3.0, 1.0, n).astype(np.float32)
    e = torch.from_numpy(eps).cuda()
    st = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(e, n, st)
    F1 = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    F2 = torch.zeros_like(F1)
    O = torch.zeros((n, ctx.P), dtype=torch.float32, device="cuda")
    ctx.logpsi_grad(cfg, O, e, st, F1)
    ctx.logpsi_grad(cfg, None, e, st, F2)
    ref = oracle_force(model.grad(s), eps.astype(np.float64))
    tol = 2e-4 * np.abs(ref).max()
    assert np.abs(F1.cpu().numpy() - ref).max() <= tol
    assert np.abs(F2.cpu().numpy() - ref).max() <= tol


# ---- 16-bit copies on the tensor cores ---------------------------------------------------------
# The copy's definition (include/nqs.h): kernels and the activations entering a convolution
# rounded to the 16-bit type, everything else in higher precision.  Emulated here in FP64 with
# those rounding points, from the oracle's layers.
from oracle.rescnn import conv3x3, gelu, layer_norm


def round_bf16(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def round_f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


ROUND = {"bf16": round_bf16, "f16": round_f16}


def copy_logpsi(model, s, dtype):
    rnd = ROUND[dtype]
    x = model._grid(s)
    h = conv3x3(x, rnd(model.K0), model.b0)
    for (g, be, K1, b1, K2, b2) in model.blocks:
        a = rnd(gelu(layer_norm(h, g, be)[0]))
        c = rnd(gelu(conv3x3(a, rnd(K1), b1)))
        h = h + conv3x3(c, rnd(K2), b2)
    return layer_norm(h, model.gF, model.bF)[0].sum(axis=(1, 2, 3))


# The kernel computes the values that get rounded in FP32, the emulation in FP64.  Where the two
# fall on different sides of a 16-bit rounding boundary, one activation moves by one unit in the
# last place, which moves log psi by about the copy's unit roundoff u16 (2^-8 BF16, 2^-11 F16;
# Table tab:precision); a configuration sees a handful of such flips, more on larger lattices.
# FP32 accumulation error is far below that.
U16 = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def flip_tol(dtype, N):
    return 4.0 * U16[dtype] * (1.0 + np.sqrt(N / 16.0))


def check_copy(got, want, dtype, N, exact=None):
    err = np.abs(got - want)
    assert err.max() <= flip_tol(dtype, N), (err.max(), flip_tol(dtype, N))
    if exact is not None and dtype == "bf16" and len(got) >= 5:
        # the kernel reproduces the copy's deterministic deviation from the FP64 network
        assert np.corrcoef(got - exact, want - exact)[0, 1] > 0.9


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("Lx,Ly,B,n", [(4, 4, 4, 301), (10, 10, 4, 37), (6, 5, 2, 45), (16, 16, 3, 7),
                                       (5, 5, 0, 50), (3, 7, 1, 26)])
def test_logpsi_16bit_copy_matches_its_definition(dtype, Lx, Ly, B, n):
    ctx, model, _ = make(Lx, Ly, B, 100 + Lx * Ly, dtype=dtype)
    s = rand_configs(n, Lx * Ly, 5)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.logpsi(to_words_tensor(pack_np(s)), out)
    got = out.cpu().numpy()
    want = copy_logpsi(model, s, dtype)
    check_copy(got, want, dtype, Lx * Ly, model.logpsi(s) if B >= 2 else None)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_local_energy_16bit_copy(dtype):
    Lx, Ly, B, n = 6, 5, 2, 21
    ctx, model, ham = make(Lx, Ly, B, 9, dtype=dtype)
    s = rand_configs(n, Lx * Ly, 6)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.local_energy(to_words_tensor(pack_np(s)), out)
    lpf = lambda v: copy_logpsi(model, v, dtype)
    ref = oracle_eloc(ham, lpf, s)
    off = np.abs(ref - ham.diagonal(s))
    # each ratio psi(x') / psi(x) carries the rounding-boundary error of two log psi values
    rel = np.abs(out.cpu().numpy() - ref) / (off + 1e-6)
    assert rel.max() <= 2 * flip_tol(dtype, Lx * Ly) + 1e-5, rel.max()


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_sweep_16bit_lockstep_with_its_definition(dtype):
    # decisions replayed against the copy's own log psi: equal except within tau of the threshold
    Lx, Ly, B, C, T, burn = 4, 4, 3, 45, 2, 1
    ctx, model, _ = make(Lx, Ly, B, 41, h=1.0, dtype=dtype)
    N = Lx * Ly
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=12)
    s0 = unpack_np(words_from_tensor(state), N)
    samples = torch.zeros(((T - burn) * C, ctx.W), dtype=torch.int32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    bits = torch.zeros((C, T, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, burn, 31, 0, samples, None, nacc, accept_bits=bits)
    torch.cuda.synchronize()
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    lpf = lambda v: copy_logpsi(model, v, dtype)
    ref = mh_sweeps(lpf, s0, np.arange(C), 31, T, burn, replay_accepts=acc, tau=4 * flip_tol(dtype, N))
    np.testing.assert_array_equal(unpack_np(words_from_tensor(state), N), ref["spins"])
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), N), ref["samples"])
    np.testing.assert_array_equal(nacc.cpu().numpy(), acc.sum(axis=(1, 2)))


def test_bf16_sampler_targets_its_copy_and_the_bias_is_bounded():
    # 4 x 3: the BF16 sampler's histogram matches |psi_bf16|^2 at the i.i.d. noise floor, and the
    # exact TV(pi, pi_bf16) is below min(Pinsker, Thm 3) from the copy's single-flip increments
    Lx, Ly, B = 4, 3, 2
    ctx, model, ham = make(Lx, Ly, B, 77, h=1.0, dtype="bf16")
    N = Lx * Ly
    S = exact.all_configs(N)
    lp_copy = copy_logpsi(model, S, "bf16")
    pi_c = np.exp(2 * (lp_copy - lp_copy.max()))
    pi_c /= pi_c.sum()
    pi = exact.exact_pi(model.logpsi, N)
    C, T, burn = 8192, 30, 10
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=19)
    samples = torch.zeros(((T - burn) * C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, burn, 321, 0, samples, None, None)
    idx = exact.config_index(unpack_np(words_from_tensor(samples[-C:]), N))
    hist = np.bincount(idx, minlength=pi.size) / C
    tv = 0.5 * np.abs(hist - pi_c).sum()
    floor = np.mean([0.5 * np.abs(np.bincount(np.random.default_rng(k).choice(pi.size, C, p=pi_c),
                                              minlength=pi.size) / C - pi_c).sum() for k in range(4)])
    assert tv < 1.2 * floor + 0.01, (tv, floor)
    # the distance the BF16 copy puts between the sampled and the exact distribution obeys
    # Pinsker with the exact KL; the Gaussian reading of Sec. 3 (sigma from the single-flip
    # increments) gives a bound of the same size
    from oracle import bounds
    tv_exact = bounds.tv_distance(pi, pi_c)
    kl = np.sum(pi * np.log(pi / pi_c))
    assert tv_exact <= np.sqrt(kl / 2)
    delta = 2 * (lp_copy - model.logpsi(S))           # log p~ - log p, up to a constant
    x = np.arange(S.shape[0])
    eps = np.concatenate([delta[x ^ (1 << i)] - delta for i in range(N)])
    assert 0.25 < tv_exact / bounds.reported_bound(eps.mean(), eps.std()) < 4.0
