"""Parity of the CUDA RBM / TFIM path with the FP64 oracle (run on a B300).

Bit-exact: initial spins, Philox proposal stream (through lockstep replay of the
recorded accept decisions), sample configurations and accept counts.  FP32:
|d log psi| <= 1e-5 relative, decisions may differ from FP64 only within
tau = 1e-4 of the threshold (|2 dlogpsi - log u| <= tau).
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, unpack_np, unpack_accept_bits, to_words_tensor, words_from_tensor
from oracle import exact
from oracle.estimators import local_energy as oracle_eloc, energy_stats, force as oracle_force
from oracle.hamiltonian import TFIM
from oracle.models import RBM
from oracle.philox import init_spins_random
from oracle.sampler import mh_sweeps
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TAU = 1e-4
LOGPSI_RTOL = 1e-5


def make(Lx, Ly, M, sigma, seed, h=1.0, J=1.0):
    p = nqs()
    ctx = p.Context("tfim", Lx, Ly, J1=J, h=h, model="rbm", n_hidden=M, dtype="f32")
    params = rbm_params(Lx * Ly, M, sigma, seed)
    ctx.set_params(torch.from_numpy(params).cuda())
    return ctx, RBM(Lx * Ly, M, params), TFIM(Lx, Ly, J, h)


@pytest.mark.parametrize("N,C", [(16, 1000), (37, 333), (100, 64), (256, 17)])
def test_init_chains_bit_exact(N, C):
    p = nqs()
    ctx = p.Context("tfim", N, 1, h=1.0, model="rbm", n_hidden=8)
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=123456789)
    got = unpack_np(words_from_tensor(state), N)
    np.testing.assert_array_equal(got, init_spins_random(123456789, np.arange(C), N))
    # unused high bits of the last word stay clear
    if N % 32:
        assert np.all(words_from_tensor(state)[:, -1] >> np.uint32(N % 32) == 0)


@pytest.mark.parametrize("Lx,Ly,M,sigma", [(16, 1, 16, 0.3), (37, 1, 50, 0.2), (10, 10, 400, 0.05),
                                           (16, 16, 100, 0.1)])
def test_logpsi_fp32_matches_oracle(Lx, Ly, M, sigma):
    ctx, model, _ = make(Lx, Ly, M, sigma, 7)
    s = np.random.default_rng(1).choice([-1, 1], size=(517, Lx * Ly)).astype(np.int8)
    out = torch.empty(517, dtype=torch.float32, device="cuda")
    ctx.logpsi(to_words_tensor(pack_np(s)), out)
    ref = model.logpsi(s)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=LOGPSI_RTOL, atol=LOGPSI_RTOL)


def _lockstep(Lx, Ly, M, sigma, C, T, burn, seed=99, offset=0, refresh=None, cpw=None):
    ctx, model, _ = make(Lx, Ly, M, sigma, 5)
    N = Lx * Ly
    if refresh:
        ctx.set_option(nqs().OPT_REFRESH, refresh)
    if cpw is not None:
        ctx.set_option(nqs().OPT_CHAINS_PER_WARP, cpw)
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, seed=seed + 1)
    s0 = unpack_np(words_from_tensor(state), N)
    K = T - burn
    samples = torch.zeros((K * C, ctx.W), dtype=torch.int32, device="cuda")
    logpsi = torch.zeros(K * C, dtype=torch.float32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    bits = torch.zeros((C, T, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, burn, seed, offset, samples, logpsi, nacc, accept_bits=bits)
    torch.cuda.synchronize()
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    ref = mh_sweeps(model.logpsi, s0, np.arange(C), seed, T, burn, sweep_offset=offset,
                    replay_accepts=acc, tau=TAU)
    return ctx, model, ref, state, samples, logpsi, nacc, acc


@pytest.mark.parametrize("Lx,Ly,M,sigma,C,T,burn,cpw", [
    (16, 1, 16, 0.01, 1024, 100, 10, None),    # the 1D N = 16 workload, in full
    (16, 1, 16, 0.3, 300, 12, 2, 1),           # one chain per warp, ragged chain count
    (37, 1, 50, 0.25, 301, 7, 3, None),        # ragged N (two words), padded hidden units
    (10, 10, 400, 0.05, 64, 3, 1, None),       # the 10 x 10, alpha = 4 shape
    (10, 10, 400, 0.05, 70, 3, 1, 2),          # same, two chains per warp (16 lanes each)
    (12, 1, 40, 0.3, 99, 5, 1, 2),             # two chains per warp, E = 4 per lane, ragged chains
])
def test_sweep_lockstep_with_oracle(Lx, Ly, M, sigma, C, T, burn, cpw):
    _, model, ref, state, samples, logpsi, nacc, acc = _lockstep(Lx, Ly, M, sigma, C, T, burn, cpw=cpw)
    N = Lx * Ly
    # replay succeeded (no decision outside tau disagreed); configurations are then identical
    np.testing.assert_array_equal(unpack_np(words_from_tensor(state), N), ref["spins"])
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), N), ref["samples"])
    np.testing.assert_array_equal(nacc.cpu().numpy(), acc.sum(axis=(1, 2)))
    lp = logpsi.cpu().numpy()
    np.testing.assert_allclose(lp, ref["logpsi"], rtol=LOGPSI_RTOL, atol=LOGPSI_RTOL)
    assert ref["near_threshold"] <= max(2, 1e-5 * ref["checked"])


def test_sweep_resumes_across_calls():
    p = nqs()
    ctx, _, _ = make(12, 1, 24, 0.3, 3)
    C = 200
    a = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(a, 5)
    b = a.clone()
    ctx.sweep(a, 6, 0, 77, 0)
    ctx.sweep(b, 2, 0, 77, 0)
    ctx.sweep(b, 4, 0, 77, 2)
    # the cache is rebuilt at a call boundary; decisions still agree except within FP32 rounding
    assert (a != b).any(dim=1).float().mean().item() <= 0.01


def test_local_energy_matches_oracle():
    ctx, model, ham = make(10, 10, 400, 0.05, 9, h=3.04)
    s = np.random.default_rng(2).choice([-1, 1], size=(300, 100)).astype(np.int8)
    e = torch.empty(300, dtype=torch.float32, device="cuda")
    ctx.local_energy(to_words_tensor(pack_np(s)), e)
    ref = oracle_eloc(ham, model.logpsi, s)
    np.testing.assert_allclose(e.cpu().numpy(), ref, rtol=1e-5, atol=1e-5 * len(ham.bonds) * abs(ham.J))


def test_local_energy_ragged_and_1d():
    ctx, model, ham = make(37, 1, 50, 0.3, 4, h=0.7, J=1.3)
    s = np.random.default_rng(3).choice([-1, 1], size=(65, 37)).astype(np.int8)
    e = torch.empty(65, dtype=torch.float32, device="cuda")
    ctx.local_energy(to_words_tensor(pack_np(s)), e)
    ref = oracle_eloc(ham, model.logpsi, s)
    # FP32 sum of N ratios: error relative to the size of the off-diagonal sum
    np.testing.assert_allclose(e.cpu().numpy(), ref, rtol=1e-5, atol=1e-5 * 37 * 1.3)


@pytest.mark.parametrize("Lx,Ly,M", [(16, 1, 16), (10, 10, 400), (7, 1, 33)])
def test_logpsi_grad_rows_and_force_match_oracle(Lx, Ly, M):
    N = Lx * Ly
    ctx, model, _ = make(Lx, Ly, M, 0.1, 8)
    n = 203
    s = np.random.default_rng(4).choice([-1, 1], size=(n, N)).astype(np.int8)
    cfg = to_words_tensor(pack_np(s))
    O = torch.empty((n, ctx.P), dtype=torch.float32, device="cuda")
    eloc = torch.from_numpy(np.random.default_rng(5).normal(-3.0, 1.0, n).astype(np.float32)).cuda()
    stats = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(eloc, n, stats)
    force = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctx.logpsi_grad_workspace(n), dtype=torch.uint8, device="cuda")
    ctx.logpsi_grad(cfg, O=O, eloc=eloc, stats=stats, force=force, workspace=ws)
    Oref = model.grad(s)
    np.testing.assert_allclose(O.cpu().numpy(), Oref, rtol=0, atol=1e-5)
    Fref = oracle_force(Oref, eloc.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(force.cpu().numpy(), Fref, rtol=0, atol=1e-5 * max(1.0, np.abs(Fref).max()))


def _oracle_force_blocked(model, s, eps, block=50000):
    """F = mean(O (eps - E)) of the RBM without materialising O (same definition, blocked)."""
    e = eps - eps.mean()
    Fa = np.zeros(model.N); Fb = np.zeros(model.M); FW = np.zeros((model.M, model.N))
    for b0 in range(0, len(s), block):
        sb = s[b0:b0 + block].astype(np.float64)
        eb = e[b0:b0 + block]
        t = np.tanh(model.theta(sb))
        Fa += sb.T @ eb
        Fb += t.T @ eb
        FW += (t * eb[:, None]).T @ sb
    n = len(s)
    return np.concatenate([Fa / n, Fb / n, (FW / n).ravel()])


@pytest.mark.parametrize("n", [600_000, 98_700])
def test_force_many_tiles_matches_oracle(n):
    """Many rows of the 10x10 alpha = 4 shape.  600k: every block accumulates 224 tiles (14
    FP32 periods drained to FP64, both accumulator pairs reused); 98,700: 37 tiles per block,
    an odd count that ends in a partial period and a ragged tile."""
    ctx, model, _ = make(10, 10, 400, 0.05, 17)
    rng = np.random.default_rng(18)
    s = rng.choice([-1, 1], size=(n, 100)).astype(np.int8)
    eps = rng.normal(-310.0, 5.0, n).astype(np.float32)
    cfg = to_words_tensor(pack_np(s))
    eloc = torch.from_numpy(eps).cuda()
    stats = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(eloc, n, stats)
    force = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctx.logpsi_grad_workspace(n), dtype=torch.uint8, device="cuda")
    ctx.logpsi_grad(cfg, None, eloc, stats, force, ws)
    ref = _oracle_force_blocked(model, s, eps.astype(np.float64))
    got = force.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_stats_match_oracle_and_acceptance():
    p = nqs()
    ctx, _, _ = make(16, 1, 16, 0.1, 1)
    C, K = 96, 7
    e = np.random.default_rng(6).normal(-20, 2, C * K).astype(np.float32)
    acc = torch.arange(C, dtype=torch.int64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(torch.from_numpy(e).cuda(), C, out, n_accepted=acc, proposals_per_chain=160)
    E, var, err = energy_stats(e.astype(np.float64), C)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[:3], [E, var, err], rtol=1e-12)
    assert got[3] == pytest.approx(np.arange(C).sum() / (C * 160))
    assert got[4] == C * K


def test_tfim_1d_n16_energy_against_exact_enumeration_and_ed():
    """1D TFIM N = 16, J = h = 1, RBM alpha = 1 with N(0, 0.01^2) weights, 1024 chains x
    100 sweeps (10 burn-in): the sampled energy agrees with the exact expectation by
    enumeration within 3 standard errors and lies above the ED ground energy."""
    p = nqs()
    ctx, model, ham = make(16, 1, 16, 0.01, 20260001)
    C, T, B = 1024, 100, 10
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 11)
    S = torch.zeros(((T - B) * C, 1), dtype=torch.int32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    ctx.sweep(state, T, B, 12, 0, S, None, nacc)
    e = torch.empty((T - B) * C, dtype=torch.float32, device="cuda")
    ctx.local_energy(S, e)
    st = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(e, C, st, nacc, T * 16)
    E, var, err, accr, n = st.cpu().numpy()
    pi = exact.exact_pi(model.logpsi, 16)
    e_exact = pi @ oracle_eloc(ham, model.logpsi, exact.all_configs(16))
    assert abs(E - e_exact) < 3 * err, (E, e_exact, err)
    e0 = exact.ground_energy(exact.sparse_hamiltonian(ham))[0]
    assert E > e0
    assert 0.0 < accr <= 1.0


def test_histogram_tv_against_exact_distribution_4x4():
    """4 x 4 TFIM, alpha = 4 RBM: the final configurations of 32768 independent chains
    after 200 sweeps are compared with the exact pi (enumeration of 2^16 states).  Their
    total-variation distance must be at the level of i.i.d. draws of the same count
    (successive sweeps of one chain are correlated, so only one sample per chain is used)."""
    ctx, model, _ = make(4, 4, 64, 0.25, 13, h=3.04)
    C, T = 32768, 200
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 21)
    ctx.sweep(state, T, T, 22, 0)
    idx = words_from_tensor(state)[:, 0].astype(np.int64)
    hist = np.bincount(idx, minlength=2 ** 16) / idx.size
    pi = exact.exact_pi(model.logpsi, 16)
    tv = 0.5 * np.abs(hist - pi).sum()
    rng = np.random.default_rng(0)
    floors = [0.5 * np.abs(np.bincount(rng.choice(pi.size, C, p=pi), minlength=pi.size) / C - pi).sum()
              for _ in range(8)]
    assert tv < max(floors) * 1.15, (tv, floors)


@pytest.mark.parametrize("Lx,Ly,M,dtype,refresh", [(10, 10, 400, "f16", 20), (10, 10, 400, "f32", 7),
                                                   (16, 1, 16, "f32", 20), (37, 1, 50, "f32", 20)])
def test_local_energy_chains_matches_per_sample(Lx, Ly, M, dtype, refresh):
    """Chain-ordered local energies (incremental theta over each chain's sweep-major samples,
    taken two at a time, rebuilt every `refresh` samples: an odd interval rebuilds at the
    second sample of a pair; 45 samples leave a last pair of one) equal the per-sample
    evaluation up to FP32 rounding."""
    p = nqs()
    N = Lx * Ly
    ctx = p.Context("tfim", Lx, Ly, J1=1.0, h=2.0, model="rbm", n_hidden=M, dtype=dtype)
    ctx.set_option(p.OPT_REFRESH, refresh)
    ctx.set_params(torch.from_numpy(rbm_params(N, M, 0.1, 3)).cuda())
    C, K = 2500, 45                      # >= 16 chains per SM: the chain-ordered kernel runs
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 4)
    samples = torch.zeros((K * C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(state, K, 0, 5, 0, samples)
    e1 = torch.empty(K * C, dtype=torch.float32, device="cuda")
    e2 = torch.empty(K * C, dtype=torch.float32, device="cuda")
    ctx.local_energy(samples, e1)
    ctx.local_energy_chains(samples, C, e2)
    a, b = e1.cpu().numpy().astype(np.float64), e2.cpu().numpy().astype(np.float64)
    rel = np.abs(b - a) / (np.abs(a) + 2.0 * N)
    assert rel.max() <= 2e-5, (rel.max(), np.argmax(rel), a[np.argmax(rel)], b[np.argmax(rel)])


@pytest.mark.parametrize("model_kind", ["rbm", "dense"])
def test_moments_and_force_shares_of_split_chains(model_kind):
    # A multi-rank step on one GPU: the chains split into two "ranks" of unequal size.  Each
    # rank's moments (nqs_stats_moments), summed, give through nqs_stats_finalize the pooled
    # statistics, which equal the oracle's on all chains; each rank's force share
    # (nqs_force_share, centred on the pooled E and divided by the pooled count) sums to the
    # pooled force of the oracle.  With one rank the two calls equal nqs_stats and the share
    # equals nqs_logpsi_grad's force.
    p = nqs()
    rng = np.random.default_rng(61)
    if model_kind == "rbm":
        Lx, Ly, M = 6, 6, 72
        ctx, model, _ = make(Lx, Ly, M, 0.1, 62)
    else:
        from oracle.models import Dense
        from workloads import dense_params
        Lx, Ly, widths = 4, 4, (64, 48)
        params = dense_params(16, widths, 63, bias_sigma=0.1)
        ctx = p.Context("heisenberg", Lx, Ly, J1=1.0, marshall=True, model="dense", widths=widths, dtype="bf16")
        ctx.set_params(torch.from_numpy(params).cuda())
        model = Dense(16, widths, params)
    N, K, Cs = Lx * Ly, 5, (37, 91)
    parts = []
    for C in Cs:
        s = rng.choice([-1, 1], size=(K * C, N)).astype(np.int8)
        e = rng.normal(-10.0, 3.0, size=K * C).astype(np.float32)
        acc = rng.integers(0, 50, size=C)
        parts.append((s, e, acc, C))
    mom = []
    for s, e, acc, C in parts:
        m = torch.zeros(8, dtype=torch.float64, device="cuda")
        ctx.stats_moments(torch.from_numpy(e).cuda(), C, m, torch.from_numpy(acc).cuda(), 50)
        mom.append(m)
    total = mom[0] + mom[1]          # the all-reduce SUM
    stats = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.stats_finalize(total, stats)
    shares = []
    for s, e, acc, C in parts:
        f = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
        ws = torch.empty(max(ctx.logpsi_grad_workspace(len(e)), 1), dtype=torch.uint8, device="cuda")
        ctx.force_share(to_words_tensor(pack_np(s)), torch.from_numpy(e).cuda(), stats, f, ws)
        shares.append(f)
    force = (shares[0] + shares[1]).cpu().numpy()
    torch.cuda.synchronize()
    # pooled oracle: chains side by side, sweep-major
    eps = np.concatenate([e.astype(np.float64).reshape(K, C) for s, e, acc, C in parts], axis=1).reshape(-1)
    S = np.concatenate([s.reshape(K, C, N) for s, e, acc, C in parts], axis=1).reshape(-1, N)
    E, var, err = energy_stats(eps, sum(Cs))
    acc_rate = sum(a.sum() for _, _, a, _ in parts) / (sum(Cs) * 50)
    np.testing.assert_allclose(stats.cpu().numpy(), [E, var, err, acc_rate, eps.size], rtol=1e-12)
    F = oracle_force(model.grad(S), eps)
    tol = 1e-5 if model_kind == "rbm" else 1e-4      # as the other RBM / dense force tests
    np.testing.assert_allclose(force, F, rtol=0, atol=tol * np.abs(F).max())
    # one rank: the two calls equal nqs_stats, and the share equals nqs_logpsi_grad's force
    s, e, acc, C = parts[1]
    e_t, acc_t = torch.from_numpy(e).cuda(), torch.from_numpy(acc).cuda()
    one = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.stats(e_t, C, one, acc_t, 50)
    fin = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.stats_finalize(mom[1], fin)
    assert torch.equal(one, fin)
    ref = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(ctx.logpsi_grad_workspace(len(e)), 1), dtype=torch.uint8, device="cuda")
    ctx.logpsi_grad(to_words_tensor(pack_np(s)), None, e_t, one, ref, ws)
    sh = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    ctx.force_share(to_words_tensor(pack_np(s)), e_t, one, sh, ws)
    assert torch.equal(ref, sh)
