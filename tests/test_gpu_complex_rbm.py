"""GPU parity of the complex-parameter RBM (App. G with complex a, b, W) against the FP64
oracle ``oracle.complex_rbm``:

* log psi (real part, imaginary part modulo 2 pi) on several lattices and hidden widths;
* complex TFIM local energies (App. I, Eq. local_energies), ragged sample counts, with the
  relative tolerance widened by u / min_j |cosh theta_j|^2 near zeros of psi;
* the |psi|^2 sampler replayed decision by decision in the oracle (decisions outside a
  10-sigma window of the FP32 increment agree with the FP64 rule, final chains and kept
  samples identical), traced equal to untraced, refresh every sweep equal in law;
* O rows and the conjugate force (App. I, Eq. forces) over several unit tiles and row blocks,
  at the workload's shape with a ragged row count, for one row, and beyond the tensor-core
  path's site limit;
* the FP64 statistics, including the mean of Im eps;
* the sampled energy of a small chain against the exact Rayleigh quotient;
* range checks and the empty cases.
The FP32 tolerances follow from unit roundoff 2^-24 times the number of terms summed.
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, unpack_np, unpack_accept_bits, to_words_tensor, words_from_tensor
from oracle import exact
from oracle.complex_rbm import ComplexRBM, local_energy_tfim, force as oracle_force
from oracle.estimators import energy_stats
from oracle.hamiltonian import TFIM
from oracle.sampler import mh_sweeps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def cparams(N, M, sigma, seed):
    rng = np.random.default_rng(seed)
    n = N + M + N * M
    return rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)


def make(Lx, Ly, M, sigma, seed, J=1.0, h=0.8):
    p = nqs()
    c = p.ComplexContext(Lx, Ly, J1=J, h=h, n_hidden=M)
    params = cparams(Lx * Ly, M, sigma, seed)
    c.set_params(torch.from_numpy(params).cuda())
    return c, params, ComplexRBM(Lx * Ly, M, params), TFIM(Lx, Ly, J, h)


def rand_configs(n, N, seed):
    return np.random.default_rng(seed).choice([-1, 1], size=(n, N)).astype(np.int8)


SHAPES = [(10, 1, 7, 0.3), (4, 4, 40, 0.2), (6, 6, 144, 0.08), (10, 10, 400, 0.04), (16, 16, 512, 0.02)]


@pytest.mark.parametrize("Lx,Ly,M,sigma", SHAPES)
def test_logpsi_matches_oracle(Lx, Ly, M, sigma):
    c, _, model, _ = make(Lx, Ly, M, sigma, 1)
    N = Lx * Ly
    s = rand_configs(67, N, 2)
    out = torch.zeros(67, dtype=torch.complex64, device="cuda")
    c.logpsi(to_words_tensor(pack_np(s)), out)
    got = out.cpu().numpy().astype(np.complex128)
    ref = model.logpsi(s)
    tol = 2e-6 * (N + M) + 1e-5
    np.testing.assert_allclose(got.real, ref.real, rtol=1e-5, atol=tol)
    dphi = np.angle(np.exp(1j * (got.imag - ref.imag)))
    assert np.abs(dphi).max() < tol


@pytest.mark.parametrize("Lx,Ly,M,sigma", SHAPES[:4])
@pytest.mark.parametrize("n", [1, 37, 130])
def test_local_energy_matches_oracle(Lx, Ly, M, sigma, n):
    c, _, model, ham = make(Lx, Ly, M, sigma, 3, h=-0.9)
    N = Lx * Ly
    s = rand_configs(n, N, 4)
    re = torch.zeros(n, dtype=torch.float32, device="cuda")
    im = torch.zeros_like(re)
    c.local_energy(to_words_tensor(pack_np(s)), re, im)
    got = re.cpu().numpy().astype(np.float64) + 1j * im.cpu().numpy().astype(np.float64)
    ref = local_energy_tfim(ham, model, s)
    scale = len(ham.bonds) + N * abs(ham.h)
    # near a zero of psi (some |cosh theta_j| small) tanh theta_j sits near a pole and FP32
    # loses about u / |cosh theta_j|^2 of relative accuracy: the tolerance carries that factor
    kappa = (1.0 / np.abs(np.cosh(model.theta(s))) ** 2).max(axis=1)
    rtol = 1e-4 + 8 * 2.0 ** -24 * kappa
    bad = np.abs(got - ref) > rtol * np.abs(ref) + 2e-5 * scale
    assert not bad.any(), (np.flatnonzero(bad), got[bad], ref[bad], kappa[bad])


@pytest.mark.parametrize("C,refresh", [(4096, 5), (4096, 20), (100, 5)])
def test_local_energy_chains_matches_per_sample(C, refresh):
    """nqs_crbm_local_energy_chains on the sweep-major samples of nqs_crbm_sweep (10 x 10,
    M = 400): the chain-ordered theta updates (rebuilt every `refresh` samples, inside and
    across the warp's blocks of four; 11 samples per chain, a ragged last block) give the
    per-sample values to FP32 rounding, with the same pole widening as against the oracle; a
    subset is also held to the oracle.  100 chains (fewer than 16 per SM) take the per-sample
    path and match it exactly."""
    c, _, model, ham = make(10, 10, 400, 0.04, 21, h=-0.9)
    c.set_refresh(refresh)
    N, W, T, B = 100, 4, 12, 1
    st = torch.zeros((C, W), dtype=torch.int32, device="cuda")
    c.init_chains(st, 31)
    samples = torch.zeros(((T - B) * C, W), dtype=torch.int32, device="cuda")
    c.sweep(st, T, B, 32, 0, samples)
    n = samples.shape[0]
    re1, im1 = torch.zeros(n, dtype=torch.float32, device="cuda"), torch.zeros(n, dtype=torch.float32, device="cuda")
    re2, im2 = torch.zeros_like(re1), torch.zeros_like(re1)
    c.local_energy(samples, re1, im1)
    c.local_energy_chains(samples, C, re2, im2)
    c.check_status()
    if C < 2368:
        assert torch.equal(re1, re2) and torch.equal(im1, im2)
        return
    a = re1.cpu().numpy().astype(np.float64) + 1j * im1.cpu().numpy().astype(np.float64)
    b = re2.cpu().numpy().astype(np.float64) + 1j * im2.cpu().numpy().astype(np.float64)
    s = unpack_np(words_from_tensor(samples), N)
    kappa = (1.0 / np.abs(np.cosh(model.theta(s))) ** 2).max(axis=1)
    scale = len(ham.bonds) + N * abs(ham.h)
    rtol = 1e-4 + 8 * 2.0 ** -24 * kappa
    bad = np.abs(a - b) > rtol * np.abs(a) + 2e-5 * scale
    assert not bad.any(), (np.flatnonzero(bad)[:8], a[bad][:8], b[bad][:8])
    assert np.abs(a - b).max() > 0 or refresh == 1   # the incremental path ran (not the per-sample one)
    sub = np.random.default_rng(3).choice(n, 64, replace=False)
    ref = local_energy_tfim(ham, model, s[sub])
    bad = np.abs(b[sub] - ref) > rtol[sub] * np.abs(ref) + 2e-5 * scale
    assert not bad.any(), (sub[bad], b[sub][bad], ref[bad])


@pytest.mark.parametrize("refresh,sigma,strict", [(1, 0.3, True), (20, 0.1, True), (20, 0.3, False)])
def test_sweep_replays_in_the_oracle(refresh, sigma, strict):
    Lx, Ly, M = 4, 4, 24
    c, _, model, _ = make(Lx, Ly, M, sigma, 5)
    c.set_refresh(refresh)
    N, W, C, T, B, seed = Lx * Ly, 1, 96, 7, 2, 77
    z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device="cuda")
    st = z(C, W)
    c.init_chains(st, 9)
    s0 = unpack_np(words_from_tensor(st), N)
    st_t, samp_t, nacc_t, bits, delta = st.clone(), z((T - B) * C, W), z(C, dt=torch.int64), z(C, T, W), \
        z(C, T, N, dt=torch.float32)
    c.sweep(st_t, T, B, seed, 3, samp_t, nacc_t, accept_bits=bits, delta=delta)
    st_u, samp_u, nacc_u = st.clone(), z((T - B) * C, W), z(C, dt=torch.int64)
    c.sweep(st_u, T, B, seed, 3, samp_u, nacc_u)
    torch.cuda.synchronize()
    assert torch.equal(st_t, st_u) and torch.equal(samp_t, samp_u) and torch.equal(nacc_t, nacc_u)
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    d = delta.cpu().numpy().astype(np.float64)
    ref = mh_sweeps(model.log_density, s0, np.arange(C), seed, T, B, sweep_offset=3, replay_accepts=acc,
                    tau=1.0, record_deltas=True)
    # below 2 Re delta = -17 every u >= 2^-24 rejects: there only the decision is compared
    # (FP32 cannot resolve |cosh theta'| near its zeros, where delta runs to -infinity)
    live = 2.0 * ref["deltas"] > -17.0
    err = (d - ref["deltas"])[live]
    # K cache updates since the last rebuild leave sinh x with an absolute error ~ K u cosh x,
    # so log D_j errs by ~ K u / sqrt(D_j): near u times the unit count while theta stays away
    # from the zeros of cosh (small weights, or a rebuild every sweep); with large weights a
    # unit near a zero carries more until the next rebuild, and only the decisions are exact
    sig = (2.0 * err).std()
    assert np.abs(err).max() < (1e-4 if strict else 1e-2), np.abs(err).max()
    assert np.all(2.0 * d[~live] < -15.0)
    r2 = mh_sweeps(model.log_density, s0, np.arange(C), seed, T, B, sweep_offset=3, replay_accepts=acc,
                   tau=max(10 * sig, 1e-6))
    np.testing.assert_array_equal(r2["spins"], unpack_np(words_from_tensor(st_t), N))
    np.testing.assert_array_equal(r2["samples"], unpack_np(words_from_tensor(samp_t), N))
    np.testing.assert_array_equal(r2["n_accepted"], nacc_t.cpu().numpy())
    assert 0.05 < acc.mean() < 0.95


def test_sampled_energy_matches_exact_rayleigh_quotient():
    Lx, M = 8, 10
    c, _, model, ham = make(Lx, 1, M, 0.3, 11, J=1.0, h=-1.0)
    N, C, T, B = Lx, 2048, 120, 20
    z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device="cuda")
    st, samples, nacc = z(C, 1), z((T - B) * C, 1), z(C, dt=torch.int64)
    c.init_chains(st, 3)
    c.sweep(st, T, B, 21, 0, samples, nacc)
    n = (T - B) * C
    re, im = z(n, dt=torch.float32), z(n, dt=torch.float32)
    c.local_energy(samples, re, im)
    stats = z(6, dt=torch.float64)
    c.stats(re, im, C, stats, nacc, T * N)
    torch.cuda.synchronize()
    E, var, err, accr = stats.cpu().numpy()[:4]
    S = exact.all_configs(N)
    lp = model.logpsi(S)
    psi = np.exp(lp - lp.real.max())
    H = exact.sparse_hamiltonian(ham)
    E_ex = ((np.conj(psi) @ (H @ psi)) / (np.conj(psi) @ psi)).real
    assert abs(E - E_ex) < 5 * err + 1e-6, (E, E_ex, err)
    assert 0.0 < accr < 1.0


def test_O_rows_and_force_match_oracle():
    Lx, Ly, M = 6, 6, 144
    c, _, model, ham = make(Lx, Ly, M, 0.08, 13)
    N, n = Lx * Ly, 2000
    s = rand_configs(n, N, 6)
    cfg = to_words_tensor(pack_np(s))
    re = torch.zeros(n, dtype=torch.float32, device="cuda")
    im = torch.zeros_like(re)
    c.local_energy(cfg, re, im)
    stats = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.stats(re, im, 1, stats)
    O = torch.zeros(n, c.P, dtype=torch.complex64, device="cuda")
    F = torch.zeros(c.P, dtype=torch.complex128, device="cuda")
    c.logpsi_grad(cfg, O, re, im, stats, F)
    torch.cuda.synchronize()
    eps = re.cpu().numpy().astype(np.float64) + 1j * im.cpu().numpy().astype(np.float64)
    st = stats.cpu().numpy()
    np.testing.assert_allclose(st[0], eps.real.mean(), rtol=1e-12)
    np.testing.assert_allclose(st[5], eps.imag.mean(), rtol=1e-12, atol=1e-14)
    Oref = model.grad(s)
    # an FP32 error of theta reaches tanh theta multiplied by |1 - tanh^2 theta|
    Og = O.cpu().numpy()
    bad = np.abs(Og - Oref) > 1e-5 * (1.0 + np.abs(Oref) ** 2)
    assert not bad.any(), (np.argwhere(bad)[:5], Og[bad][:5], Oref[bad][:5])
    Fref = oracle_force(Oref, eps)
    Fg = F.cpu().numpy()
    np.testing.assert_allclose(Fg, Fref, rtol=0, atol=2e-5 * np.abs(Fref).max())
    # the force alone (no O rows) is the same computation
    F2 = torch.zeros_like(F)
    c.logpsi_grad(cfg, None, re, im, stats, F2)
    torch.cuda.synchronize()
    # the row chunks' partials are added in a fixed order: the same inputs give the same bits
    assert torch.equal(F2, F)


def _cforce_blocked(model, s, eps, block=20000):
    """F = mean(conj(O) (eps - E)) over all rows, block by block: O_a = s, O_b = tanh theta,
    O_W[j][i] = tanh(theta_j) s_i (the oracle's force without materialising the O rows)."""
    e = eps - eps.mean()
    Fa = np.zeros(model.N, complex); Fb = np.zeros(model.M, complex); FW = np.zeros((model.M, model.N), complex)
    for b0 in range(0, len(eps), block):
        sb = s[b0:b0 + block].astype(np.float64)
        eb = e[b0:b0 + block]
        ct = np.conj(np.tanh(model.theta(sb)))
        Fa += sb.T @ eb
        Fb += ct.T @ eb
        FW += (ct * eb[:, None]).T @ sb
    n = len(eps)
    return np.concatenate([Fa / n, Fb / n, (FW / n).ravel()])


@pytest.mark.parametrize("Lx,Ly,M,sigma,n", [(10, 10, 400, 0.04, 40077), (4, 4, 40, 0.2, 1), (16, 8, 32, 0.02, 3001)])
def test_force_at_workload_shape_and_edges(Lx, Ly, M, sigma, n):
    """The force over ragged row counts: the workload's 10 x 10, M = 400 shape (tensor-core
    path: 13 unit tiles of 32, the last holding the a-entries; 313 full row tiles and a tail
    of 13 rows), a single row, and N = 128 (beyond the tensor-core path's K, the CUDA-core path),
    against the oracle's force accumulated block by block.  An FP32 rounding of theta reaches
    tanh theta amplified by |1 - tanh^2 theta|, which is large near the poles at Im theta =
    pi/2; the weights keep the std of Im theta at or below 0.4 so that few samples come near one
    (at N = 128, std 0.05 put Im theta within reach of pi/2 and gave 1e-4 relative errors on
    the CUDA-core path)."""
    c, _, model, _ = make(Lx, Ly, M, sigma, 29)
    N = Lx * Ly
    s = rand_configs(n, N, 31)
    cfg = to_words_tensor(pack_np(s))
    re = torch.zeros(n, dtype=torch.float32, device="cuda")
    im = torch.zeros_like(re)
    c.local_energy(cfg, re, im)
    stats = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.stats(re, im, 1, stats)
    F = torch.zeros(c.P, dtype=torch.complex128, device="cuda")
    c.logpsi_grad(cfg, None, re, im, stats, F)
    torch.cuda.synchronize()
    eps = re.cpu().numpy().astype(np.float64) + 1j * im.cpu().numpy().astype(np.float64)
    Fref = _cforce_blocked(model, s, eps)
    Fg = F.cpu().numpy()
    scale = max(np.abs(Fref).max(), 1e-12 * np.abs(eps).max())
    np.testing.assert_allclose(Fg, Fref, rtol=0, atol=2e-5 * scale)


def test_stats_match_oracle_statistics():
    c, _, _, _ = make(4, 4, 16, 0.2, 17)
    rng = np.random.default_rng(8)
    C, K = 64, 9
    er = rng.normal(-3.0, 0.5, K * C).astype(np.float32)
    ei = rng.normal(0.01, 0.2, K * C).astype(np.float32)
    nacc = rng.integers(0, 100, C)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.stats(torch.from_numpy(er).cuda(), torch.from_numpy(ei).cuda(), C, out,
            torch.from_numpy(nacc).cuda(), 100)
    got = out.cpu().numpy()
    E, var, err = energy_stats(er.astype(np.float64), C)
    np.testing.assert_allclose(got[:3], [E, var, err], rtol=1e-12)
    assert got[3] == pytest.approx(nacc.sum() / (C * 100), rel=1e-14)
    assert got[4] == K * C
    assert got[5] == pytest.approx(ei.astype(np.float64).mean(), rel=1e-12)


def test_range_checks_and_empty_calls():
    p = nqs()
    with pytest.raises(p.NQSError) as e:
        p.ComplexContext(17, 16, n_hidden=8)
    assert e.value.code == p.NQS_EUNSUPPORTED
    with pytest.raises(p.NQSError) as e:
        p.ComplexContext(4, 4, n_hidden=513)
    assert e.value.code == p.NQS_EUNSUPPORTED
    c = p.ComplexContext(4, 4, h=1.0, n_hidden=8)
    big = cparams(16, 8, 0.1, 0)
    big[16 + 8 + 3] = 1.5  # |Re W| > 1
    with pytest.raises(p.NQSError) as e:
        c.set_params(torch.from_numpy(big).cuda())
    assert e.value.code == p.NQS_EINVAL
    st = torch.zeros(4, 1, dtype=torch.int32, device="cuda")
    with pytest.raises(p.NQSError):
        c.sweep(st, 2, 0, 1)  # parameters unset after the rejected call
    c.set_params(torch.from_numpy(cparams(16, 8, 0.1, 0)).cuda())
    e0 = torch.zeros(0, 1, dtype=torch.int32, device="cuda")
    f0 = torch.zeros(0, dtype=torch.float32, device="cuda")
    c.local_energy(e0, f0, f0.clone())
    c.sweep(torch.zeros(0, 1, dtype=torch.int32, device="cuda"), 3, 1, 1)
    F = torch.ones(c.P, dtype=torch.complex128, device="cuda")
    c.logpsi_grad(e0, None, f0, f0.clone(), torch.zeros(6, dtype=torch.float64, device="cuda"), F)
    torch.cuda.synchronize()
    assert torch.count_nonzero(F).item() == 0
    c.check_status()
