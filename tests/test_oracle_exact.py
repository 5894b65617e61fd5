"""Pins of the oracle's Hamiltonians, enumeration, ED and local energies.

Each check compares two independent routes or a closed form derived from the
physics, never the oracle against a re-typing of itself.
"""
import numpy as np
import pytest

from oracle import exact
from oracle.estimators import local_energy, energy_stats, force
from oracle.hamiltonian import TFIM, Heisenberg
from oracle.lattice import nn_bonds, nnn_bonds, sublattice_a
from oracle.models import RBM, Dense, marshall_sign
from workloads import rbm_params, dense_params


@pytest.mark.parametrize("N,J,h", [(6, 1.0, 1.0), (8, 1.0, 0.5), (10, 0.7, 1.3), (12, 1.0, 3.04)])
def test_tfim_1d_ed_matches_free_fermions(N, J, h):
    H = exact.sparse_hamiltonian(TFIM(N, 1, J, h))
    e0 = exact.ground_energy(H)[0]
    assert e0 == pytest.approx(exact.tfim_1d_free_fermion_e0(N, J, h), abs=1e-9)


def test_free_fermion_critical_point_identity():
    # at J = h the dispersion is 2|sin(k/2)| and the sum over odd momenta is 1/sin(pi/2N)
    assert exact.tfim_1d_free_fermion_e0(16, 1.0, 1.0) == pytest.approx(-2.0 / np.sin(np.pi / 32), abs=1e-12)
    assert exact.tfim_1d_free_fermion_e0(16, 1.0, 1.0) == pytest.approx(-20.4045944748, abs=1e-9)


def test_tfim_limits():
    # h = 0: Neel order on an even ring, E0 = -J * N; J = 0: E0 = -|h| N
    assert exact.ground_energy(exact.sparse_hamiltonian(TFIM(8, 1, 1.0, 0.0)))[0] == pytest.approx(-8.0)
    assert exact.ground_energy(exact.sparse_hamiltonian(TFIM(8, 1, 0.0, 0.6)))[0] == pytest.approx(-4.8)


def test_heisenberg_four_site_ring_closed_form():
    # sum over the 4 ring bonds of S_i.S_j = S_A.S_B = (S^2 - S_A^2 - S_B^2)/2 -> -2 at S=0, S_A=S_B=1;
    # sigma = 2S, so E0 = -8 J with Pauli matrices.
    H = exact.sparse_hamiltonian(Heisenberg(4, 1, 1.0))
    assert exact.ground_energy(H)[0] == pytest.approx(-8.0, abs=1e-10)


def test_heisenberg_marshall_rotation_preserves_spectrum_and_gs_is_positive():
    sub = sublattice_a(4, 4)
    ham = Heisenberg(4, 4, 1.0)
    H = exact.sparse_hamiltonian(ham)
    Hm = exact.sparse_hamiltonian(ham, sub_a=sub)
    e, em = exact.ground_energy(H, 3), exact.ground_energy(Hm, 3)
    np.testing.assert_allclose(e, em, atol=1e-9)
    # rotated off-diagonals are non-positive -> Perron-Frobenius ground state has one sign
    assert Hm.tocoo().data[Hm.tocoo().row != Hm.tocoo().col].max() <= 0
    # singlet: total S^z = 0
    from scipy.sparse.linalg import eigsh
    _, v = eigsh(Hm, k=1, which="SA")
    sz = exact.all_configs(16).sum(axis=1)
    assert abs(np.sum(v[:, 0] ** 2 * sz)) < 1e-8


def test_bond_counts():
    assert len(nn_bonds(16, 1)) == 16
    assert len(nn_bonds(10, 10)) == 200
    assert len(nnn_bonds(16, 16)) == 512
    b = nn_bonds(5, 4)
    assert len({tuple(sorted(x)) for x in b}) == len(b)


def _rbm(N, M, sigma, seed):
    return RBM(N, M, rbm_params(N, M, sigma, seed))


@pytest.mark.parametrize("kind", ["tfim", "heis"])
def test_local_energy_expectation_equals_rayleigh_quotient(kind):
    N = 8
    model = _rbm(N, 8, 0.3, 1)
    if kind == "tfim":
        ham, sub = TFIM(N, 1, 1.0, 0.8), None
    else:
        ham, sub = Heisenberg(N, 1, 1.0, 0.4), sublattice_a(N, 1)
    S = exact.all_configs(N)
    pi = exact.exact_pi(model.logpsi, N)
    eps = local_energy(ham, model.logpsi, S, sub_a=sub)
    psi = np.exp(model.logpsi(S))
    if sub is not None:
        psi = psi * marshall_sign(S, sub)
    H = exact.sparse_hamiltonian(ham)
    rq = psi @ (H @ psi) / (psi @ psi)
    assert np.sum(pi * eps) == pytest.approx(rq, abs=1e-11)


def test_zero_variance_at_tfim_ground_state():
    N = 8
    ham = TFIM(N, 1, 1.0, -0.9)     # negative field: positive ground state
    H = exact.sparse_hamiltonian(ham)
    from scipy.sparse.linalg import eigsh
    e0, v = eigsh(H, k=1, which="SA")
    g = np.abs(v[:, 0])
    lookup = lambda s: np.log(g[exact.config_index(s)])
    eps = local_energy(ham, lookup, exact.all_configs(N))
    np.testing.assert_allclose(eps, e0[0], atol=1e-8)


def test_zero_variance_at_heisenberg_ground_state_with_marshall_sign():
    N = 8
    sub = sublattice_a(N, 1)
    ham = Heisenberg(N, 1, 1.0)
    Hm = exact.sparse_hamiltonian(ham, sub_a=sub)
    from scipy.sparse.linalg import eigsh
    e0, v = eigsh(Hm, k=1, which="SA")
    g = np.abs(v[:, 0])
    S = exact.all_configs(N)
    sector = S.sum(axis=1) == 0
    lookup = lambda s: np.log(np.maximum(g[exact.config_index(s)], 1e-300))
    eps = local_energy(ham, lookup, S[sector], sub_a=sub)
    np.testing.assert_allclose(eps, e0[0], atol=1e-8)


def test_product_state_closed_forms():
    # W = 0: pi(s) = prod_i exp(2 a_i s_i) / (2 cosh 2 a_i); <s_i> = tanh 2a_i,
    # E = J sum_<ij> tanh 2a_i tanh 2a_j + h sum_i 1 / cosh 2a_i.
    N, M = 6, 4
    p = rbm_params(N, M, 0.4, 3)
    p[N:] = 0.0
    model = RBM(N, M, p)
    a = p[:N]
    S = exact.all_configs(N)
    pi = exact.exact_pi(model.logpsi, N)
    np.testing.assert_allclose(pi @ S, np.tanh(2 * a), atol=1e-13)
    ham = TFIM(N, 1, 1.0, 0.7)
    eps = local_energy(ham, model.logpsi, S)
    t = np.tanh(2 * a)
    expect = sum(t[i] * t[j] for i, j in nn_bonds(N, 1)) + 0.7 * np.sum(1 / np.cosh(2 * a))
    assert pi @ eps == pytest.approx(expect, abs=1e-12)


def test_uniform_psi_local_energy():
    N = 7
    model = RBM(N, 3, np.zeros(N + 3 + 3 * N))
    ham = TFIM(N, 1, 1.3, 0.4)
    S = exact.all_configs(N)
    eps = local_energy(ham, model.logpsi, S)
    np.testing.assert_allclose(eps, ham.diagonal(S) + 0.4 * N, atol=1e-13)


def test_variational_principle():
    N = 8
    ham = TFIM(N, 1, 1.0, 1.0)
    e0 = exact.tfim_1d_free_fermion_e0(N, 1.0, 1.0)
    for seed in range(3):
        model = _rbm(N, 8, 0.5, seed)
        pi = exact.exact_pi(model.logpsi, N)
        e = pi @ local_energy(ham, model.logpsi, exact.all_configs(N))
        assert e >= e0 - 1e-12


@pytest.mark.parametrize("model_kind", ["rbm", "dense"])
def test_force_is_half_the_exact_energy_gradient(model_kind):
    # real parameters: dE/dtheta_k = 2 (E[O_k eps] - E[O_k] E[eps]) = 2 F_k (Eq. forces)
    N = 6
    ham = TFIM(N, 1, 1.0, 0.9)
    if model_kind == "rbm":
        p = rbm_params(N, 5, 0.3, 4)
        build = lambda q: RBM(N, 5, q)
    else:
        p = dense_params(N, (5, 4), 4, bias_sigma=0.2) * 0.7
        build = lambda q: Dense(N, (5, 4), q)
    S = exact.all_configs(N)

    def energy(q):
        m = build(q)
        pi = exact.exact_pi(m.logpsi, N)
        return pi @ local_energy(ham, m.logpsi, S)

    m = build(p)
    pi = exact.exact_pi(m.logpsi, N)
    eps = local_energy(ham, m.logpsi, S)
    O = m.grad(S)
    E = pi @ eps
    F = (pi[:, None] * O * (eps - E)[:, None]).sum(axis=0)
    h = 1e-5
    for k in np.random.default_rng(0).choice(p.size, 12, replace=False):
        e = np.zeros_like(p); e[k] = h
        g = (energy(p + e) - energy(p - e)) / (2 * h)
        assert 2 * F[k] == pytest.approx(g, abs=1e-7, rel=1e-6)


def test_sample_force_and_stats():
    rng = np.random.default_rng(0)
    O = rng.normal(size=(40, 3))
    eps = rng.normal(size=40)
    F = force(O, eps)
    np.testing.assert_allclose(F, np.cov(O.T, eps, bias=True)[-1, :3], atol=1e-14)
    E, var, err = energy_stats(eps, 8)
    assert E == pytest.approx(eps.mean()) and var == pytest.approx(eps.var())
    cm = eps.reshape(5, 8).mean(axis=0)
    assert err == pytest.approx(cm.std(ddof=1) / np.sqrt(8))


def test_energy_error_from_chain_blocks_matches_independent_routes():
    # The error of E from per-chain means (statistics reading) against routes that do not use
    # chain blocks: (i) i.i.d. draws, whose error of the mean is sigma / sqrt(n); (ii) AR(1)
    # chains x_{t+1} = rho x_t + sqrt(1 - rho^2) z, whose long-chain error of the mean is
    # sigma sqrt((1 + rho) / (1 - rho) / n).  The chain-block estimate must see the
    # autocorrelation that the naive sqrt(Var / n) misses.
    rng = np.random.default_rng(12)
    K, C, sigma = 400, 512, 1.7
    eps = rng.normal(3.0, sigma, size=(K, C)).reshape(-1)      # sweep-major rows k * C + c
    E, var, err = energy_stats(eps, C)
    assert var == pytest.approx(sigma ** 2, rel=0.01)
    assert err == pytest.approx(sigma / np.sqrt(K * C), rel=0.08)
    rho = 0.8
    x = np.empty((K, C))
    x[0] = rng.normal(size=C)
    for k in range(1, K):
        x[k] = rho * x[k - 1] + np.sqrt(1 - rho ** 2) * rng.normal(size=C)
    E, var, err = energy_stats(sigma * x.reshape(-1), C)
    want = sigma * np.sqrt((1 + rho) / (1 - rho) / (K * C))
    assert err == pytest.approx(want, rel=0.1)
    assert err > 2.5 * np.sqrt(var / (K * C))
