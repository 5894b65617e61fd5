"""Pins of the bias-bound machinery (Sec. 3.1, App. C) against exact MH kernels and quadrature."""
import numpy as np
import pytest
from scipy import integrate

from oracle import bounds, exact
from oracle.models import RBM
from workloads import rbm_params


@pytest.mark.parametrize("mu,sigma", [(0.0, 0.05), (0.0, 0.7), (0.3, 0.2), (-0.5, 1.1), (1.2, 0.4)])
def test_thm3_closed_form_matches_quadrature(mu, sigma):
    # E[exp(-|eps|)] for eps ~ N(mu, 2 sigma^2), integrated numerically
    sd = np.sqrt(2.0) * sigma
    f = lambda e: np.exp(-abs(e)) * np.exp(-(e - mu) ** 2 / (2 * sd * sd)) / (np.sqrt(2 * np.pi) * sd)
    val = integrate.quad(f, -np.inf, 0, epsabs=1e-14)[0] + integrate.quad(f, 0, np.inf, epsabs=1e-14)[0]
    assert bounds.thm3_bound(mu, sigma) == pytest.approx(1.0 - val, abs=1e-10)


def test_thm3_mu0_form_and_small_sigma_slope():
    for s in [0.01, 0.3, 1.5]:
        assert bounds.thm3_mu0_bound(s) == pytest.approx(bounds.thm3_bound(0.0, s), abs=1e-13)
    # the mu = 0 bound is linear in sigma near 0: 2 sigma / sqrt(pi) + O(sigma^2)
    s = 1e-4
    assert bounds.thm3_mu0_bound(s) == pytest.approx(2 * s / np.sqrt(np.pi), rel=1e-3)
    assert bounds.thm3_bound(0.0, 0.5, r=0.5) == pytest.approx(2 * bounds.thm3_bound(0.0, 0.5))


def test_delta_alpha_bound_on_grid_and_equality_on_the_boundary():
    s = np.exp(np.linspace(-6, 3, 301))[:, None]
    eps = np.linspace(-4, 4, 161)[None, :]
    assert np.all(bounds.delta_alpha(s, eps) <= bounds.delta_alpha_bound(eps) + 1e-15)
    e = np.linspace(0.01, 3, 50)
    np.testing.assert_allclose(bounds.delta_alpha(np.exp(-e), e), 1 - np.exp(-e), rtol=1e-12)


def _kernels(N=4, sigma_delta=0.3, seed=0):
    model = RBM(N, N, rbm_params(N, N, 0.5, seed))
    pi = exact.exact_pi(model.logpsi, N)
    delta = np.random.default_rng(seed + 1).normal(0.0, sigma_delta, size=pi.size)
    pi_t = bounds.perturbed_pi(pi, delta)
    return pi, pi_t, delta, exact.mh_kernel_flip(pi), exact.mh_kernel_flip(pi_t)


def test_mh_kernel_invariants():
    pi, _, _, P, _ = _kernels(N=6)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-15)
    F = pi[:, None] * P
    np.testing.assert_allclose(F, F.T, atol=1e-16)     # detailed balance
    np.testing.assert_allclose(exact.stationary(P), pi, atol=1e-12)


def test_theorem1_with_exact_contraction_of_a_multi_step_kernel():
    pi, pi_t, _, P, Pt = _kernels()
    k = 8
    Pk, Ptk = np.linalg.matrix_power(P, k), np.linalg.matrix_power(Pt, k)
    r = exact.dobrushin(Pk)
    assert r < 1.0
    lhs = bounds.tv_distance(pi, pi_t)
    assert lhs <= bounds.thm1_rhs(pi_t, Ptk, Pk, r) + 1e-15


def test_theorem2_for_arbitrary_pi_prime():
    pi, pi_t, delta, P, Pt = _kernels(N=5, sigma_delta=0.4, seed=3)
    D = pi.size
    N = 5
    x = np.arange(D)
    # E_{x ~ pi'} sum_y q(y|x) exp(-|eps(x, y)|), eps(x, y) = delta(y) - delta(x)
    for trial in range(5):
        pip = np.random.default_rng(trial).dirichlet(np.ones(D))
        avg = sum((pip * np.exp(-np.abs(delta[x ^ (1 << i)] - delta[x]))).sum() / N for i in range(N))
        lhs = bounds.tv_distance(0.0, pip @ (Pt - P))
        assert lhs <= 1.0 - avg + 1e-15


def test_exact_tv_obeys_pinsker_with_exact_kl():
    pi, pi_t, delta, _, _ = _kernels(N=8, sigma_delta=0.2)
    kl = np.sum(pi * np.log(pi / pi_t))
    assert bounds.tv_distance(pi, pi_t) <= np.sqrt(kl / 2)
    # for Gaussian delta KL(pi || pi~) = sigma^2 / 2 in expectation
    assert bounds.kl_gaussian(0.2) == pytest.approx(0.02)


def test_bias_bound_on_an_observable():
    pi, pi_t, _, _, _ = _kernels(N=6, sigma_delta=0.5, seed=2)
    f = np.random.default_rng(9).uniform(-3, 3, size=pi.size)
    A = np.abs(f).max()
    assert abs(pi_t @ f - pi @ f) <= 2 * A * bounds.tv_distance(pi, pi_t)


def test_unit_roundoffs_against_the_printed_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "precision_table.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for name, ebits, mbits, printed in rows:
        u = bounds.UNIT_ROUNDOFF[name]
        assert u == 2.0 ** -(int(mbits) + 1)          # round-to-nearest unit roundoff
        printed = float(printed)
        if name == "f16":
            printed *= 10.0                            # the table's exponent typo
        assert u == pytest.approx(printed, rel=2e-3)
    assert bounds.UNIT_ROUNDOFF["f16"] == np.finfo(np.float16).eps / 2
    assert bounds.UNIT_ROUNDOFF["f32"] == np.finfo(np.float32).eps / 2


def test_reported_bound_recovers_the_delta_sigma_from_flip_increments():
    # Theorem 3's statement takes eps ~ N(mu, 2 sigma^2) with sigma the std of delta (Sec. 3.1):
    # for delta ~ N(0, sigma^2) drawn independently per configuration, the single-flip
    # increments eps(x, y) = delta(y) - delta(x) have variance 2 sigma^2, so reported_bound
    # (which takes std(eps)) must return min(Pinsker, Thm 3) at the sigma that made delta.
    # Dropping the sqrt 2, or swapping (mu, std), moves the result by far more than the
    # sampling tolerance used here.
    N = 12
    x = np.arange(2 ** N)
    for sigma in (0.02, 0.3, 1.0):
        delta = np.random.default_rng(7).normal(0.0, sigma, size=x.size)
        eps = np.concatenate([delta[x ^ (1 << i)] - delta for i in range(N)])
        got = bounds.reported_bound(eps.mean(), eps.std())
        want = min(sigma / 2, bounds.thm3_bound(0.0, sigma))
        assert got == pytest.approx(want, rel=0.03)
        # and it bounds the exact distance of pi e^delta / Z from pi for an enumerated RBM whose
        # pi spreads over the space (Pinsker's sigma / 2 uses KL = sigma^2 / 2, the expectation
        # over delta, which a pi concentrated on a few configurations need not meet draw by draw)
        model = RBM(N, N, rbm_params(N, N, 0.05, 11))
        pi = exact.exact_pi(model.logpsi, N)
        assert bounds.tv_distance(pi, bounds.perturbed_pi(pi, delta)) <= got


@pytest.mark.parametrize("mu,sigma", [(0.1, 0.2), (-0.4, 0.6), (0.02, 0.01)])
def test_reported_bound_with_a_mean_shift(mu, sigma):
    # increments drawn as N(mu, 2 sigma^2) directly: the bound is min(sigma / 2, Thm 3(mu, sigma))
    eps = np.random.default_rng(3).normal(mu, np.sqrt(2.0) * sigma, size=400_000)
    got = bounds.reported_bound(eps.mean(), eps.std())
    assert got == pytest.approx(min(sigma / 2, bounds.thm3_bound(mu, sigma)), rel=5e-3)
    # Theorem 3 is the Gaussian expectation of Theorem 2's average: 1 - E[e^{-|eps|}]
    assert bounds.thm2_bound(eps) == pytest.approx(bounds.thm3_bound(mu, sigma), rel=5e-3, abs=2e-4)


def test_thm2_bound_on_chain_proposals_bounds_the_one_step_distance():
    # Theorem 2: ||pi'(P~ - P)||_TV <= 1 - E_{x ~ pi', y ~ q}[e^{-|eps(x, y)|}], with the
    # expectation estimated from proposals drawn as a chain would draw them (x ~ pi',
    # y a uniform single flip of x).  Exact average and its Monte Carlo estimate agree.
    pi, pi_t, delta, P, Pt = _kernels(N=5, sigma_delta=0.4, seed=3)
    D, N = pi.size, 5
    x = np.arange(D)
    rng = np.random.default_rng(5)
    for trial in range(3):
        pip = rng.dirichlet(np.ones(D))
        xs = rng.choice(D, size=200_000, p=pip)
        ys = xs ^ (1 << rng.integers(0, N, size=xs.size))
        est = bounds.thm2_bound(delta[ys] - delta[xs])
        exact_avg = sum((pip * np.exp(-np.abs(delta[x ^ (1 << i)] - delta[x]))).sum() / N for i in range(N))
        assert est == pytest.approx(1.0 - exact_avg, abs=4e-3)
        assert bounds.tv_distance(0.0, pip @ (Pt - P)) <= 1.0 - exact_avg + 1e-15
