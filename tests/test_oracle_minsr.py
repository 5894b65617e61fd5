"""Pins of the minSR oracle: two routes to the SR update, the ridge-regression optimality
condition it solves, the solve residual, and closed forms for one sample and for orthogonal
rows."""
import numpy as np
import pytest

from oracle.estimators import force
from oracle.minsr import centred, gram, minsr_update, sr_update


@pytest.mark.parametrize("S,P,lam", [(8, 30, 1e-3), (40, 12, 1e-1), (64, 200, 1e-3), (5, 5, 0.5)])
def test_push_through_identity_matches_the_p_by_p_solve(S, P, lam):
    rng = np.random.default_rng(S * 1000 + P)
    O = rng.normal(size=(S, P)) + rng.normal(size=P)      # non-zero column means
    eps = rng.normal(-3.0, 2.0, size=S)
    d, _, _ = minsr_update(O, eps, lam)
    np.testing.assert_allclose(d, sr_update(O, eps, lam), rtol=1e-9, atol=1e-11)


def test_update_solves_the_regularised_least_squares_problem():
    # dtheta minimises |Obar d - ebar|^2 + lam |d|^2: gradient Obar^T (Obar d - ebar) + lam d = 0
    rng = np.random.default_rng(3)
    O, eps, lam = rng.normal(size=(50, 120)), rng.normal(size=50), 1e-3
    d, y, T = minsr_update(O, eps, lam)
    Ob, eb, _ = centred(O, eps)
    g = Ob.T @ (Ob @ d - eb) + lam * d
    assert np.abs(g).max() <= 1e-10 * (1 + np.abs(Ob.T @ eb).max())
    assert np.linalg.norm((T + lam * np.eye(50)) @ y - eb) / np.linalg.norm(eb) <= 1e-10


def test_force_is_the_unpreconditioned_limit():
    # lam -> infinity: lam * dtheta -> Obar^T ebar = F (App. I, Eq. forces)
    rng = np.random.default_rng(4)
    O, eps = rng.normal(size=(30, 17)), rng.normal(size=30)
    d, _, _ = minsr_update(O, eps, 1e9)
    np.testing.assert_allclose(1e9 * d, force(O, eps), rtol=1e-6, atol=1e-12)


def test_orthogonal_centred_rows_closed_form():
    # rows with Obar Obar^T = diag(q): y_x = ebar_x / (q_x + lam)
    S, P = 6, 10
    Q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(P, P)))
    base = Q[:S] * np.arange(1, S + 1)[:, None]
    O = np.vstack([base, -base])                            # column means zero; 2S rows
    eps = np.random.default_rng(6).normal(size=2 * S)
    lam = 0.3
    d, y, T = minsr_update(O, eps, lam)
    Ob, eb, _ = centred(O, eps)
    np.testing.assert_allclose(gram(O), Ob @ Ob.T, rtol=0, atol=1e-14)
    # T has the block form [[D, -D], [-D, D]] with D = diag(k^2) / (2S)
    Dg = np.arange(1, S + 1) ** 2 / (2 * S)
    np.testing.assert_allclose(np.diag(T)[:S], Dg, rtol=1e-12)
    np.testing.assert_allclose(T[:S, S:], -np.diag(Dg), atol=1e-12)
    # the solution in closed form: along u = (e_k, -e_k) eigenvalue 2 D_k, along v = (e_k, e_k) zero
    u = (eb[:S] - eb[S:]) / 2
    v = (eb[:S] + eb[S:]) / 2
    np.testing.assert_allclose(y[:S], u / (2 * Dg + lam) + v / lam, rtol=1e-10)
    np.testing.assert_allclose(y[S:], -u / (2 * Dg + lam) + v / lam, rtol=1e-10)
