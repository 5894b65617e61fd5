"""Pins of the oracle's ansaetze and their O_k (finite differences, closed forms)."""
import numpy as np
import pytest

from oracle.models import RBM, Dense, log_cosh
from workloads import rbm_params, dense_params, dense_n_params, rbm_n_params


def test_log_cosh_against_numpy_and_asymptote():
    z = np.linspace(-20, 20, 2001)
    np.testing.assert_allclose(log_cosh(z), np.log(np.cosh(z)), rtol=1e-14, atol=1e-15)
    big = np.array([400.0, -800.0])
    np.testing.assert_allclose(log_cosh(big), np.abs(big) - np.log(2.0), rtol=1e-15)


def test_parameter_counts_of_the_workloads():
    assert dense_n_params(100, (400, 400)) == 201_201
    assert dense_n_params(256, (1024, 1024, 1024)) == 2_363_393
    assert rbm_n_params(100, 400) == 40_500
    assert rbm_n_params(16, 16) == 288


def test_rbm_reduces_to_visible_bias_without_hidden_weights():
    N, M = 9, 4
    p = rbm_params(N, M, 0.5, 0)
    p[N:] = 0.0
    s = np.random.default_rng(1).choice([-1, 1], size=(20, N))
    np.testing.assert_allclose(RBM(N, M, p).logpsi(s), s @ p[:N] + M * 0.0, atol=1e-14)


def test_rbm_single_hidden_unit_by_hand():
    N = 3
    a = np.array([0.1, -0.2, 0.3]); b = np.array([0.05]); W = np.array([[0.4, -0.5, 0.6]])
    m = RBM(N, 1, np.concatenate([a, b, W.ravel()]))
    s = np.array([1, -1, 1])
    z = 0.05 + 0.4 + 0.5 + 0.6
    assert m.logpsi(s[None])[0] == pytest.approx(a @ s + np.log(np.cosh(z)), abs=1e-15)


def _fd_grad(fn, p, s, h=1e-5):
    g = np.zeros((s.shape[0], p.size))
    for k in range(p.size):
        e = np.zeros_like(p); e[k] = h
        g[:, k] = (fn(p + e, s) - fn(p - e, s)) / (2 * h)
    return g


def test_rbm_grad_matches_finite_differences():
    N, M = 6, 5
    p = rbm_params(N, M, 0.4, 2)
    s = np.random.default_rng(3).choice([-1, 1], size=(7, N))
    g = RBM(N, M, p).grad(s)
    fd = _fd_grad(lambda q, x: RBM(N, M, q).logpsi(x), p, s)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)


def test_dense_grad_matches_finite_differences():
    N, widths = 6, (5, 4, 3)
    p = dense_params(N, widths, 5, bias_sigma=0.3)
    s = np.random.default_rng(4).choice([-1, 1], size=(5, N))
    g = Dense(N, widths, p).grad(s)
    fd = _fd_grad(lambda q, x: Dense(N, widths, q).logpsi(x), p, s)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)


def test_dense_single_layer_by_hand():
    N = 2
    W1 = np.array([[0.3, -0.2]]); b1 = np.array([0.1]); w_out = np.array([1.5]); b_out = 0.25
    m = Dense(N, (1,), np.concatenate([W1.ravel(), b1, w_out, [b_out]]))
    s = np.array([[1, 1]])
    assert m.logpsi(s)[0] == pytest.approx(1.5 * np.log(np.cosh(0.2)) + 0.25, abs=1e-15)
