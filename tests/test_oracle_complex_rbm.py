"""The complex-parameter RBM oracle (App. G with a, b, W complex) pinned by what the physics
and mathematics fix, not by restating its formulas:

* real parameters reduce it to the real RBM oracle (log psi, O rows, local energies, force);
* a phase i pi/2 on every visible bias multiplies psi by i^N (-1)^{#down}, which maps the TFIM
  with +h onto the one with -h: local energies agree exactly;
* the local-energy expectation under |psi|^2 equals the Rayleigh quotient psi^dag H psi /
  psi^dag psi of the sparse Hamiltonian (a matrix-vector route), with a vanishing imaginary part;
* the force is half the gradient of the exact energy in the real and in the imaginary
  direction of each parameter (App. I, Eq. forces with O^*), checked by central differences;
* O is the holomorphic derivative of log psi (real and imaginary steps agree);
* log cosh is even, finite for large arguments, and its exponential is cosh.
"""
import numpy as np
import pytest

from oracle import exact
from oracle.complex_rbm import ComplexRBM, log_cosh_c, local_energy_tfim, force
from oracle.estimators import local_energy as real_local_energy, force as real_force
from oracle.hamiltonian import TFIM
from oracle.models import RBM
from workloads import rbm_params


def complex_params(N, M, sigma, seed):
    rng = np.random.default_rng(seed)
    n = N + M + N * M
    return rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)


def test_real_parameters_reduce_to_the_real_rbm():
    N, M = 8, 12
    p = rbm_params(N, M, 0.2, 3)
    c, r = ComplexRBM(N, M, p.astype(np.complex128)), RBM(N, M, p)
    s = np.random.default_rng(1).choice([-1, 1], size=(64, N)).astype(np.int8)
    np.testing.assert_allclose(c.logpsi(s).real, r.logpsi(s), rtol=0, atol=1e-12)
    np.testing.assert_allclose(c.logpsi(s).imag, 0.0, atol=1e-12)
    np.testing.assert_allclose(c.grad(s), r.grad(s), rtol=0, atol=1e-12)
    ham = TFIM(N, 1, 1.0, 0.7)
    ec, er = local_energy_tfim(ham, c, s), real_local_energy(ham, r.logpsi, s)
    np.testing.assert_allclose(ec, er, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(force(c.grad(s), ec), real_force(r.grad(s), er), rtol=1e-10, atol=1e-12)


def test_visible_phase_maps_plus_h_onto_minus_h():
    # a_i -> a_i + i pi/2 multiplies psi(s) by exp(i pi/2 sum_i s_i) = i^N (-1)^{#down}: every single
    # flip changes #down by one, so psi(flip_i x)/psi(x) changes sign and eps(+h) = eps(-h)
    N, M = 9, 7
    p = complex_params(N, M, 0.25, 5)
    q = p.copy()
    q[:N] += 0.5j * np.pi
    s = np.random.default_rng(2).choice([-1, 1], size=(50, N)).astype(np.int8)
    e_shift = local_energy_tfim(TFIM(3, 3, 1.0, 1.3), ComplexRBM(N, M, q), s)
    e_ref = local_energy_tfim(TFIM(3, 3, 1.0, -1.3), ComplexRBM(N, M, p), s)
    np.testing.assert_allclose(e_shift, e_ref, rtol=1e-11, atol=1e-11)


def _exact_energy(ham, model, N):
    S = exact.all_configs(N)
    lp = model.logpsi(S)
    psi = np.exp(lp - lp.real.max())
    H = exact.sparse_hamiltonian(ham)
    return (np.conj(psi) @ (H @ psi)) / (np.conj(psi) @ psi)


def test_local_energy_expectation_equals_rayleigh_quotient():
    N, M = 8, 10
    ham = TFIM(N, 1, 1.0, 0.8)
    m = ComplexRBM(N, M, complex_params(N, M, 0.3, 7))
    S = exact.all_configs(N)
    pi = exact.exact_pi(m.log_density, N)
    E_loc = pi @ local_energy_tfim(ham, m, S)
    E_rq = _exact_energy(ham, m, N)
    assert abs(E_rq.imag) < 1e-12
    assert abs(E_loc.imag) < 1e-10
    assert E_loc.real == pytest.approx(E_rq.real, abs=1e-10)


def test_force_is_half_the_exact_energy_gradient_in_both_directions():
    # holomorphic psi: dE/dRe(theta_k) = 2 Re F_k and dE/dIm(theta_k) = 2 Im F_k with
    # F_k = E[O_k^* eps] - E[O_k^*] E[eps] (App. I, Eq. forces)
    N, M = 6, 5
    ham = TFIM(N, 1, 1.0, 0.9)
    p = complex_params(N, M, 0.3, 11)
    S = exact.all_configs(N)
    m = ComplexRBM(N, M, p)
    pi = exact.exact_pi(m.log_density, N)
    F = force(m.grad(S), local_energy_tfim(ham, m, S), weights=pi)
    energy = lambda q: _exact_energy(ham, ComplexRBM(N, M, q), N).real
    h = 1e-5
    for k in np.random.default_rng(0).choice(p.size, 10, replace=False):
        e = np.zeros_like(p); e[k] = h
        g_re = (energy(p + e) - energy(p - e)) / (2 * h)
        g_im = (energy(p + 1j * e) - energy(p - 1j * e)) / (2 * h)
        assert 2 * F[k].real == pytest.approx(g_re, abs=1e-7, rel=1e-6)
        assert 2 * F[k].imag == pytest.approx(g_im, abs=1e-7, rel=1e-6)


def test_O_is_the_holomorphic_derivative():
    N, M = 7, 6
    p = complex_params(N, M, 0.3, 13)
    s = np.random.default_rng(3).choice([-1, 1], size=(5, N)).astype(np.int8)
    O = ComplexRBM(N, M, p).grad(s)
    h = 1e-6
    for k in np.random.default_rng(4).choice(p.size, 8, replace=False):
        e = np.zeros_like(p); e[k] = h
        lp = lambda q: ComplexRBM(N, M, q).logpsi(s)
        d_re = (lp(p + e) - lp(p - e)) / (2 * h)
        d_im = (lp(p + 1j * e) - lp(p - 1j * e)) / (2j * h)
        np.testing.assert_allclose(d_re, O[:, k], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(d_im, O[:, k], rtol=1e-6, atol=1e-8)


def test_log_cosh_c():
    rng = np.random.default_rng(5)
    z = rng.normal(0, 2, 200) + 1j * rng.normal(0, 2, 200)
    np.testing.assert_allclose(np.exp(log_cosh_c(z)), np.cosh(z), rtol=1e-12)
    np.testing.assert_allclose(np.exp(log_cosh_c(-z)), np.exp(log_cosh_c(z)), rtol=1e-12)
    big = np.array([800.0 + 3j, -900.0 - 1j])
    v = log_cosh_c(big)
    assert np.all(np.isfinite(v))
    np.testing.assert_allclose(v.real, np.abs(big.real) - np.log(2.0), rtol=1e-14)
