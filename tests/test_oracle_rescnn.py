"""Pins of the ResCNN oracle (App. H) against routes that do not share its code.

* The whole forward pass rebuilt from library layers in FP64 (torch: circular padding +
  conv2d, layer_norm, gelu in its tanh form), not from the oracle's roll / matmul code.
* The periodic convolution against scipy.ndimage.correlate in wrap mode.
* Lattice translations leave log psi unchanged (periodic padding and a sum readout);
  zero padding would not.
* A residual block whose second convolution is zero is the identity.
* Layer normalisation over the channels of one site: mean 0 and variance var/(var + eps).
* O_k against central finite differences of log psi.
* <H> from local energies equals the Rayleigh quotient of the sparse Hamiltonian.
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import exact
from oracle.estimators import local_energy
from oracle.hamiltonian import TFIM
from oracle.rescnn import LN_EPS, ResCNN, conv3x3, layer_norm, n_params
from workloads import rescnn_params

torch = pytest.importorskip("torch")
import torch.nn.functional as Fnn


def _torch_logpsi(m, s):
    """log psi through torch's layers (NCHW, float64)."""
    x = torch.from_numpy(np.asarray(s, dtype=np.float64).reshape(-1, 1, m.Ly, m.Lx))

    def conv(v, K, b):
        return Fnn.conv2d(Fnn.pad(v, (1, 1, 1, 1), mode="circular"), torch.from_numpy(K), torch.from_numpy(b))

    def ln(v, g, be):   # over channels: NCHW -> NHWC, normalise the last axis, back
        y = Fnn.layer_norm(v.permute(0, 2, 3, 1), (m.F,), torch.from_numpy(g), torch.from_numpy(be), eps=LN_EPS)
        return y.permute(0, 3, 1, 2)

    h = conv(x, m.K0, m.b0)
    for (g, be, K1, b1, K2, b2) in m.blocks:
        a = Fnn.gelu(ln(h, g, be), approximate="tanh")
        h = h + conv(Fnn.gelu(conv(a, K1, b1), approximate="tanh"), K2, b2)
    return ln(h, m.gF, m.bF).sum(dim=(1, 2, 3)).numpy()


@pytest.mark.parametrize("Lx,Ly,F,B", [(4, 4, 16, 4), (6, 5, 8, 2), (10, 10, 16, 4), (3, 7, 4, 1)])
def test_forward_matches_library_layers(Lx, Ly, F, B):
    m = ResCNN(Lx, Ly, F, B, rescnn_params(F, B, 11 + Lx))
    s = np.random.default_rng(Lx * Ly).choice([-1, 1], size=(40, Lx * Ly))
    np.testing.assert_allclose(m.logpsi(s), _torch_logpsi(m, s), rtol=1e-12, atol=1e-10)


def test_conv_matches_scipy_wrap_correlation():
    rng = np.random.default_rng(3)
    inp = rng.normal(size=(2, 5, 7, 3))
    K = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    out = conv3x3(inp, K, b)
    for sidx in range(2):
        for o in range(4):
            ref = b[o] + sum(ndimage.correlate(inp[sidx, :, :, c], K[o, c], mode="wrap") for c in range(3))
            np.testing.assert_allclose(out[sidx, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_translation_invariance():
    L = 6
    m = ResCNN(L, L, 8, 3, rescnn_params(8, 3, 5))
    s = np.random.default_rng(2).choice([-1, 1], size=(8, L, L))
    base = m.logpsi(s.reshape(8, -1))
    for dy, dx in [(1, 0), (0, 1), (2, 5), (5, 3)]:
        moved = np.roll(s, shift=(dy, dx), axis=(1, 2)).reshape(8, -1)
        np.testing.assert_allclose(m.logpsi(moved), base, rtol=1e-12, atol=1e-11)
    # and it is not a constant function
    assert np.ptp(base) > 1.0


def test_zero_second_conv_makes_blocks_the_identity():
    F, B, L = 8, 3, 4
    p = rescnn_params(F, B, 9)
    m = ResCNN(L, L, F, B, p)
    q = p.copy()
    off = 10 * F
    for _ in range(B):
        off += 2 * F + 9 * F * F + F
        q[off:off + 9 * F * F + F] = 0.0      # K2, b2
        off += 9 * F * F + F
    m0 = ResCNN(L, L, F, 0, np.concatenate([p[:10 * F], p[-2 * F:]]))
    s = np.random.default_rng(4).choice([-1, 1], size=(16, L * L))
    np.testing.assert_allclose(ResCNN(L, L, F, B, q).logpsi(s), m0.logpsi(s), rtol=1e-13, atol=1e-12)
    assert np.abs(m.logpsi(s) - m0.logpsi(s)).max() > 1e-3


def test_layer_norm_normalises_channels_of_each_site():
    v = np.random.default_rng(6).normal(2.0, 3.0, size=(3, 4, 5, 16))
    y, zhat, var = layer_norm(v, np.ones(16), np.zeros(16))
    np.testing.assert_allclose(y.mean(axis=-1), 0.0, atol=1e-12)
    np.testing.assert_allclose((y ** 2).mean(axis=-1), (var / (var + LN_EPS))[..., 0], rtol=1e-12)


def test_grad_matches_central_differences():
    F, B, L = 4, 2, 4
    p = rescnn_params(F, B, 21)
    m = ResCNN(L, L, F, B, p)
    assert m.n_params == n_params(F, B) == p.size
    s = np.random.default_rng(8).choice([-1, 1], size=(3, L * L))
    O = m.grad(s)
    h = 1e-5
    for k in np.random.default_rng(1).choice(p.size, 40, replace=False).tolist() + [0, p.size - 1, 10 * F]:
        e = np.zeros_like(p)
        e[k] = h
        fd = (ResCNN(L, L, F, B, p + e).logpsi(s) - ResCNN(L, L, F, B, p - e).logpsi(s)) / (2 * h)
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-6, atol=1e-7)


def test_energy_from_local_energies_is_the_rayleigh_quotient():
    L = 3
    m = ResCNN(L, L, 4, 2, rescnn_params(4, 2, 31))
    ham = TFIM(L, L, 1.0, 3.04)
    S = exact.all_configs(L * L)
    pi = exact.exact_pi(m.logpsi, L * L)
    e_loc = pi @ local_energy(ham, m.logpsi, S)
    psi = np.exp(m.logpsi(S) - m.logpsi(S).max())
    H = exact.sparse_hamiltonian(ham)
    assert e_loc == pytest.approx(psi @ (H @ psi) / (psi @ psi), rel=1e-12)
