"""LogPsi, the torch.autograd.Function over the library's forward (nqs_logpsi) and hand-written
backward (the force kernel with eloc = upstream gradient, E = 0): the parameter gradient of
sum_x g_x log psi(x) against the oracle's O rows, for the RBM (FP32 copy), the dense ansatz and
the ResCNN."""
import numpy as np
import pytest

from helpers import nqs, pack_np, to_words_tensor
from oracle.models import RBM, Dense
from workloads import rbm_params, dense_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(ctx, model, params, N, n=300, seed=1):
    p = nqs()
    rng = np.random.default_rng(seed)
    s = rng.choice([-1, 1], size=(n, N)).astype(np.int8)
    if hasattr(model, "widths"):                        # the Heisenberg dense ansatz: zero magnetisation
        from oracle.philox import init_spins_balanced
        s = init_spins_balanced(seed, np.arange(n), N)
    cfg = to_words_tensor(pack_np(s))
    theta = torch.from_numpy(params).cuda().requires_grad_(True)
    lp = p.LogPsi.apply(ctx, theta, cfg)
    g = torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda()
    (lp * g).sum().backward()
    ref = model.grad(s).T @ g.cpu().numpy().astype(np.float64)
    got = theta.grad.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * (np.abs(ref).max() + 1.0), np.abs(got - ref).max()
    return lp


def test_rbm_logpsi_autograd_matches_oracle():
    N, M = 16, 24
    params = rbm_params(N, M, 0.2, 3)
    ctx = nqs().Context("tfim", N, 1, J1=1.0, h=1.0, model="rbm", n_hidden=M, dtype="f32")
    lp = _check(ctx, RBM(N, M, params), params, N)
    assert lp.dtype == torch.float32


def test_dense_logpsi_autograd_matches_oracle():
    N, widths = 16, (64, 48)
    params = dense_params(N, widths, 5, bias_sigma=0.1)
    ctx = nqs().Context("heisenberg", 4, 4, J1=1.0, model="dense", widths=widths, dtype="bf16")
    _check(ctx, Dense(N, widths, params), params, N, n=200)


def test_rescnn_logpsi_autograd_matches_oracle():
    from oracle.rescnn import ResCNN
    from workloads import rescnn_params
    params = rescnn_params(16, 2, 9)
    ctx = nqs().Context("tfim", 4, 4, J1=1.0, h=1.0, model="rescnn", n_hidden=16, n_blocks=2, dtype="f32")
    _check(ctx, ResCNN(4, 4, 16, 2, params), params, 16, n=150)
