"""minSR update on the GPU (nqs_minsr) against the FP64 oracle (oracle/minsr.py), on the same
FP32 O rows:

* the Gram matrix T = Obar Obar^T (tensor cores, three BF16 terms per FP32 value, FP64 partial
  sums) within GRAM_TOL of max |T|.  The tensor cores add each MMA's result into the FP32
  accumulator without round-to-nearest (measured: sums of positive terms come out short); one
  FP64 drain follows 16 K blocks x 4 MMAs = 64 accumulations, each short by at most one ulp
  (2^-23 relative) of the running sum, and on average half of it: a relative shortfall of at
  most 64 x 2^-24 ~ 3.8e-6 (measured 1.9e-6 on K = 2e5 diagonals).  That is more accurate than
  a round-to-nearest FP32 sum of the same 2e5 products (~sqrt(K) 2^-24 ~ 2.7e-5);
* dtheta = Obar^T (T + lambda I)^-1 ebar (FP64 Cholesky and solves) within 1e-5 of max |dtheta|;
* ragged sizes (row tiles and K blocks with tails), many K parts and FP64 drains, and O rows of
  a sampled RBM.
"""
import numpy as np
import pytest

from helpers import nqs
from oracle.minsr import gram, minsr_update
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAM_TOL = 64 * 2.0 ** -24


def _ctx_with_P(P):
    """An RBM context whose parameter count is exactly P = N + M + M N (only P is used)."""
    for N in range(3, 400):
        if (P - N) % (N + 1) == 0 and (P - N) // (N + 1) >= 1:
            M = (P - N) // (N + 1)
            if M <= 1024:
                return nqs().Context("tfim", N, 1, J1=1.0, h=1.0, model="rbm", n_hidden=M, dtype="f32")
    raise ValueError(P)


def _run(ctx, O, eps, lam):
    n = O.shape[0]
    Od = torch.from_numpy(O).cuda()
    ed = torch.from_numpy(eps).cuda()
    stats = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(ed, n, stats)
    d = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    T = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx.minsr(Od, ed, stats, lam, d, T)
    ctx.check_status()
    return d.cpu().numpy(), T.cpu().numpy()


@pytest.mark.parametrize("n,P,lam", [(300, 1000, 1e-3), (129, 4097, 1e-1), (256, 199_999, 1e-3),
                                     (2, 1000, 1e-1), (65, 2999, 1e-3), (2200, 4999, 1e-3)])
def test_minsr_matches_oracle_on_gaussian_rows(n, P, lam):
    """Also the edges of the blocked Cholesky and triangular solves (64-row blocks): n = 2, one
    block and a row (65), and 35 blocks with a 24-row last block and an odd count of 128-row
    Gram tiles (2200)."""
    ctx = _ctx_with_P(P)
    P = ctx.P
    rng = np.random.default_rng(n + P)
    O = (rng.normal(size=(n, P)) + rng.normal(size=P)).astype(np.float32)    # non-zero column means
    eps = rng.normal(-5.0, 2.0, size=n).astype(np.float32)
    d, T = _run(ctx, O, eps, lam)
    O64, e64 = O.astype(np.float64), eps.astype(np.float64)
    Tref = gram(O64)
    assert np.abs(T - Tref).max() <= GRAM_TOL * np.abs(Tref).max(), np.abs(T - Tref).max()
    np.testing.assert_allclose(T, T.T, rtol=0, atol=0)
    dref, _, _ = minsr_update(O64, e64, lam)
    assert np.abs(d - dref).max() <= 1e-5 * np.abs(dref).max(), (np.abs(d - dref).max(), np.abs(dref).max())


def test_minsr_on_sampled_rbm_rows():
    p = nqs()
    N, M, C = 36, 72, 512
    ctx = p.Context("tfim", 6, 6, J1=1.0, h=2.0, model="rbm", n_hidden=M, dtype="f32")
    ctx.set_params(torch.from_numpy(rbm_params(N, M, 0.1, 17)).cuda())
    st = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(st, 3)
    S = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(st, 20, 19, 4, 0, S)
    e = torch.empty(C, dtype=torch.float32, device="cuda")
    ctx.local_energy(S, e)
    O = torch.empty((C, ctx.P), dtype=torch.float32, device="cuda")
    ctx.logpsi_grad(S, O)
    d, T = _run(ctx, O.cpu().numpy(), e.cpu().numpy(), 1e-3)
    O64, e64 = O.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    Tref = gram(O64)
    assert np.abs(T - Tref).max() <= GRAM_TOL * np.abs(Tref).max()
    dref, _, _ = minsr_update(O64, e64, 1e-3)
    assert np.abs(d - dref).max() <= 1e-4 * np.abs(dref).max(), (np.abs(d - dref).max(), np.abs(dref).max())


def test_minsr_rejects_bad_arguments():
    p = nqs()
    ctx = _ctx_with_P(1000)
    O = torch.zeros((1, ctx.P), dtype=torch.float32, device="cuda")
    e = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = torch.zeros(5, dtype=torch.float64, device="cuda")
    d = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    with pytest.raises(p.NQSError):
        ctx.minsr(O, e, st, 1e-3, d, workspace=torch.zeros(16, dtype=torch.uint8, device="cuda"))   # n = 1
    O = torch.zeros((4, ctx.P), dtype=torch.float32, device="cuda")
    e = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(p.NQSError):
        ctx.minsr(O, e, st, 0.0, d)                                      # lambda must be positive


def test_minsr_on_sampled_rescnn_rows():
    """The minSR step of a ResCNN VMC iteration (the ansatz the paper trains with SR): O rows of
    the ResCNN's reverse pass on samples of its F16 sampler, local energies, then nqs_minsr,
    against the oracle's minSR of the same rows."""
    from workloads import rescnn_params
    p = nqs()
    C = 384
    ctx = p.Context("tfim", 6, 5, J1=1.0, h=3.0, model="rescnn", n_hidden=16, n_blocks=2, dtype="f16")
    ctx.set_params(torch.from_numpy(rescnn_params(16, 2, 23)).cuda())
    st = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(st, 5)
    S = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(st, 6, 5, 6, 0, S)
    e = torch.empty(C, dtype=torch.float32, device="cuda")
    ctx.local_energy(S, e)
    O = torch.empty((C, ctx.P), dtype=torch.float32, device="cuda")
    ctx.logpsi_grad(S, O)
    d, T = _run(ctx, O.cpu().numpy(), e.cpu().numpy(), 1e-3)
    O64, e64 = O.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    assert np.abs(T - gram(O64)).max() <= GRAM_TOL * np.abs(gram(O64)).max()
    dref, _, _ = minsr_update(O64, e64, 1e-3)
    assert np.abs(d - dref).max() <= 1e-4 * np.abs(dref).max(), (np.abs(d - dref).max(), np.abs(dref).max())
