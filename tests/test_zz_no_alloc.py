"""nqs_force_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (code under another framework's memory budget, plugins that may not
allocate after start-up) get the force without passing a workspace: the library
uses a built-in device array instead.  This checks, through the C ABI, that two
calls in a row agree with the force of nqs_logpsi_grad (which uses a caller
workspace) on the same inputs, with the tolerance of the other force tests.
Kept in its own file, collected last.
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, to_words_tensor
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _force_with_workspace(ctx, cfg, eloc, stats):
    n = cfg.shape[0]
    f = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctx.logpsi_grad_workspace(n), dtype=torch.uint8, device="cuda")
    ctx.logpsi_grad(cfg, None, eloc, stats, f, ws)
    return f


@pytest.mark.parametrize("Lx,Ly,M,n", [(10, 10, 400, 3000), (16, 1, 16, 777)])
def test_force_noalloc_matches_workspace_entry_point_twice(Lx, Ly, M, n):
    p = nqs()
    N = Lx * Ly
    ctx = p.Context("tfim", Lx, Ly, J1=1.0, h=3.04, model="rbm", n_hidden=M)
    ctx.set_params(torch.from_numpy(rbm_params(N, M, 0.05, 31)).cuda())
    rng = np.random.default_rng(32)
    for call in range(2):           # two calls in a row, different inputs each time
        s = rng.choice([-1, 1], size=(n, N)).astype(np.int8)
        cfg = to_words_tensor(pack_np(s))
        eloc = torch.from_numpy(rng.normal(-300.0 + call, 4.0, n).astype(np.float32)).cuda()
        stats = torch.zeros(5, dtype=torch.float64, device="cuda")
        ctx.stats(eloc, n, stats)
        ref = _force_with_workspace(ctx, cfg, eloc, stats)
        got = torch.full((ctx.P,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.force_noalloc(cfg, eloc, stats, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-5 * max(1.0, np.abs(r).max()))


def test_force_noalloc_rejects_bad_sizes():
    p = nqs()
    ctx = p.Context("tfim", 8, 1, h=1.0, model="rbm", n_hidden=8)
    ctx.set_params(torch.from_numpy(rbm_params(8, 8, 0.1, 1)).cuda())
    cfg = torch.zeros((0, 1), dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.float32, device="cuda")
    st = torch.zeros(5, dtype=torch.float64, device="cuda")
    f = torch.zeros(ctx.P, dtype=torch.float64, device="cuda")
    with pytest.raises(p.NQSError):
        ctx.force_noalloc(cfg, e, st, f)
