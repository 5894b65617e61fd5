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


# (16, 16, 1024) is the largest RBM the library takes (N <= 256, M <= 1024): the most
# parameters (263,424) and so the most of the built-in scratch any call can use.
@pytest.mark.parametrize("Lx,Ly,M,n", [(10, 10, 400, 3000), (16, 1, 16, 777), (16, 16, 1024, 1500)])
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


def test_force_noalloc_empty_batch_and_rejections():
    p = nqs()
    ctx = p.Context("tfim", 8, 1, h=1.0, model="rbm", n_hidden=8)
    ctx.set_params(torch.from_numpy(rbm_params(8, 8, 0.1, 1)).cuda())
    cfg = torch.zeros((0, 1), dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.float32, device="cuda")
    st = torch.zeros(5, dtype=torch.float64, device="cuda")
    # no rows: the force is zero, as nqs_logpsi_grad gives it
    f = torch.full((ctx.P,), 7.0, dtype=torch.float64, device="cuda")
    ctx.force_noalloc(cfg, e, st, f)
    ref = torch.full((ctx.P,), 7.0, dtype=torch.float64, device="cuda")
    ctx.logpsi_grad(cfg, None, e, st, ref, None)
    torch.cuda.synchronize()
    assert torch.equal(f, ref) and not f.any()
    # NULL force, or NULL inputs with rows, through the C ABI: NQS_EINVAL
    assert p._lib.nqs_force_noalloc(ctx._h, None, 0, None, None, None, None) == 1
    assert p._lib.nqs_force_noalloc(ctx._h, None, 4, None, None, f.data_ptr(), None) == 1
    # the dense ansatz has no allocation-free force
    dctx = p.Context("heisenberg", 4, 4, J1=1.0, model="dense", widths=(32, 32), dtype="bf16")
    from workloads import dense_params
    dctx.set_params(torch.from_numpy(dense_params(16, (32, 32), 2)).cuda())
    with pytest.raises(p.NQSError):
        dctx.force_noalloc(cfg, e, st, torch.zeros(dctx.P, dtype=torch.float64, device="cuda"))
