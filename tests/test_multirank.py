"""The step's exchange across ranks (two gloo ranks on the CPU): statistics and force of
the pooled samples from per-rank partials, against the oracle on the pooled data.

Each rank stands in for one GPU: its local statistics and force are computed here in
FP64 the way the product's kernels define them (mean, variance 1/n, force centred on
the E held in stats[0]); the reduction code under test is bench.py's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td
import torch.multiprocessing as mp

import bench
from oracle.estimators import force as oracle_force


def _data(rank):
    rng = np.random.default_rng(100 + rank)
    n = 300 + 137 * rank                       # uneven sample counts
    O = rng.normal(size=(n, 7)) + rank         # rank-dependent means: E_r != E
    eps = rng.normal(-3.0 + 2.0 * rank, 1.0 + rank, size=n)
    return O, eps


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    O, eps = _data(rank)
    n = len(eps)
    stats = torch.tensor([eps.mean(), eps.var(), eps.std() / np.sqrt(n), 0.5, n], dtype=torch.float64)
    n_total = bench.reduce_stats_across_ranks(stats, n, td)
    E = float(stats[0])
    force = torch.from_numpy(O.T @ (eps - E) / n)       # the force kernel's definition with stats[0]
    bench.reduce_force_across_ranks(force, n, n_total, td)
    out[rank] = (float(n_total), stats.numpy().copy(), force.numpy().copy())
    td.destroy_process_group()


def test_two_rank_reduction_matches_pooled_oracle():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    O = np.concatenate([_data(r)[0] for r in range(2)])
    eps = np.concatenate([_data(r)[1] for r in range(2)])
    for r in range(2):
        n, stats, force = out[r]
        assert n == len(eps)
        np.testing.assert_allclose(stats[0], eps.mean(), rtol=1e-13)
        np.testing.assert_allclose(stats[1], eps.var(), rtol=1e-12)
        np.testing.assert_allclose(force, oracle_force(O, eps), rtol=1e-12, atol=1e-12)
    # centring each rank on its own E_r instead would be wrong by a visible margin
    naive = sum(len(_data(r)[1]) * oracle_force(*_data(r)) for r in range(2)) / len(eps)
    assert np.abs(naive - oracle_force(O, eps)).max() > 1e-2
