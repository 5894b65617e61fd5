"""The step's exchange across ranks (two gloo ranks on the CPU): statistics and force of
the pooled samples from per-rank buffers, against the oracle on the pooled data.

Each rank stands in for one GPU.  Its moments and force share are built here in FP64 the
way nqs_stats_moments and nqs_force_share define them (include/nqs.h); the exchange under
test is the package's (paper_2601_20782_b300.distributed).  nqs_stats_finalize is a GPU
kernel, so the ranks' context here is a stand-in whose finalize applies the header's
formula; the kernel itself is checked on the GPU against the pooled oracle
(tests/test_gpu_rbm.py::test_moments_and_force_shares_of_split_chains)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td
import torch.multiprocessing as mp

from oracle.estimators import energy_stats as oracle_stats
from oracle.estimators import force as oracle_force

K = 6   # samples per chain


def _data(rank):
    rng = np.random.default_rng(100 + rank)
    C = 50 + 23 * rank                         # uneven chain counts
    O = rng.normal(size=(K * C, 7)) + rank     # rank-dependent means: E_r != E
    eps = rng.normal(-3.0 + 2.0 * rank, 1.0 + rank, size=K * C)
    acc = rng.integers(0, 40, size=C)
    return O, eps, acc, C


def _moments(eps, acc, C, proposals):
    m = eps.reshape(K, C).mean(axis=0)
    return torch.tensor([eps.size, eps.sum(), (eps ** 2).sum(), C, m.sum(), (m ** 2).sum(), acc.sum(),
                         C * proposals], dtype=torch.float64)


class _FinalizeStandIn:
    """nqs_stats_finalize's formula (include/nqs.h) for CPU ranks."""

    def stats_finalize(self, m, out):
        n, C = m[0], m[3]
        mean = m[1] / n
        mm = m[4] / C
        out[:] = torch.stack([mean, m[2] / n - mean ** 2, torch.sqrt((m[5] - C * mm * mm) / (C - 1) / C),
                              m[6] / m[7], n])


def _worker(rank, world, port, out):
    from paper_2601_20782_b300.distributed import exchange_force, exchange_stats
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    O, eps, acc, C = _data(rank)
    moments = _moments(eps, acc, C, 40)
    stats = torch.zeros(5, dtype=torch.float64)
    exchange_stats(_FinalizeStandIn(), moments, stats)
    force = torch.from_numpy(O.T @ (eps - float(stats[0])) / float(stats[4]))   # nqs_force_share
    exchange_force(force)
    out[rank] = (stats.numpy().copy(), force.numpy().copy())
    td.destroy_process_group()


def test_two_rank_exchange_matches_pooled_oracle():
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
    d = [_data(r) for r in range(2)]
    # pooled chains in one sweep-major array: row k * C_total + c
    eps = np.concatenate([x[1].reshape(K, x[3]) for x in d], axis=1).reshape(-1)
    C_tot = sum(x[3] for x in d)
    E, var, err = oracle_stats(eps, C_tot)
    acc_rate = sum(x[2].sum() for x in d) / (C_tot * 40)
    O_pooled = np.concatenate([x[0].reshape(K, x[3], 7) for x in d], axis=1).reshape(-1, 7)
    for r in range(2):
        stats, force = out[r]
        np.testing.assert_allclose(stats, [E, var, err, acc_rate, eps.size], rtol=1e-12)
        np.testing.assert_allclose(force, oracle_force(O_pooled, eps), rtol=1e-12, atol=1e-12)
    # centring each rank on its own E_r instead would be wrong by a visible margin
    naive = sum(len(x[1]) * oracle_force(x[0], x[1]) for x in d) / eps.size
    assert np.abs(naive - oracle_force(O_pooled, eps)).max() > 1e-2
