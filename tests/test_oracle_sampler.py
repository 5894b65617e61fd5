"""Pins of the oracle's MH sampler: exact stationary law, closed forms, conserved quantities."""
import numpy as np
import pytest

from oracle import exact
from oracle.lattice import nn_bonds
from oracle.models import RBM
from oracle.philox import init_spins_random, init_spins_balanced
from oracle.sampler import mh_sweeps, ReplayMismatch
from workloads import rbm_params


def test_histogram_matches_exact_distribution():
    N, C = 8, 512
    model = RBM(N, 8, rbm_params(N, 8, 0.35, 11))
    s0 = init_spins_random(1, np.arange(C), N)
    out = mh_sweeps(model.logpsi, s0, np.arange(C), seed=2, n_sweeps=60, burn_in=10)
    idx = exact.config_index(out["samples"])
    hist = np.bincount(idx, minlength=2 ** N) / idx.size
    pi = exact.exact_pi(model.logpsi, N)
    tv = 0.5 * np.abs(hist - pi).sum()
    # noise floor: i.i.d. draws of the same count from the exact law
    rng = np.random.default_rng(0)
    floors = [0.5 * np.abs(np.bincount(rng.choice(pi.size, idx.size, p=pi), minlength=pi.size) / idx.size - pi).sum()
              for _ in range(5)]
    assert tv < 1.5 * max(floors) + 0.01
    # a wrong target (sign error in log p) is far away
    pi_wrong = exact.exact_pi(lambda s: -model.logpsi(s), N)
    assert 0.5 * np.abs(hist - pi_wrong).sum() > 5 * tv


def test_uniform_target_accepts_every_proposal():
    N, C = 10, 64
    model = RBM(N, 4, np.zeros(N + 4 + 4 * N))
    s0 = init_spins_random(3, np.arange(C), N)
    out = mh_sweeps(model.logpsi, s0, np.arange(C), seed=4, n_sweeps=5, burn_in=0)
    assert np.all(out["n_accepted"] == 5 * N)


def test_product_state_magnetisation():
    N, M, C = 6, 3, 2048
    p = rbm_params(N, M, 0.3, 5)
    p[N:] = 0.0
    model = RBM(N, M, p)
    s0 = init_spins_random(6, np.arange(C), N)
    out = mh_sweeps(model.logpsi, s0, np.arange(C), seed=7, n_sweeps=25, burn_in=5)
    m = out["samples"].mean(axis=0)
    np.testing.assert_allclose(m, np.tanh(2 * p[:N]), atol=5 * np.sqrt(1.0 / out["samples"].shape[0]) * 2)


def test_exchange_moves_conserve_magnetisation_and_null_moves_accept():
    N, C = 8, 128
    model = RBM(N, 8, rbm_params(N, 8, 0.3, 8))
    s0 = init_spins_balanced(9, np.arange(C), N)
    out = mh_sweeps(model.logpsi, s0, np.arange(C), seed=10, n_sweeps=6, burn_in=0,
                    proposal="exchange", bonds=nn_bonds(N, 1))
    assert np.all(out["samples"].sum(axis=1) == 0)
    # uniform target: every exchange (including equal-spin null moves) is accepted
    flat = RBM(N, 2, np.zeros(N + 2 + 2 * N))
    out2 = mh_sweeps(flat.logpsi, s0, np.arange(C), seed=10, n_sweeps=3, burn_in=0,
                     proposal="exchange", bonds=nn_bonds(N, 1))
    assert np.all(out2["n_accepted"] == 3 * N)


def test_sweep_is_a_deterministic_function_of_seed_and_offset():
    N, C = 6, 16
    model = RBM(N, 6, rbm_params(N, 6, 0.4, 1))
    s0 = init_spins_random(1, np.arange(C), N)
    a = mh_sweeps(model.logpsi, s0, np.arange(C), seed=3, n_sweeps=4, burn_in=0)
    b1 = mh_sweeps(model.logpsi, s0, np.arange(C), seed=3, n_sweeps=2, burn_in=0)
    b2 = mh_sweeps(model.logpsi, b1["spins"], np.arange(C), seed=3, n_sweeps=2, burn_in=0, sweep_offset=2)
    np.testing.assert_array_equal(a["spins"], b2["spins"])


def test_replay_accepts_its_own_decisions_and_rejects_a_planted_flip():
    N, C, T = 6, 32, 3
    model = RBM(N, 6, rbm_params(N, 6, 0.4, 2))
    s0 = init_spins_random(2, np.arange(C), N)
    # record own decisions through the deltas and draws
    ref = mh_sweeps(model.logpsi, s0, np.arange(C), seed=5, n_sweeps=T, burn_in=0, record_deltas=True)
    from oracle.philox import sweep_draws
    acc = np.zeros((C, T, N), dtype=bool)
    for t in range(T):
        _, u = sweep_draws(5, np.arange(C), t, N, N)
        acc[:, t, :] = u < np.exp(2 * ref["deltas"][:, t, :])
    rep = mh_sweeps(model.logpsi, s0, np.arange(C), seed=5, n_sweeps=T, burn_in=0, replay_accepts=acc)
    np.testing.assert_array_equal(rep["spins"], ref["spins"])
    assert rep["near_threshold"] == 0
    bad = acc.copy()
    bad[3, 1, 2] = not bad[3, 1, 2]
    with pytest.raises(ReplayMismatch):
        mh_sweeps(model.logpsi, s0, np.arange(C), seed=5, n_sweeps=T, burn_in=0, replay_accepts=bad)
