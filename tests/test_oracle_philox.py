"""Pins of the oracle's Philox4x32-10 and of its draw layout.

The generator is pinned against an independent implementation: cuRAND's
host-side PHILOX4_32_10 generator (NVIDIA's library, run on the CPU), whose
first output blocks are Philox4x32-10 of counter (0, 0, b, 0) under key
(seed mod 2^32, seed >> 32).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle.philox import (philox4x32_10, sweep_draws, init_spins_random, init_spins_balanced,
                           index_from_word, uniform_from_word)


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path and (os.path.exists(path) or not path.startswith("/")):
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


CURAND = _curand()


@pytest.mark.skipif(CURAND is None, reason="libcurand not found")
@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 20260002, 2 ** 64 - 1])
def test_philox_matches_curand_host_generator(seed):
    gen = ctypes.c_void_p()
    assert CURAND.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
    try:
        assert CURAND.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 64
        out = np.zeros(n, dtype=np.uint32)
        assert CURAND.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        CURAND.curandDestroyGenerator(gen)
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    b = np.arange(n // 4, dtype=np.uint64)
    w = philox4x32_10(np.zeros_like(b), np.zeros_like(b), b, np.zeros_like(b), k0, k1)
    mine = np.stack(w, axis=1).reshape(-1).astype(np.uint32)
    np.testing.assert_array_equal(mine, out)


def test_index_and_uniform_maps():
    w = np.array([0, 1, 2 ** 31, 2 ** 32 - 1], dtype=np.uint64)
    np.testing.assert_array_equal(index_from_word(w, 100), [0, 0, 50, 99])
    u = uniform_from_word(w)
    assert u[0] == 0.0 and u[-1] == 1.0 - 2.0 ** -24
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))


def test_sweep_draws_ranges_and_uniformity():
    idx, u = sweep_draws(seed=7, chains=np.arange(4096), sweep=3, n_steps=17, n_choices=17)
    assert idx.min() == 0 and idx.max() == 16
    assert np.all((u >= 0) & (u < 1))
    counts = np.bincount(idx.ravel(), minlength=17)
    expected = idx.size / 17
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 60.0          # 16 dof; p < 1e-6 above this
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)


def test_sweep_draws_odd_step_count_is_prefix_of_even():
    a, ua = sweep_draws(11, np.arange(8), 5, 9, 9)
    b, ub = sweep_draws(11, np.arange(8), 5, 10, 9)
    np.testing.assert_array_equal(a, b[:, :9])
    np.testing.assert_array_equal(ua, ub[:, :9])


def test_init_spins_random_is_balanced_in_distribution():
    s = init_spins_random(3, np.arange(2048), 200)
    assert set(np.unique(s)) == {-1, 1}
    assert abs(s.mean()) < 5 / np.sqrt(s.size)
    # different chains differ
    assert not np.array_equal(s[0], s[1])


def test_init_spins_balanced_zero_magnetisation_and_uniform_positions():
    s = init_spins_balanced(5, np.arange(4000), 16)
    assert np.all(s.sum(axis=1) == 0)
    up = (s > 0).mean(axis=0)
    assert np.all(np.abs(up - 0.5) < 5 * np.sqrt(0.25 / 4000))
