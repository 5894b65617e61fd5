"""Pins of the noisy-RBM oracle: the noise is a fixed function of the configuration, it is
standard normal in distribution (moments and a Kolmogorov-Smirnov test against the normal
CDF), it vanishes at sigma = 0, the hash is chained over every word, and the exact noisy
distribution is pi e^zeta / Z."""
import numpy as np
from scipy import stats

from oracle import exact
from oracle.models import RBM
from oracle.noisy import config_hash, noisy_logpsi, zeta
from workloads import rbm_params


def test_noise_is_a_fixed_function_of_the_configuration():
    rng = np.random.default_rng(1)
    s = rng.choice([-1, 1], size=(50, 40)).astype(np.int8)
    a = zeta(s, 0.3, 7)
    np.testing.assert_array_equal(a, zeta(s.copy(), 0.3, 7))
    np.testing.assert_array_equal(a[::-1], zeta(s[::-1], 0.3, 7))      # per row, not per position
    assert not np.allclose(a, zeta(s, 0.3, 8))                           # the key matters
    np.testing.assert_allclose(zeta(s, 0.6, 7), 2 * a, rtol=1e-15)       # linear in sigma
    np.testing.assert_array_equal(zeta(s, 0.0, 7), 0.0)


def test_noise_is_standard_normal_over_configurations():
    s = exact.all_configs(16)                                            # 65536 configurations
    z = zeta(s, 1.0, 20260006)
    assert abs(z.mean()) < 4 / np.sqrt(len(z))
    assert abs(z.std() - 1) < 4 / np.sqrt(2 * len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(stats.skew(z)) < 0.05 and abs(stats.kurtosis(z)) < 0.1


def test_hash_covers_every_word():
    # configurations differing only in a spin of the second or ninth word hash differently
    base = -np.ones((1, 300), dtype=np.int8)
    for i in (0, 40, 255, 299):
        y = base.copy()
        y[0, i] = 1
        assert any(int(a[0]) != int(b[0]) for a, b in zip(config_hash(base, 3), config_hash(y, 3)))


def test_exact_noisy_distribution_is_tilted_by_exp_zeta():
    N, M = 10, 10
    model = RBM(N, M, rbm_params(N, M, 0.3, 2))
    sig, key = 0.5, 11
    pi = exact.exact_pi(model.logpsi, N)
    pit = exact.exact_pi(noisy_logpsi(model.logpsi, sig, key), N)
    w = pi * np.exp(zeta(exact.all_configs(N), sig, key))
    np.testing.assert_allclose(pit, w / w.sum(), rtol=1e-12)
