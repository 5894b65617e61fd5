"""Noisy RBM (Sec. 4.1): log psi~(x) = log psi(x) + zeta(x) / 2 with zeta(x) ~ N(0, sigma)
drawn once per configuration x and held fixed across evaluations, so that the sampled
density changes by log p~(x) - log p(x) = zeta(x), of standard deviation sigma (reading
of the garbled "variance sigma": sigma is the standard deviation).

zeta(x) is a function of the configuration, so both sides compute it from one
counter-based construction of this project, from published definitions only:
  * hash: Philox4x32-10 (Salmon et al., SC'11) chained over the packed configuration
    words w_0 .. w_{W-1} (zero-padded to a multiple of 4): h = (TAG_NOISE, W, 0, 0);
    for every block b of four words, h = Philox(h XOR (w_4b .. w_4b+3); key);
  * normal deviate: Box-Muller (Box and Muller, 1958) on u1 = ((h0 >> 8) + 1) 2^-24 in
    (0, 1] and u2 = (h1 >> 8) 2^-24 in [0, 1): z = sqrt(-2 ln u1) cos(2 pi u2);
  * zeta(x) = sigma z.
"""
import numpy as np

from .philox import MASK32, philox4x32_10

TAG_NOISE = 0x4E4F4953   # "NOIS"


def pack_words(s):
    """[n, N] +-1 -> [n, W] uint64 words (bit i % 32 of word i // 32 set iff s_i = +1)."""
    s = np.asarray(s)
    n, N = s.shape
    W = (N + 31) // 32
    bits = np.zeros((n, W * 32), dtype=np.uint64)
    bits[:, :N] = s > 0
    return (bits.reshape(n, W, 32) << np.arange(32, dtype=np.uint64)).sum(axis=2)


def config_hash(s, key):
    """The four Philox output words of the chained hash of each configuration."""
    w = pack_words(s)
    n, W = w.shape
    Wp = (W + 3) // 4 * 4
    wp = np.zeros((n, Wp), dtype=np.uint64)
    wp[:, :W] = w
    k0, k1 = key & MASK32, (key >> 32) & MASK32
    h = [np.full(n, TAG_NOISE, dtype=np.uint64), np.full(n, W, dtype=np.uint64),
         np.zeros(n, dtype=np.uint64), np.zeros(n, dtype=np.uint64)]
    for b in range(Wp // 4):
        h = list(philox4x32_10(h[0] ^ wp[:, 4 * b], h[1] ^ wp[:, 4 * b + 1], h[2] ^ wp[:, 4 * b + 2],
                               h[3] ^ wp[:, 4 * b + 3], k0, k1))
    return h


def zeta(s, sigma, key):
    """zeta(x) = sigma z(x), z standard normal by Box-Muller on the configuration hash (FP64)."""
    h = config_hash(s, key)
    u1 = ((h[0] >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (h[1] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def noisy_logpsi(logpsi_fn, sigma, key):
    """log psi~ = log psi + zeta / 2 as a function of configurations."""
    return lambda s: logpsi_fn(s) + 0.5 * zeta(s, sigma, key)
