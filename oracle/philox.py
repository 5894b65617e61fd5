"""Philox4x32-10 counter-based generator, and the draw layout of the sampler.

Test infrastructure only: the oracle is imported by tests/, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg, never by
the product path.

The paper does not fix a random-number generator (its code uses the JAX/NetKet
default).  Both sides of this project draw from Philox4x32-10 as defined by
Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC'11): a 4 x 32-bit counter, a 2 x 32-bit key, ten rounds, each round two
32x32->64 multiplications by the published multipliers followed by a swap and
an xor with the round key; the key is bumped by the published Weyl constants
between rounds.  The layout of counters and the mapping from words to sites,
bonds and uniforms below is this project's own convention; the CUDA side
re-implements it independently and must agree bit for bit.

Counter layout (all words 32-bit):
    sweep proposals : ctr = (pair k, sweep index t, chain c, TAG_SWEEP)
    initial spins   : ctr = (block b, sub-stream, chain c, TAG_INIT)
Key = (seed mod 2^32, seed >> 32).

Within a sweep, proposal 2k uses output words (w0, w1) of pair k and proposal
2k+1 uses (w2, w3): the first word picks the site (or bond) by the
multiply-shift map idx = (w * n) >> 32, the second gives u = (w >> 8) * 2^-24.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_SWEEP = 0x53574550   # "SWEP"
TAG_INIT = 0x494E4954    # "INIT"


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit words held in uint64.

    Returns the four output words (uint64 arrays with values < 2^32).
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    sh = np.uint64(32)
    msk = np.uint64(MASK32)
    for rnd in range(10):
        if rnd > 0:   # key schedule: bump by the Weyl constants between rounds
            k0 = (k0 + np.uint64(PHILOX_W0)) & msk
            k1 = (k1 + np.uint64(PHILOX_W1)) & msk
        p0 = m0 * c0          # < 2^64, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & msk
        hi1, lo1 = p1 >> sh, p1 & msk
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def key_from_seed(seed):
    seed = int(seed) & ((1 << 64) - 1)
    return seed & MASK32, seed >> 32


def index_from_word(w, n):
    """Multiply-shift map of a 32-bit word onto {0, ..., n-1}."""
    return ((np.asarray(w, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def uniform_from_word(w):
    """u = (w >> 8) * 2^-24, an exact multiple of 2^-24 in [0, 1)."""
    return (np.asarray(w, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def sweep_draws(seed, chains, sweep, n_steps, n_choices):
    """Proposal draws of one sweep for the given chains.

    Returns (idx [len(chains), n_steps] int64, u [len(chains), n_steps] f64):
    idx is the flipped site (single-flip moves) or the exchanged bond.
    """
    chains = np.asarray(chains, dtype=np.uint64)
    k0, k1 = key_from_seed(seed)
    n_pairs = (n_steps + 1) // 2
    idx = np.empty((chains.size, 2 * n_pairs), dtype=np.int64)
    u = np.empty((chains.size, 2 * n_pairs), dtype=np.float64)
    for k in range(n_pairs):
        w0, w1, w2, w3 = philox4x32_10(np.full(chains.shape, k, np.uint64),
                                       np.full(chains.shape, sweep, np.uint64),
                                       chains,
                                       np.full(chains.shape, TAG_SWEEP, np.uint64),
                                       k0, k1)
        idx[:, 2 * k] = index_from_word(w0, n_choices)
        u[:, 2 * k] = uniform_from_word(w1)
        idx[:, 2 * k + 1] = index_from_word(w2, n_choices)
        u[:, 2 * k + 1] = uniform_from_word(w3)
    return idx[:, :n_steps], u[:, :n_steps]


def init_spins_random(seed, chains, n_sites):
    """Independent uniform +-1 spins: site i takes bit (i mod 128) of block i // 128."""
    chains = np.asarray(chains, dtype=np.uint64)
    k0, k1 = key_from_seed(seed)
    s = np.empty((chains.size, n_sites), dtype=np.int8)
    for b in range((n_sites + 127) // 128):
        words = philox4x32_10(np.full(chains.shape, b, np.uint64), np.zeros(chains.shape, np.uint64),
                              chains, np.full(chains.shape, TAG_INIT, np.uint64), k0, k1)
        for i in range(b * 128, min(n_sites, (b + 1) * 128)):
            r = i - b * 128
            bit = (words[r // 32] >> np.uint64(r % 32)) & np.uint64(1)
            s[:, i] = np.where(bit == 1, 1, -1)
    return s


def init_spins_balanced(seed, chains, n_sites):
    """Uniformly random configuration with zero total magnetisation (n_sites even).

    Start from s_i = +1 for i < n/2 and -1 otherwise, then run a Fisher-Yates
    shuffle from the top: for i = n-1 .. 1 swap positions i and j, with
    j = (w_i * (i + 1)) >> 32 and w_i word (i mod 4) of block i // 4 of
    sub-stream 1.
    """
    chains = np.asarray(chains, dtype=np.uint64)
    k0, k1 = key_from_seed(seed)
    s = np.where(np.arange(n_sites) < n_sites // 2, 1, -1).astype(np.int8)
    s = np.tile(s, (chains.size, 1))
    rows = np.arange(chains.size)
    for i in range(n_sites - 1, 0, -1):
        words = philox4x32_10(np.full(chains.shape, i // 4, np.uint64), np.ones(chains.shape, np.uint64),
                              chains, np.full(chains.shape, TAG_INIT, np.uint64), k0, k1)
        j = index_from_word(words[i % 4], i + 1)
        si = s[rows, i].copy()
        s[rows, i] = s[rows, j]
        s[rows, j] = si
    return s
