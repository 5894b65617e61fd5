"""Exact references for small systems (N <= 16): enumeration, sparse H, ED, exact MH kernels.

* Enumeration of pi(x) = |psi(x)|^2 / Z over all 2^N configurations (Sec. 2).
  Configuration index n <-> spins s_i = +1 if bit i of n is set, else -1.
* The Hamiltonian as a sparse 2^N x 2^N matrix built from its matrix elements
  (Eq. TFIM; App. E) and its ground energy by Lanczos (scipy eigsh).
* Free-fermion ground energy of the periodic 1D TFIM for even N (textbook
  Jordan-Wigner result, even-parity sector with antiperiodic fermion momenta):
      E0 = - sum_{m=0}^{N-1} sqrt(J^2 + h^2 - 2 J h cos(pi (2m + 1) / N)).
* The MH transition matrix P (Sec. 3.1): P(x, y) = q(y|x) alpha(x, y) for
  x != y and P(x, x) = 1 - sum_{z != x} P(x, z).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hamiltonian import TFIM, Heisenberg


def all_configs(N):
    n = np.arange(2 ** N, dtype=np.int64)
    bits = (n[:, None] >> np.arange(N)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def config_index(s):
    s = np.atleast_2d(np.asarray(s))
    return ((s > 0).astype(np.int64) << np.arange(s.shape[1])[None, :]).sum(axis=1)


def exact_pi(logpsi_fn, N, mask=None):
    """pi over all 2^N configurations (optionally restricted to mask)."""
    lp = logpsi_fn(all_configs(N))
    logp = 2.0 * lp
    if mask is not None:
        logp = np.where(mask, logp, -np.inf)
    logp -= logp.max()
    p = np.exp(logp)
    return p / p.sum()


def sparse_hamiltonian(ham, sub_a=None):
    """H in the computational basis; with sub_a the Marshall-rotated basis is used
    (off-diagonal elements multiplied by sign(x') sign(x))."""
    N = ham.N
    S = all_configs(N)
    idx = np.arange(2 ** N)
    rows, cols, vals = [idx], [idx], [ham.diagonal(S)]
    if isinstance(ham, TFIM):
        for i in range(N):
            rows.append(idx)
            cols.append(idx ^ (1 << i))
            vals.append(np.full(idx.size, ham.h))
    else:
        for (i, j), J in zip(ham.bonds, ham.coupling):
            anti = S[:, i] != S[:, j]
            r = idx[anti]
            rows.append(r)
            cols.append(r ^ (1 << i) ^ (1 << j))
            v = np.full(r.size, 2.0 * J)
            if sub_a is not None and sub_a[i] != sub_a[j]:
                v = -v   # exchange across sublattices changes the Marshall sign
            vals.append(v)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(2 ** N, 2 ** N))


def ground_energy(H, k=1):
    vals = spla.eigsh(H, k=k, which="SA", tol=1e-12)[0]
    return np.sort(vals)


def tfim_1d_free_fermion_e0(N, J, h):
    m = np.arange(N)
    k = np.pi * (2 * m + 1) / N
    return -np.sum(np.sqrt(J * J + h * h - 2.0 * J * h * np.cos(k)))


def mh_kernel_flip(pi):
    """Exact single-flip MH kernel on 2^N states (q = 1/N per flip, App. C Eq. app:local_prop)."""
    D = pi.size
    N = int(round(np.log2(D)))
    P = np.zeros((D, D))
    x = np.arange(D)
    for i in range(N):
        y = x ^ (1 << i)
        with np.errstate(divide="ignore", invalid="ignore"):
            alpha = np.minimum(1.0, pi[y] / pi[x])
        P[x, y] += alpha / N
    P[x, x] = 1.0 - P.sum(axis=1)
    return P


def stationary(P):
    """Left eigenvector of P with eigenvalue 1, normalised to a probability vector."""
    w, v = np.linalg.eig(P.T)
    k = np.argmin(np.abs(w - 1.0))
    p = np.real(v[:, k])
    return p / p.sum()


def dobrushin(P):
    """Exact TV contraction coefficient r = max_{x, x'} ||P(x, .) - P(x', .)||_TV."""
    r = 0.0
    for a in range(P.shape[0]):
        r = max(r, 0.5 * np.abs(P[a][None, :] - P).sum(axis=1).max())
    return r
