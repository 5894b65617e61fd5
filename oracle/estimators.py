"""Local energies, energy statistics and forces, in FP64.

Local energy (App. I, Eq. local_energies):
    eps(x) = sum_{x' in C(x)} H(x, x') psi(x') / psi(x),
evaluated by re-computing log psi(x') for every connected x'.  With the
Marshall sign (Heisenberg workloads) psi(x) = sign(x) exp(log psi_net(x)).

Energy (Sec. 2, Eq. loss): E = mean of eps over samples x ~ pi.
Force (App. I, Eq. forces), real parameters so O* = O:
    F_k = mean(O_k eps) - mean(O_k) mean(eps) = mean(O_k (eps - E)).
Statistics (reading): Var = mean((eps - E)^2); the error of E is the standard
deviation of the per-chain means (ddof 1) over sqrt(number of chains).
"""
import numpy as np

from .hamiltonian import TFIM, Heisenberg
from .models import marshall_sign


def local_energy(ham, logpsi_fn, samples, sub_a=None):
    """eps(x) for every row of samples [S, N] (+-1).  sub_a: Marshall sublattice mask or None."""
    s = np.asarray(samples, dtype=np.int8)
    S, N = s.shape
    lp = logpsi_fn(s)
    sign = marshall_sign(s, sub_a) if sub_a is not None else np.ones(S)
    eps = ham.diagonal(s).astype(np.float64)
    rows = np.arange(S)
    if isinstance(ham, TFIM):
        for i in range(N):
            y = s.copy()
            y[:, i] = -s[:, i]
            sy = marshall_sign(y, sub_a) if sub_a is not None else np.ones(S)
            eps += ham.h * (sy / sign) * np.exp(logpsi_fn(y) - lp)
    elif isinstance(ham, Heisenberg):
        for (i, j), J in zip(ham.bonds, ham.coupling):
            anti = s[:, i] != s[:, j]
            if not np.any(anti):
                continue
            y = s[anti].copy()
            y[:, i], y[:, j] = s[anti, j], s[anti, i]
            sy = marshall_sign(y, sub_a) if sub_a is not None else np.ones(len(y))
            eps[rows[anti]] += 2.0 * J * (sy / sign[anti]) * np.exp(logpsi_fn(y) - lp[anti])
    else:
        raise TypeError(type(ham))
    return eps


def energy_stats(eps, n_chains):
    """(mean, variance, error of the mean from chain blocks).  eps is sweep-major [K*C]."""
    eps = np.asarray(eps, dtype=np.float64)
    E = eps.mean()
    var = np.mean((eps - E) ** 2)
    if n_chains >= 2 and eps.size % n_chains == 0:
        chain_means = eps.reshape(-1, n_chains).mean(axis=0)
        err = chain_means.std(ddof=1) / np.sqrt(n_chains)
    else:
        err = np.sqrt(var / max(eps.size, 1))
    return E, var, err


def force(O, eps):
    """F_k = mean(O_k (eps - E)) over the sample rows of O [S, P]."""
    O = np.asarray(O, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    return (O * (eps - eps.mean())[:, None]).mean(axis=0)
