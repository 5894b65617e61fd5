"""Complex-parameter RBM in FP64/complex128: the oracle of the complex-RBM row (test
infrastructure: only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package).

App. G writes the RBM with complex parameters a in C^N, b in C^M, W in C^{M x N}:
    log psi(s) = a . s + sum_j log cosh(theta_j),   theta = W s + b,
with s in {-1, +1}^N.  Sec. 2: the sampled density is p(s) = |psi(s)|^2 / Z, so log p = 2 Re log psi
and a Metropolis-Hastings chain decides on 2 Re(log psi(y) - log psi(x)).

Local energy (App. I, Eq. local_energies) of the TFIM (Sec. 4.1, Eq. TFIM, +h as printed):
    eps(x) = J sum_<ij> s_i s_j + h sum_i psi(flip_i x) / psi(x),   complex for complex psi.
Force (App. I, Eq. forces): F_k = E[O_k^* eps] - E[O_k^*] E[eps] with O_k = d log psi / d theta_k
(log psi is holomorphic in the parameters): O_a = s, O_b = tanh(theta), O_W[j, i] = tanh(theta_j) s_i.

Parameters are passed as one complex vector in the order [a | b | W] (W row-major, [M][N]).
"""
import numpy as np

from .hamiltonian import TFIM


def log_cosh_c(z):
    """log cosh z for complex z without overflow: z + log(1 + e^{-2z}) - log 2 for Re z >= 0, the
    mirror form for Re z < 0 (log cosh is even).  The imaginary part is fixed only modulo 2 pi,
    which exp(log psi) does not see."""
    z = np.asarray(z, dtype=np.complex128)
    w = np.where(z.real >= 0.0, z, -z)
    return w + np.log1p(np.exp(-2.0 * w)) - np.log(2.0)


class ComplexRBM:
    def __init__(self, n_visible, n_hidden, params):
        self.N, self.M = int(n_visible), int(n_hidden)
        p = np.asarray(params, dtype=np.complex128)
        if p.size != self.N + self.M + self.M * self.N:
            raise ValueError("RBM parameter vector has the wrong length")
        self.a = p[:self.N]
        self.b = p[self.N:self.N + self.M]
        self.W = p[self.N + self.M:].reshape(self.M, self.N)
        self.n_params = p.size

    def theta(self, s):
        s = np.asarray(s, dtype=np.float64)
        return s @ self.W.T + self.b

    def logpsi(self, s):
        """App. G: a . s + sum_j log cosh(theta_j), complex."""
        s = np.asarray(s, dtype=np.float64)
        return s @ self.a + log_cosh_c(self.theta(s)).sum(axis=-1)

    def log_density(self, s):
        """log p(s) / 2 = Re log psi(s): what the sampler compares."""
        return self.logpsi(s).real

    def grad(self, s):
        """O_k = d log psi / d theta_k (holomorphic): O_a = s, O_b = tanh(theta), O_W = tanh(theta_j) s_i."""
        s = np.atleast_2d(np.asarray(s, dtype=np.float64))
        t = np.tanh(self.theta(s))
        ow = t[:, :, None] * s[:, None, :]
        return np.concatenate([s.astype(np.complex128), t, ow.reshape(s.shape[0], -1)], axis=1)


def local_energy_tfim(ham, model, samples):
    """Complex eps(x) of the TFIM for every row of samples [S, N] (+-1), by re-evaluating log psi
    of every single-flip neighbour."""
    if not isinstance(ham, TFIM):
        raise TypeError(type(ham))
    s = np.asarray(samples, dtype=np.int8)
    S, N = s.shape
    lp = model.logpsi(s)
    eps = ham.diagonal(s).astype(np.complex128)
    for i in range(N):
        y = s.copy()
        y[:, i] = -s[:, i]
        eps += ham.h * np.exp(model.logpsi(y) - lp)
    return eps


def force(O, eps, weights=None):
    """F_k = E[O_k^* eps] - E[O_k^*] E[eps]: sample means, or expectations under the given
    probabilities (weights summing to 1, e.g. an enumerated |psi|^2)."""
    O = np.asarray(O, dtype=np.complex128)
    eps = np.asarray(eps, dtype=np.complex128)
    w = np.full(len(eps), 1.0 / len(eps)) if weights is None else np.asarray(weights, dtype=np.float64)
    E = w @ eps
    return (np.conj(O) * (w * (eps - E))[:, None]).sum(axis=0)
