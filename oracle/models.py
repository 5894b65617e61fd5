"""Variational ansaetze log psi(s) in FP64, and their per-sample log-derivatives O_k.

Spins are s in {-1, +1}^N (the paper writes x in {0, 1}^N in Sec. 2 and App. G;
s = 2x - 1 is a reparametrisation).  Parameters are real, so log psi is real
and log p = 2 log psi (Sec. 2, log p = 2 Re log psi).

RBM (App. G): log psi(s) = a . s + sum_{j < alpha N} log cosh((W s + b)_j).
Dense feed-forward ansatz (the paper names "feed-forward networks" in Sec. 1.1
without an architecture; reading): a_1 = log cosh(W_1 s + b_1),
a_l = tanh(W_l a_{l-1} + b_l) for l >= 2, log psi = w_out . a_L + b_out.

O_k(s) = d log psi(s) / d theta_k (App. I, Eq. forces), in the flat parameter
order of the input generators: RBM [a | b | W], dense [W1 | b1 | ... | w_out | b_out].
"""
import numpy as np


def log_cosh(z):
    """log cosh z = |z| + log1p(exp(-2|z|)) - log 2, exact in FP64 for all z."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    return z + np.log1p(np.exp(-2.0 * z)) - np.log(2.0)


class RBM:
    def __init__(self, n_visible, n_hidden, params):
        self.N, self.M = int(n_visible), int(n_hidden)
        p = np.asarray(params, dtype=np.float64)
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
        """App. G, with s in {-1, +1}: a . s + sum_j log cosh(theta_j)."""
        s = np.asarray(s, dtype=np.float64)
        return s @ self.a + log_cosh(self.theta(s)).sum(axis=-1)

    def grad(self, s):
        """Closed-form O_k: O_a = s, O_b = tanh(theta), O_W[j, i] = tanh(theta_j) s_i."""
        s = np.atleast_2d(np.asarray(s, dtype=np.float64))
        t = np.tanh(self.theta(s))
        ow = t[:, :, None] * s[:, None, :]
        return np.concatenate([s, t, ow.reshape(s.shape[0], -1)], axis=1)


class Dense:
    def __init__(self, n_visible, widths, params):
        self.N = int(n_visible)
        self.widths = tuple(int(w) for w in widths)
        p = np.asarray(params, dtype=np.float64)
        self.Ws, self.bs = [], []
        off, fan = 0, self.N
        for w in self.widths:
            self.Ws.append(p[off:off + w * fan].reshape(w, fan)); off += w * fan
            self.bs.append(p[off:off + w]); off += w
            fan = w
        self.w_out = p[off:off + fan]; off += fan
        self.b_out = p[off]; off += 1
        if off != p.size:
            raise ValueError("dense parameter vector has the wrong length")
        self.n_params = p.size

    def forward(self, s):
        """Returns (log psi, pre-activations z_l, activations a_l)."""
        a = np.asarray(s, dtype=np.float64)
        zs, acts = [], [a]
        for l, (W, b) in enumerate(zip(self.Ws, self.bs)):
            z = a @ W.T + b
            a = log_cosh(z) if l == 0 else np.tanh(z)
            zs.append(z)
            acts.append(a)
        return a @ self.w_out + self.b_out, zs, acts

    def logpsi(self, s):
        return self.forward(s)[0]

    def grad(self, s):
        """Reverse-mode derivative written out by hand, one sample row at a time in batch."""
        s = np.atleast_2d(np.asarray(s, dtype=np.float64))
        _, zs, acts = self.forward(s)
        S = s.shape[0]
        L = len(self.widths)
        g_w_out = acts[-1]
        g_b_out = np.ones((S, 1))
        grads = [None] * (2 * L)
        # delta_L = d out / d z_L
        delta = self.w_out[None, :] * self._dact(L - 1, zs[L - 1])
        for l in range(L - 1, -1, -1):
            grads[2 * l] = (delta[:, :, None] * acts[l][:, None, :]).reshape(S, -1)
            grads[2 * l + 1] = delta
            if l > 0:
                delta = (delta @ self.Ws[l]) * self._dact(l - 1, zs[l - 1])
        return np.concatenate(grads + [g_w_out, g_b_out], axis=1)

    @staticmethod
    def _dact(l, z):
        # layer 0 uses log cosh (derivative tanh); deeper layers use tanh (derivative 1 - tanh^2)
        return np.tanh(z) if l == 0 else 1.0 - np.tanh(z) ** 2


def make_model(kind, n_visible, params, n_hidden=0, widths=()):
    if kind == "rbm":
        return RBM(n_visible, n_hidden, params)
    if kind == "dense":
        return Dense(n_visible, widths, params)
    raise ValueError(kind)


def marshall_sign(s, sub_a):
    """(-1)^(number of up spins on sublattice A), the Marshall sign rule (reading for the
    Heisenberg workloads; the paper's App. E states no sign structure)."""
    s = np.asarray(s)
    n_up_a = ((s > 0) & sub_a[None, :]).sum(axis=-1) if s.ndim == 2 else ((s > 0) & sub_a).sum()
    return np.where(n_up_a % 2 == 0, 1.0, -1.0)
