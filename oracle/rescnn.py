"""Residual convolutional ansatz (App. H, "ResCNN"), in FP64.  Test infrastructure: only
tests, the smoke check and the benchmark's CPU baseline use it.

App. H defines the network on a two-dimensional configuration x:
  h(0) = Conv(x)                                                   (embedding)
  h(l+1) = h(l) + Conv[phi(Conv(phi(LN(h(l)))))],  l = 0 .. N_res - 1
  log psi(x) = sum over sites (i, j) and channels c of LN(h(N_res))_{ijc}
with 3 x 3 kernels, F filters and phi = GELU.

Readings where App. H is silent (each is stated once here and in the design notes):
* x is the spin configuration s in {-1, +1} on an Lx x Ly periodic lattice, site
  i = x + Lx y, as one input channel.
* Conv is a 3 x 3 cross-correlation with periodic (circular) padding and a bias per output
  channel: out[y, x, o] = b[o] + sum_{c, dy, dx} K[o, c, dy, dx] in[(y + dy - 1) mod Ly,
  (x + dx - 1) mod Lx, c].
* LN normalises the F channels of each site: (v - mean) / sqrt(var + 1e-6) (biased variance),
  then a learnable scale and shift per channel (gamma, beta); one LN per residual block and
  the final one.
* phi is the tanh form of GELU, 0.5 z (1 + tanh(sqrt(2 / pi) (z + 0.044715 z^3))), the
  default GELU of the JAX stack the paper's code uses.
* Parameters are real, so log psi is real.

Flat parameter order (FP64): [K0 (F x 1 x 3 x 3) | b0 (F) | per block: gamma (F) | beta (F) |
K1 (F x F x 3 x 3) | b1 (F) | K2 (F x F x 3 x 3) | b2 (F) | final gamma (F) | final beta (F)].

O_k(s) = d log psi(s) / d theta_k (App. I, Eq. forces) by reverse-mode differentiation
written out layer by layer.
"""
import numpy as np

LN_EPS = 1e-6
_C = np.sqrt(2.0 / np.pi)


def n_params(n_filters, n_blocks):
    F = n_filters
    return 10 * F + n_blocks * (2 * F + 2 * (9 * F * F + F)) + 2 * F


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    u = _C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3 * 0.044715 * z * z)


def conv3x3(inp, K, b):
    """Periodic 3 x 3 cross-correlation: inp [S, Ly, Lx, C], K [O, C, 3, 3], b [O] -> [S, Ly, Lx, O]."""
    out = np.broadcast_to(b, inp.shape[:3] + (K.shape[0],)).copy()
    for dy in range(3):
        for dx in range(3):
            # shifted[y, x] = inp[(y + dy - 1) mod Ly, (x + dx - 1) mod Lx]
            shifted = np.roll(inp, shift=(1 - dy, 1 - dx), axis=(1, 2))
            out += shifted @ K[:, :, dy, dx].T
    return out


def conv3x3_transpose(g, K):
    """Adjoint of the kernel part of conv3x3: d(sum g * conv(inp)) / d inp."""
    out = np.zeros(g.shape[:3] + (K.shape[1],))
    for dy in range(3):
        for dx in range(3):
            out += np.roll(g @ K[:, :, dy, dx], shift=(dy - 1, dx - 1), axis=(1, 2))
    return out


def conv3x3_kernel_grad(inp, g):
    """d(sum g * conv(inp)) / dK [O, C, 3, 3], summed over the batch axis of inp and g
    separately per sample: returns [S, O, C, 3, 3]."""
    S = inp.shape[0]
    out = np.zeros((S, g.shape[-1], inp.shape[-1], 3, 3))
    for dy in range(3):
        for dx in range(3):
            shifted = np.roll(inp, shift=(1 - dy, 1 - dx), axis=(1, 2))
            out[:, :, :, dy, dx] = np.einsum("syxo,syxc->soc", g, shifted)
    return out


def layer_norm(v, gamma, beta):
    mean = v.mean(axis=-1, keepdims=True)
    var = ((v - mean) ** 2).mean(axis=-1, keepdims=True)
    zhat = (v - mean) / np.sqrt(var + LN_EPS)
    return zhat * gamma + beta, zhat, var


def layer_norm_grad(g, zhat, var, gamma):
    """Input gradient of layer_norm for upstream g (same shape as zhat)."""
    gz = g * gamma
    return (gz - gz.mean(axis=-1, keepdims=True) - zhat * (gz * zhat).mean(axis=-1, keepdims=True)) \
        / np.sqrt(var + LN_EPS)


class ResCNN:
    def __init__(self, Lx, Ly, n_filters, n_blocks, params):
        self.Lx, self.Ly, self.F, self.n_blocks = int(Lx), int(Ly), int(n_filters), int(n_blocks)
        self.N = self.Lx * self.Ly
        p = np.asarray(params, dtype=np.float64)
        if p.size != n_params(self.F, self.n_blocks):
            raise ValueError("ResCNN parameter vector has the wrong length")
        F = self.F
        self.n_params = p.size
        off = 0

        def take(n, shape=None):
            nonlocal off
            v = p[off:off + n]
            off += n
            return v.reshape(shape) if shape else v

        self.K0 = take(9 * F, (F, 1, 3, 3))
        self.b0 = take(F)
        self.blocks = []
        for _ in range(self.n_blocks):
            g, be = take(F), take(F)
            K1, b1 = take(9 * F * F, (F, F, 3, 3)), take(F)
            K2, b2 = take(9 * F * F, (F, F, 3, 3)), take(F)
            self.blocks.append((g, be, K1, b1, K2, b2))
        self.gF, self.bF = take(F), take(F)

    def _grid(self, s):
        s = np.atleast_2d(np.asarray(s, dtype=np.float64))
        return s.reshape(s.shape[0], self.Ly, self.Lx, 1)

    def forward(self, s):
        """log psi and the intermediate values the backward pass needs."""
        x = self._grid(s)
        h = conv3x3(x, self.K0, self.b0)
        cache = []
        for (g, be, K1, b1, K2, b2) in self.blocks:
            y, zhat, var = layer_norm(h, g, be)
            a = gelu(y)
            z1 = conv3x3(a, K1, b1)
            c = gelu(z1)
            h_new = h + conv3x3(c, K2, b2)
            cache.append((h, y, zhat, var, a, z1, c))
            h = h_new
        out, zhat, var = layer_norm(h, self.gF, self.bF)
        return out.sum(axis=(1, 2, 3)), (x, cache, h, zhat, var)

    def logpsi(self, s):
        return self.forward(s)[0]

    def grad(self, s):
        """O_k(s) [S, P] in the flat parameter order."""
        _, (x, cache, h, zhat, var) = self.forward(s)
        S, F = x.shape[0], self.F
        parts_rev = []
        # final LN: d/d gamma_c = sum_sites zhat_c, d/d beta_c = N; input gradient
        parts_rev.append(np.full((S, F), float(self.N)))
        parts_rev.append(zhat.sum(axis=(1, 2)))
        gh = layer_norm_grad(np.ones_like(zhat), zhat, var, self.gF)
        for (g, be, K1, b1, K2, b2), (h_in, y, zh, vr, a, z1, c) in zip(reversed(self.blocks), reversed(cache)):
            # h_out = h_in + conv(c, K2, b2)
            dK2 = conv3x3_kernel_grad(c, gh)
            db2 = gh.sum(axis=(1, 2))
            gc = conv3x3_transpose(gh, K2)
            gz1 = gc * gelu_grad(z1)
            dK1 = conv3x3_kernel_grad(a, gz1)
            db1 = gz1.sum(axis=(1, 2))
            ga = conv3x3_transpose(gz1, K1)
            gy = ga * gelu_grad(y)
            dgamma = (gy * zh).sum(axis=(1, 2))
            dbeta = gy.sum(axis=(1, 2))
            gh = gh + layer_norm_grad(gy, zh, vr, g)
            parts_rev += [db2, dK2.reshape(S, -1), db1, dK1.reshape(S, -1), dbeta, dgamma]
        db0 = gh.sum(axis=(1, 2))
        dK0 = conv3x3_kernel_grad(x, gh)
        parts_rev += [db0, dK0.reshape(S, -1)]
        return np.concatenate(parts_rev[::-1], axis=1)
