"""Hamiltonian matrix elements H(x, x') and connected sets C(x), in FP64.

TFIM (Sec. 4.1, Eq. TFIM): H = J sum_<ij> sz_i sz_j + h sum_i sx_i, with +h as
printed.  C(x) = {x} and the N single flips; H(x, x) = J sum_<ij> s_i s_j and
H(x, flip_i x) = h.

Heisenberg (App. E): H = J1 sum_<ij> sigma_i . sigma_j (+ J2 sum_<<ij>> for the
J1-J2 workload), Pauli matrices.  Diagonal J s_i s_j on every bond; each
anti-aligned bond (s_i != s_j) connects x to the configuration with s_i and
s_j exchanged, with matrix element 2J.
"""
import numpy as np

from .lattice import nn_bonds, nnn_bonds


class TFIM:
    def __init__(self, Lx, Ly, J, h):
        self.bonds = nn_bonds(Lx, Ly)
        self.N = Lx * Ly
        self.J, self.h = float(J), float(h)

    def diagonal(self, s):
        s = np.asarray(s, dtype=np.float64)
        return self.J * (s[..., self.bonds[:, 0]] * s[..., self.bonds[:, 1]]).sum(axis=-1)

    def connected(self, s):
        """Off-diagonal part of C(x) for one configuration: list of (x', H(x, x'))."""
        out = []
        for i in range(self.N):
            y = np.array(s, copy=True)
            y[i] = -y[i]
            out.append((y, self.h))
        return out


class Heisenberg:
    def __init__(self, Lx, Ly, J1, J2=0.0):
        self.N = Lx * Ly
        nn = nn_bonds(Lx, Ly)
        bonds, coup = [nn], [np.full(len(nn), float(J1))]
        if J2 != 0.0:
            nnn = nnn_bonds(Lx, Ly)
            bonds.append(nnn)
            coup.append(np.full(len(nnn), float(J2)))
        self.bonds = np.concatenate(bonds)
        self.coupling = np.concatenate(coup)

    def diagonal(self, s):
        s = np.asarray(s, dtype=np.float64)
        zz = s[..., self.bonds[:, 0]] * s[..., self.bonds[:, 1]]
        return (zz * self.coupling).sum(axis=-1)

    def connected(self, s):
        out = []
        for (i, j), J in zip(self.bonds, self.coupling):
            if s[i] != s[j]:
                y = np.array(s, copy=True)
                y[i], y[j] = s[j], s[i]
                out.append((y, 2.0 * J))
        return out


def make_hamiltonian(ham):
    """Build from a workloads.Hamiltonian description."""
    lat = ham.lattice
    if ham.kind == "tfim":
        return TFIM(lat.Lx, lat.Ly, ham.J1, ham.h)
    if ham.kind == "heisenberg":
        return Heisenberg(lat.Lx, lat.Ly, ham.J1, ham.J2)
    raise ValueError(ham.kind)
