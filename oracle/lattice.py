"""Periodic lattices: bond lists and the Marshall sublattice.

Sites are numbered i = x + Lx * y.  A 1D chain is Ly == 1.  Each bond is
listed once.  Periodic boundaries need Lx >= 3 (and Ly >= 3 in 2D) so that no
bond is listed twice.

Nearest-neighbour bonds enter both Hamiltonians (TFIM, Eq. TFIM in Sec. 4.1;
Heisenberg, App. E, where "the two nearest neighbors" is read as
nearest-neighbour pairs).  Next-nearest (diagonal) bonds carry J2 of the
J1-J2 Heisenberg workload.
"""
import numpy as np


def check_lattice(Lx, Ly):
    if Lx < 3 or (Ly != 1 and Ly < 3):
        raise ValueError("periodic lattice needs Lx >= 3 and Ly == 1 or Ly >= 3")


def nn_bonds(Lx, Ly):
    check_lattice(Lx, Ly)
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            bonds.append((i, (x + 1) % Lx + Lx * y))
            if Ly > 1:
                bonds.append((i, x + Lx * ((y + 1) % Ly)))
    return np.array(bonds, dtype=np.int64)


def nnn_bonds(Lx, Ly):
    check_lattice(Lx, Ly)
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            if Ly == 1:
                bonds.append((i, (x + 2) % Lx))
            else:
                bonds.append((i, (x + 1) % Lx + Lx * ((y + 1) % Ly)))
                bonds.append((i, (x + 1) % Lx + Lx * ((y - 1) % Ly)))
    return np.array(bonds, dtype=np.int64)


def sublattice_a(Lx, Ly):
    """Boolean mask of sites with x + y even (sublattice A of the Marshall rule)."""
    xs = np.arange(Lx * Ly) % Lx
    ys = np.arange(Lx * Ly) // Lx
    return (xs + ys) % 2 == 0
