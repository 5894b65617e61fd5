"""Natural-gradient (SR) update in the minSR form, in FP64.

The paper preconditions the force with the stochastic-reconfiguration (SR) matrix and a
diagonal shift lambda (App. I, SR paragraph: the S-matrix solve, shifts 1e-3 / 1e-1).  With
S samples the P x P matrix ObarT Obar has rank <= S, and the same update follows from an S x S
solve (the push-through identity (A^T A + l I)^-1 A^T = A^T (A A^T + l I)^-1):

    Obar  = (O - mean_x O) / sqrt(S)           [S x P]
    ebar  = (eps - E) / sqrt(S)                [S],   E = mean_x eps
    T     = Obar Obar^T                        [S x S]
    y     = (T + lambda I)^-1 ebar
    dtheta = Obar^T y                          [P]   = (Obar^T Obar + lambda I)^-1 F,  F = Obar^T ebar

Reading: the paper does not name minSR; the 16 x 16 J1-J2 workload asks for it on 4096
samples with lambda = 1e-3.  dtheta is the preconditioned force; the parameter step is
theta <- theta - eta dtheta (real parameters).
"""
import numpy as np


def centred(O, eps):
    """(Obar, ebar, E): the centred, 1/sqrt(S)-scaled rows and energies."""
    O = np.asarray(O, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    S = O.shape[0]
    E = eps.mean()
    return (O - O.mean(axis=0)) / np.sqrt(S), (eps - E) / np.sqrt(S), E


def gram(O):
    """T = Obar Obar^T of the centred rows (S x S)."""
    Ob, _, _ = centred(O, np.zeros(np.asarray(O).shape[0]))
    return Ob @ Ob.T


def minsr_update(O, eps, lam):
    """dtheta = Obar^T (Obar Obar^T + lam I)^-1 ebar, by a Cholesky solve of the S x S system."""
    Ob, eb, _ = centred(O, eps)
    T = Ob @ Ob.T
    L = np.linalg.cholesky(T + lam * np.eye(T.shape[0]))
    y = np.linalg.solve(L.T, np.linalg.solve(L, eb))
    return Ob.T @ y, y, T


def sr_update(O, eps, lam):
    """The P x P route: (Obar^T Obar + lam I)^-1 Obar^T ebar (for small P; a second route)."""
    Ob, eb, _ = centred(O, eps)
    return np.linalg.solve(Ob.T @ Ob + lam * np.eye(Ob.shape[1]), Ob.T @ eb)
