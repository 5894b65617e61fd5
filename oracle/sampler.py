"""Metropolis-Hastings sampling of pi(x) ~ |psi(x)|^2 by full re-evaluation, in FP64.

Follows Sec. 3.1 (Eq. unperturbed acceptance rate): a proposal x -> y drawn
from a symmetric q is accepted with probability min{1, exp(log pi(y) - log pi(x))},
log pi = 2 log psi.  The move is accepted iff u < exp(2 (log psi(y) - log psi(x)))
with u uniform in [0, 1) (strict '<', so u = 0 always accepts).

Proposals:
  * single-spin flip (App. C, Eq. app:local_prop): site i uniform in {0..N-1};
  * exchange (App. E): a uniform bond of the Hamiltonian's bond list, whose two
    spins are swapped.  Equal spins give y = x: ratio 1, always accepted.
Readings (the paper is silent): a sweep is N proposals per chain; one sample is
recorded per chain after each sweep once `burn_in` sweeps have passed.
Samples are returned sweep-major: row r = k * C + c for kept sweep k, chain c.

Lockstep replay: given the accept decisions of another implementation, every
decision is checked (they must agree unless |2 dlogpsi - log u| <= tau) and the
given decision is then adopted, so that both trajectories stay identical.
"""
import numpy as np

from .philox import sweep_draws


class ReplayMismatch(AssertionError):
    pass


def propose(s, idx, kind, bonds=None):
    """Apply proposal idx (site or bond) to every chain; returns y."""
    y = s.copy()
    rows = np.arange(s.shape[0])
    if kind == "flip":
        y[rows, idx] = -s[rows, idx]
    else:
        i, j = bonds[idx, 0], bonds[idx, 1]
        y[rows, i] = s[rows, j]
        y[rows, j] = s[rows, i]
    return y


def mh_sweeps(logpsi_fn, spins0, chain_ids, seed, n_sweeps, burn_in, proposal="flip",
              bonds=None, sweep_offset=0, replay_accepts=None, tau=1e-4, record_deltas=False):
    """Run n_sweeps sweeps of MH on every chain.

    spins0 [C, N] int8 (+-1); chain_ids [C] (the chain index used in the Philox counter).
    replay_accepts: optional bool array [C, n_sweeps, N] of another implementation's decisions.
    Returns a dict with spins, samples [K*C, N], logpsi [K*C], n_accepted [C],
    near_threshold (decisions inside tau that disagreed), and optionally deltas [C, n_sweeps, N].
    """
    s = np.array(spins0, dtype=np.int8, copy=True)
    C, N = s.shape
    n_choices = N if proposal == "flip" else len(bonds)
    lp = logpsi_fn(s)
    n_acc = np.zeros(C, dtype=np.int64)
    keep_s, keep_lp = [], []
    deltas = np.zeros((C, n_sweeps, N)) if record_deltas else None
    near, checked = 0, 0
    for t in range(n_sweeps):
        idx, u = sweep_draws(seed, chain_ids, sweep_offset + t, N, n_choices)
        for p in range(N):
            y = propose(s, idx[:, p], proposal, bonds)
            lp_y = logpsi_fn(y)
            delta = lp_y - lp
            with np.errstate(over="ignore"):
                acc = (u[:, p] == 0.0) | (u[:, p] < np.exp(2.0 * delta))
            if record_deltas:
                deltas[:, t, p] = delta
            if replay_accepts is not None:
                other = replay_accepts[:, t, p].astype(bool)
                differ = other != acc
                if np.any(differ):
                    with np.errstate(divide="ignore"):
                        margin = np.abs(2.0 * delta - np.log(u[:, p]))
                    bad = differ & (margin > tau)
                    if np.any(bad):
                        c = int(np.flatnonzero(bad)[0])
                        raise ReplayMismatch(
                            f"chain {c} sweep {t} step {p}: decision differs with margin {margin[c]:.3e} > tau")
                    near += int(differ.sum())
                checked += C
                acc = other
            s = np.where(acc[:, None], y, s)
            lp = np.where(acc, lp_y, lp)
            n_acc += acc
        if t >= burn_in:
            keep_s.append(s.copy())
            keep_lp.append(lp.copy())
    out = {
        "spins": s,
        "samples": np.concatenate(keep_s) if keep_s else np.zeros((0, N), np.int8),
        "logpsi": np.concatenate(keep_lp) if keep_lp else np.zeros(0),
        "n_accepted": n_acc,
        "near_threshold": near,
        "checked": checked,
    }
    if record_deltas:
        out["deltas"] = deltas
    return out
