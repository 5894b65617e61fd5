"""The default benchmark workload at its full size, in the launch configuration the bench
times: 10x10 TFIM, RBM alpha = 4, FP16 sampling copy, 16384 chains x 500 sweeps (50 burn-in),
7.37M kept samples; chain-ordered local energies on the FP32 copy, FP64 statistics and the
tensor-core force over every sample.

Checked on sampled outputs the FP64 oracle computes one by one, and on the whole arrays
where the oracle can follow:
* the untraced sweep (the bench's) equals the traced one (accept bits and increments
  recorded) state for state and sample for sample;
* sampled chains' sweeps replay in the oracle from the emitted sample before them, with the
  GPU's decisions, every decision outside 10 sigma_eps of the threshold agreeing with the
  FP64 rule (a 16-bit copy: R16), and end on the emitted sample after them;
* sampled local energies against the oracle's;
* the statistics against numpy over all 7.37M local energies;
* the force against the oracle's force over all 7.37M samples (blocked).
"""
import numpy as np
import pytest

from helpers import nqs, unpack_np, unpack_accept_bits, words_from_tensor
from oracle.estimators import local_energy as oracle_eloc, energy_stats
from oracle.hamiltonian import TFIM
from oracle.models import RBM
from oracle.sampler import mh_sweeps
import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _force_blocked(model, words, eps, N, block=50000):
    """F = mean(O (eps - E)) of the RBM over all rows, unpacking the rows block by block."""
    e = eps - eps.mean()
    Fa = np.zeros(model.N); Fb = np.zeros(model.M); FW = np.zeros((model.M, model.N))
    for b0 in range(0, len(eps), block):
        sb = unpack_np(words[b0:b0 + block], N).astype(np.float64)
        eb = e[b0:b0 + block]
        t = np.tanh(model.theta(sb))
        Fa += sb.T @ eb
        Fb += t.T @ eb
        FW += (t * eb[:, None]).T @ sb
    n = len(eps)
    return np.concatenate([Fa / n, Fb / n, (FW / n).ravel()])


def test_bench_workload_full_size_sampled_parity():
    wl = workloads.TFIM_2D_10x10
    lat = wl.ham.lattice
    N, M, C, T, B = lat.n_sites, wl.n_hidden, wl.n_chains, wl.n_sweeps, wl.burn_in
    S = (T - B) * C
    p = nqs()
    ctx = p.Context("tfim", lat.Lx, lat.Ly, J1=wl.ham.J1, h=wl.ham.h, model="rbm", n_hidden=M, dtype="f16")
    params = workloads.rbm_params(N, M, wl.weight_sigma, wl.seed)
    ctx.set_params(torch.from_numpy(params).cuda())
    W = ctx.W
    z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device="cuda")
    seed = 1000

    # the bench's calls (untraced sweep), then the same chains traced
    state, samples, nacc = z(C, W), z(S, W), z(C, dt=torch.int64)
    ctx.init_chains(state, seed)
    ctx.sweep(state, T, B, seed + 1, 0, samples, None, nacc)
    state2, samples2, nacc2 = z(C, W), z(S, W), z(C, dt=torch.int64)
    bits, delta = z(C, T, W), z(C, T, N, dt=torch.float32)
    ctx.init_chains(state2, seed)
    ctx.sweep(state2, T, B, seed + 1, 0, samples2, None, nacc2, accept_bits=bits, delta=delta)
    torch.cuda.synchronize()
    assert torch.equal(state, state2) and torch.equal(samples, samples2) and torch.equal(nacc, nacc2)
    del samples2, state2

    model = RBM(N, M, params)
    rng = np.random.default_rng(7)
    chains = rng.choice(C, 6, replace=False)
    sweeps = rng.integers(B + 1, T, 6)
    for c, t in zip(chains, sweeps):
        c, t = int(c), int(t)
        before = unpack_np(words_from_tensor(samples[(t - 1 - B) * C + c:(t - 1 - B) * C + c + 1]), N)
        after = unpack_np(words_from_tensor(samples[(t - B) * C + c:(t - B) * C + c + 1]), N)
        acc = unpack_accept_bits(words_from_tensor(bits[c:c + 1, t:t + 1]), N)
        d = delta[c:c + 1, t:t + 1].cpu().numpy().astype(np.float64)
        ref = mh_sweeps(model.logpsi, before, np.array([c]), seed + 1, 1, 0, sweep_offset=t,
                        replay_accepts=acc, tau=1.0, record_deltas=True)
        sig = (2.0 * (d - ref["deltas"])).std()
        assert sig < 0.05, sig
        mh_sweeps(model.logpsi, before, np.array([c]), seed + 1, 1, 0, sweep_offset=t,
                  replay_accepts=acc, tau=max(10 * sig, 1e-4))
        np.testing.assert_array_equal(ref["spins"], after)
    del bits, delta

    # local energies (FP32 copy), statistics, force: the bench's calls
    eloc = z(S, dt=torch.float32)
    ctx.local_energy_chains(samples, C, eloc)
    stats = z(5, dt=torch.float64)
    ctx.stats(eloc, C, stats, nacc, T * N)
    force = z(ctx.P, dt=torch.float64)
    ws = z(ctx.logpsi_grad_workspace(S), dt=torch.uint8)
    ctx.logpsi_grad(samples, None, eloc, stats, force, ws)
    torch.cuda.synchronize()
    words = words_from_tensor(samples)
    e = eloc.cpu().numpy().astype(np.float64)

    ham = TFIM(lat.Lx, lat.Ly, wl.ham.J1, wl.ham.h)
    rows = rng.choice(S, 200, replace=False)
    ref = oracle_eloc(ham, model.logpsi, unpack_np(words[rows], N))
    np.testing.assert_allclose(e[rows], ref, rtol=1e-5, atol=1e-5 * (len(ham.bonds) + N * abs(wl.ham.h)))

    # FP64 sums of 7.37M terms in another order: relative differences up to ~n 2^-53
    E, var, err = energy_stats(e, C)
    np.testing.assert_allclose(stats.cpu().numpy()[:3], [E, var, err], rtol=1e-9)

    Fref = _force_blocked(model, words, e, N)
    np.testing.assert_allclose(force.cpu().numpy(), Fref, rtol=0, atol=1e-5 * np.abs(Fref).max())


def test_batched_48_instances_full_size_against_single_context():
    """The batched workload as the bench runs it: 48 TFIM instances (N from 36 to 256, alpha
    1 / 2 / 4, 256 to 8192 chains, FP16 copies), autotuned persistent sweep and the captured
    step graph (sweep -> local energy -> statistics -> last-sweep O rows).  Four instances
    (the largest lattice, the most chains, a 1D one and one drawn at random) are run again
    through the single-context calls from the same initial chains: every output is
    bit-identical."""
    insts = workloads.batched_tfim_instances()
    T, B = insts[0].n_sweeps, insts[0].burn_in
    K = T - B
    p = nqs()
    z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device="cuda")
    items, twins = [], []
    for w in insts:
        lat = w.ham.lattice
        N, M, C = lat.n_sites, w.n_hidden, w.n_chains
        ctx = p.Context("tfim", lat.Lx, lat.Ly, J1=w.ham.J1, h=w.ham.h, model="rbm", n_hidden=M, dtype="f16")
        ctx.set_params(torch.from_numpy(workloads.rbm_params(N, M, w.weight_sigma, w.seed)).cuda())
        st = z(C, ctx.W)
        ctx.init_chains(st, w.seed + 1)
        twins.append(st.clone())
        items.append(dict(ctx=ctx, state=st, seed=w.seed + 1, samples=z(K * C, ctx.W), n_accepted=z(C, dt=torch.int64),
                          eloc=z(K * C, dt=torch.float32), stats=z(5, dt=torch.float64),
                          O=z(C, ctx.P, dt=torch.float32), N=N, C=C, oned=lat.Ly == 1))
    keys = ("ctx", "state", "seed", "samples", "n_accepted", "eloc", "stats", "O")
    b = p.Batch([{k: it[k] for k in keys} for it in items], T, B, warps_per_cta=0)
    b.step(0)
    torch.cuda.synchronize()
    picks = {max(range(48), key=lambda k: items[k]["N"]), max(range(48), key=lambda k: items[k]["C"]),
             next(k for k in range(48) if items[k]["oned"]), int(np.random.default_rng(3).integers(0, 48))}
    for k in sorted(picks):
        it, tw = items[k], twins[k]
        c, C, N = it["ctx"], it["C"], it["N"]
        r = dict(samples=z(K * C, c.W), n_accepted=z(C, dt=torch.int64), eloc=z(K * C, dt=torch.float32),
                 stats=z(5, dt=torch.float64), O=z(C, c.P, dt=torch.float32))
        c.sweep(tw, T, B, it["seed"], 0, r["samples"], None, r["n_accepted"])
        c.local_energy(r["samples"], r["eloc"])
        c.stats(r["eloc"], C, r["stats"], r["n_accepted"], T * N)
        c.logpsi_grad(r["samples"][(K - 1) * C:], r["O"])
        torch.cuda.synchronize()
        assert torch.equal(it["state"], tw), k
        for key in ("samples", "n_accepted", "eloc", "stats", "O"):
            assert torch.equal(it[key], r[key]), (k, key)
