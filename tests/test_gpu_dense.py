"""Dense feed-forward ansatz on the tensor cores (BF16 sampling copy, FP32 accumulation)
against the FP64 oracle: log psi, Heisenberg / TFIM local energies, the exchange-move
sampler (replayed in the oracle), and the FP32 O_k / force.

The oracle evaluates the network with the same BF16-rounded parameters the sampling copy
uses, so the remaining difference is the BF16 rounding of the activations between layers:
about 2^-9 per activation, i.e. a few 1e-3 in log psi for 400-wide layers (tolerances below).
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, unpack_np, unpack_accept_bits, to_words_tensor, words_from_tensor
from oracle import exact
from oracle.estimators import local_energy as oracle_eloc, force as oracle_force
from oracle.hamiltonian import TFIM, Heisenberg
from oracle.lattice import sublattice_a
from oracle.models import Dense
from oracle.philox import init_spins_balanced
from oracle.sampler import mh_sweeps
from workloads import dense_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16_round_params(p, N, widths):
    """The sampling copy: every weight and bias rounded to BF16 except b_out."""
    q = torch.from_numpy(p).to(torch.bfloat16).double().numpy()
    q[-1] = p[-1]
    return q


def make(Lx, Ly, widths, seed, ham="heisenberg", bias=0.1, marshall=True, J2=0.0, h=1.0):
    p = nqs()
    N = Lx * Ly
    params = dense_params(N, widths, seed, bias_sigma=bias)
    ctx = p.Context(ham, Lx, Ly, J1=1.0, J2=J2, h=h, marshall=marshall, model="dense", widths=widths, dtype="bf16")
    ctx.set_params(torch.from_numpy(params).cuda())
    return ctx, params, Dense(N, widths, bf16_round_params(params, N, widths)), Dense(N, widths, params)


@pytest.mark.parametrize("Lx,Ly,widths", [(10, 10, (400, 400)), (4, 4, (64, 48)), (6, 6, (128, 96, 64)),
                                          (16, 1, (1024, 512))])
def test_dense_logpsi_matches_oracle(Lx, Ly, widths):
    ctx, _, m_r, _ = make(Lx, Ly, widths, 3)
    N = Lx * Ly
    n = 1000
    s = np.random.default_rng(1).choice([-1, 1], size=(n, N)).astype(np.int8)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.logpsi(to_words_tensor(pack_np(s)), out)
    d = out.cpu().numpy() - m_r.logpsi(s)
    assert np.abs(d).max() < 0.05, np.abs(d).max()
    assert np.abs(d).mean() < 0.01, np.abs(d).mean()


@pytest.mark.parametrize("Lx,Ly,widths,ham,J2", [(10, 10, (400, 400), "heisenberg", 0.0), (4, 4, (64, 48), "heisenberg", 0.5),
                                                 (6, 1, (32, 32), "tfim", 0.0)])
def test_dense_local_energy_matches_oracle(Lx, Ly, widths, ham, J2):
    ctx, _, m_r, _ = make(Lx, Ly, widths, 5, ham=ham, J2=J2)
    N = Lx * Ly
    n = 300
    rng = np.random.default_rng(2)
    if ham == "heisenberg":
        s = init_spins_balanced(9, np.arange(n), N)
        oh = Heisenberg(Lx, Ly, 1.0, J2)
        sub = sublattice_a(Lx, Ly)
    else:
        s = rng.choice([-1, 1], size=(n, N)).astype(np.int8)
        oh = TFIM(Lx, Ly, 1.0, 1.0)
        sub = None
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.local_energy(to_words_tensor(pack_np(s)), e)
    ref = oracle_eloc(oh, m_r.logpsi, s, sub_a=sub)
    # scale: the size of the off-diagonal sum (ratios carry the log psi rounding)
    scale = np.abs(ref) + 2.0 * len(oh.bonds) if ham == "heisenberg" else np.abs(ref) + N
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 0.03 * scale), np.abs(e.cpu().numpy() - ref).max()


def test_dense_exchange_sampler_replays_in_oracle():
    """4 x 4 Heisenberg: every decision of the BF16 sampler agrees with the FP64 rule outside
    a band of 10 sigma of its increment error; magnetisation stays zero."""
    ctx, _, m_r, _ = make(4, 4, (64, 48), 7, bias=0.2)
    C, T = 256, 3
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 11)
    s0 = unpack_np(words_from_tensor(state), 16)
    assert np.all(s0.sum(axis=1) == 0)
    np.testing.assert_array_equal(s0, init_spins_balanced(11, np.arange(C), 16))
    bits = torch.zeros((C, T, 1), dtype=torch.int32, device="cuda")
    delta = torch.zeros((C, T, 16), dtype=torch.float32, device="cuda")
    samples = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, T - 1, 12, 0, samples, None, None, accept_bits=bits, delta=delta)
    acc = unpack_accept_bits(words_from_tensor(bits), 16)
    from oracle.lattice import nn_bonds
    bonds = nn_bonds(4, 4)
    ref = mh_sweeps(m_r.logpsi, s0, np.arange(C), 12, T, T - 1, proposal="exchange", bonds=bonds,
                    replay_accepts=acc, tau=1.0, record_deltas=True)
    d = delta.cpu().numpy().astype(np.float64)
    moved = ref["deltas"] != 0
    eps = 2.0 * (d - ref["deltas"])[moved]
    sig = eps.std()
    assert sig < 0.05, sig
    mh_sweeps(m_r.logpsi, s0, np.arange(C), 12, T, T - 1, proposal="exchange", bonds=bonds,
              replay_accepts=acc, tau=max(10 * sig, 1e-4))
    final = unpack_np(words_from_tensor(state), 16)
    np.testing.assert_array_equal(final, ref["spins"])
    assert np.all(final.sum(axis=1) == 0)
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), 16), ref["samples"])


@pytest.mark.parametrize("Lx,Ly,widths", [(4, 4, (64, 48)), (10, 10, (400, 400))])
def test_dense_grad_and_force_match_oracle(Lx, Ly, widths):
    ctx, params, _, m = make(Lx, Ly, widths, 13)
    N = Lx * Ly
    n = 64
    s = init_spins_balanced(3, np.arange(n), N)
    cfg = to_words_tensor(pack_np(s))
    O = torch.empty((n, ctx.P), dtype=torch.float32, device="cuda")
    eloc = torch.from_numpy(np.random.default_rng(5).normal(-40.0, 3.0, n).astype(np.float32)).cuda()
    stats = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(eloc, n, stats)
    force = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    ctx.logpsi_grad(cfg, O, eloc, stats, force)
    Oref = m.grad(s)
    np.testing.assert_allclose(O.cpu().numpy(), Oref, rtol=1e-4, atol=1e-5)
    Fref = oracle_force(Oref, eloc.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(force.cpu().numpy(), Fref, rtol=0, atol=1e-4 * np.abs(Fref).max())
    # force without materialised rows (chunked through the context's scratch)
    f2 = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    ctx.logpsi_grad(cfg, None, eloc, stats, f2)
    np.testing.assert_allclose(f2.cpu().numpy(), force.cpu().numpy(), rtol=1e-10, atol=1e-12)


def test_dense_heisenberg_4x4_energy_against_enumeration():
    """Sampled energy of a BF16 dense ansatz on the 4 x 4 Heisenberg model vs the exact
    expectation (zero-magnetisation sector, Marshall sign) within MC error + bias bound."""
    ctx, _, m_r, _ = make(4, 4, (64, 48), 21, bias=0.2)
    C, T, B = 2048, 40, 10
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 5)
    S = torch.zeros(((T - B) * C, 1), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, B, 6, 0, S)
    e = torch.empty((T - B) * C, dtype=torch.float32, device="cuda")
    ctx.local_energy(S, e)
    st = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.stats(e, C, st)
    E, var, err = st.cpu().numpy()[:3]
    allc = exact.all_configs(16)
    sector = allc.sum(axis=1) == 0
    ham = Heisenberg(4, 4, 1.0)
    pi = exact.exact_pi(m_r.logpsi, 16, mask=sector)
    eps_all = np.zeros(len(allc))
    eps_all[sector] = oracle_eloc(ham, m_r.logpsi, allc[sector], sub_a=sublattice_a(4, 4))
    e_exact = pi @ eps_all
    # the GPU evaluates the BF16 copy with BF16 activations: allow 5 % of |E| for that bias
    assert abs(E - e_exact) <= 4 * err + 0.05 * abs(e_exact), (E, e_exact, err)
