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


def round_bf16(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def bf16_copy_logpsi(params, N, widths, s):
    """log psi of the BF16 sampling copy from its definition (R19): weights and biases rounded
    to BF16 (b_out kept), layer 0 and every accumulation in higher precision, activations
    rounded to BF16 between layers, the last layer's dot with w_out unrounded."""
    m = Dense(N, widths, bf16_round_params(params, N, widths))
    a = np.asarray(s, dtype=np.float64)
    L = len(widths)
    for l in range(L):
        z = a @ m.Ws[l].T + m.bs[l]
        a = np.logaddexp(z, -z) - np.log(2.0) if l == 0 else np.tanh(z)
        if l < L - 1:
            a = round_bf16(a)
    return a @ m.w_out + m.b_out


def offdiag_abs(ham, lpf, s, sub):
    """sum over connected x' != x of |H(x, x') psi(x') / psi(x)|: the scale of the off-diagonal
    part of eps(x), which a dropped or mis-signed connected configuration moves by O(1) of."""
    from oracle.hamiltonian import Heisenberg as _H
    lp = lpf(s)
    out = np.zeros(len(s))
    if isinstance(ham, _H):
        for (i, j), J in zip(ham.bonds, ham.coupling):
            anti = s[:, i] != s[:, j]
            if not anti.any():
                continue
            y = s[anti].copy()
            y[:, i], y[:, j] = s[anti, j], s[anti, i]
            out[anti] += abs(2.0 * J) * np.exp(lpf(y) - lp[anti])
    else:
        for i in range(s.shape[1]):
            y = s.copy()
            y[:, i] = -y[:, i]
            out += abs(ham.h) * np.exp(lpf(y) - lp)
    return out


def make(Lx, Ly, widths, seed, ham="heisenberg", bias=0.1, marshall=True, J2=0.0, h=1.0):
    p = nqs()
    N = Lx * Ly
    params = dense_params(N, widths, seed, bias_sigma=bias)
    ctx = p.Context(ham, Lx, Ly, J1=1.0, J2=J2, h=h, marshall=marshall, model="dense", widths=widths, dtype="bf16")
    ctx.set_params(torch.from_numpy(params).cuda())
    return ctx, params, Dense(N, widths, bf16_round_params(params, N, widths)), Dense(N, widths, params)


@pytest.mark.parametrize("Lx,Ly,widths", [(10, 10, (400, 400)), (4, 4, (64, 48)), (6, 6, (128, 96, 64)),
                                          (16, 1, (1024, 512)), (16, 16, (1024, 1024, 1024))])
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


@pytest.mark.parametrize("Lx,Ly,widths,ham,J2,n", [(10, 10, (400, 400), "heisenberg", 0.0, 300),
                                                   (4, 4, (64, 48), "heisenberg", 0.5, 300),
                                                   (6, 1, (32, 32), "tfim", 0.0, 300),
                                                   (16, 16, (1024, 1024, 1024), "heisenberg", 0.5, 256)])
def test_dense_local_energy_matches_oracle(Lx, Ly, widths, ham, J2, n):
    """Against the BF16 copy's definition with its rounding points (bf16_copy_logpsi): within
    1e-3 of the summed off-diagonal magnitudes, which a dropped or mis-signed connected
    configuration (O(1) of that sum over up to 1024 terms) would exceed.  (16 x 16, 1024^3,
    J2 = 0.5: the J1-J2 workload's network; up to 1024 connected configurations per sample.)"""
    ctx, params, m_r, _ = make(Lx, Ly, widths, 5, ham=ham, J2=J2)
    N = Lx * Ly
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
    lpf = lambda v: bf16_copy_logpsi(params, N, widths, v)
    ref = oracle_eloc(oh, lpf, s, sub_a=sub)
    scale = offdiag_abs(oh, lpf, s, sub)
    err = np.abs(e.cpu().numpy() - ref)
    assert np.all(err <= 1e-3 * scale + 1e-4 * np.abs(ref) + 1e-4), (err / scale).max()
    # the same check against the FP64 network (BF16 parameters, unrounded activations) would not
    # hold at this tolerance: the emulation resolves the copy's activation rounding
    ref64 = oracle_eloc(oh, m_r.logpsi, s, sub_a=sub)
    assert np.median(np.abs(ref64 - ref) / scale) > 3 * np.median(err / scale)


@pytest.mark.parametrize("Lx,Ly,widths,J2,dtype,T,C", [(10, 10, (400, 400), 0.0, "bf16", 1, 8192),
                                                       (10, 10, (400, 400), 0.0, "fp8", 1, 8192),
                                                       (16, 16, (1024, 1024, 1024), 0.5, "bf16", 1, 8192),
                                                       (16, 16, (1024, 1024, 1024), 0.5, "fp8", 1, 8192),
                                                       (16, 16, (1024, 1024, 1024), 0.5, "bf16", 1, 65536)])
def test_dense_sampler_replays_at_workload_shapes(Lx, Ly, widths, J2, dtype, T, C):
    """The exchange sampler at the workloads' shapes (10 x 10 with 400 x 400, in BF16 and FP8:
    the fused sampler; the 16 x 16 J1-J2 network 1024^3 in BF16 and FP8) with 8192 chains, and with the J1-J2 workload's
    65,536 (whose products take the two-row-tile GEMM configuration); a sampled subset of
    chains is replayed in the oracle against the copy's own definition: every decision
    outside 10 sigma of the increment error agrees, and the final configurations of those
    chains are reproduced."""
    from oracle.lattice import nn_bonds, nnn_bonds
    N = Lx * Ly
    if dtype == "fp8":
        ctx, params = make_fp8(Lx, Ly, widths, 17, J2=J2)
        lpf = lambda v: fp8_copy_logpsi(params, N, widths, v)
    else:
        ctx, params, _, _ = make(Lx, Ly, widths, 17, J2=J2)
        lpf = lambda v: bf16_copy_logpsi(params, N, widths, v)
    W = ctx.W
    state = torch.zeros((C, W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 31)
    s0 = unpack_np(words_from_tensor(state), N)
    bits = torch.zeros((C, T, W), dtype=torch.int32, device="cuda")
    delta = torch.zeros((C, T, N), dtype=torch.float32, device="cuda")
    ctx.sweep(state, T, T, 32, 0, None, None, None, accept_bits=bits, delta=delta)
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    final = unpack_np(words_from_tensor(state), N)
    sub = np.unique(np.concatenate([np.arange(3), np.random.default_rng(5).choice(C, 5, replace=False)]))
    bonds = nn_bonds(Lx, Ly) if J2 == 0.0 else np.concatenate([nn_bonds(Lx, Ly), nnn_bonds(Lx, Ly)])
    ref = mh_sweeps(lpf, s0[sub], sub, 32, T, T, proposal="exchange", bonds=bonds, replay_accepts=acc[sub],
                    tau=10.0, record_deltas=True)
    d = delta.cpu().numpy().astype(np.float64)[sub]
    moved = ref["deltas"] != 0
    sig = (2.0 * (d - ref["deltas"]))[moved].std()
    mh_sweeps(lpf, s0[sub], sub, 32, T, T, proposal="exchange", bonds=bonds, replay_accepts=acc[sub],
              tau=max(10 * sig, 1e-4))
    np.testing.assert_array_equal(final[sub], ref["spins"])
    assert np.all(final.sum(axis=1) == 0)


@pytest.mark.parametrize("fused", [1, 0])
def test_dense_exchange_sampler_replays_in_oracle(fused):
    """4 x 4 Heisenberg: every decision of the BF16 sampler agrees with the FP64 rule outside
    a band of 10 sigma of its increment error; magnetisation stays zero.  fused = 1: the
    persistent fused sampler (the default for two hidden layers); 0: the multi-launch one."""
    ctx, _, m_r, _ = make(4, 4, (64, 48), 7, bias=0.2)
    ctx.set_option(nqs().OPT_DENSE_FUSED, fused)
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


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_dense_fused_sampler_independent_of_tiling(dtype):
    """The fused sampler at the 10 x 10, 400 x 400 shape (BF16 and FP8 copies): a chain's
    draws, products and sums do not depend on how many chains share its CTA or on its row in
    the tile, so 20000 chains (tiles of 128, more than one tile per CTA), 8192 (tiles of 56)
    and 1000 (tiles of 7) give bit-identical samples, log psi, acceptance counts and
    increments for the chains they share."""
    ctx = make(10, 10, (400, 400), 23)[0] if dtype == "bf16" else make_fp8(10, 10, (400, 400), 23)[0]
    W, N, T, B = ctx.W, 100, 3, 1
    out = {}
    for C in (20000, 8192, 1000):
        state = torch.zeros((C, W), dtype=torch.int32, device="cuda")
        ctx.init_chains(state, 41)
        samples = torch.zeros(((T - B) * C, W), dtype=torch.int32, device="cuda")
        logpsi = torch.zeros((T - B) * C, dtype=torch.float32, device="cuda")
        nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
        delta = torch.zeros((C, T, N), dtype=torch.float32, device="cuda")
        ctx.sweep(state, T, B, 42, 0, samples, logpsi, nacc, delta=delta)
        torch.cuda.synchronize()
        out[C] = (state.cpu(), samples.cpu().view(T - B, C, W), logpsi.cpu().view(T - B, C), nacc.cpu(), delta.cpu())
    ref = out[20000]
    for C in (8192, 1000):
        got = out[C]
        assert torch.equal(got[0], ref[0][:C])
        assert torch.equal(got[1], ref[1][:, :C])
        assert torch.equal(got[2], ref[2][:, :C])
        assert torch.equal(got[3], ref[3][:C])
        assert torch.equal(got[4], ref[4][:C])
    assert ref[3].sum().item() > 0


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_dense_fused_flip_sampler_replays_in_oracle(dtype):
    """4 x 4 TFIM with two hidden layers (the fused sampler, flip moves: the proposal adds
    -+2 times a row of the copy's layer-0 weights): every decision agrees with the MH rule on
    the copy's own log psi (bf16_copy_logpsi / fp8_copy_logpsi) outside 10 sigma of the
    increment error, and the final configurations and samples are reproduced."""
    widths = (64, 48)
    if dtype == "fp8":
        ctx, params = make_fp8(4, 4, widths, 13, ham="tfim", bias=0.2)
        lpf = lambda v: fp8_copy_logpsi(params, 16, widths, v)
    else:
        ctx, params, _, _ = make(4, 4, widths, 13, ham="tfim", bias=0.2, marshall=False)
        lpf = lambda v: bf16_copy_logpsi(params, 16, widths, v)
    C, T = 256, 3
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 19)
    s0 = unpack_np(words_from_tensor(state), 16)
    bits = torch.zeros((C, T, 1), dtype=torch.int32, device="cuda")
    delta = torch.zeros((C, T, 16), dtype=torch.float32, device="cuda")
    samples = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, T - 1, 14, 0, samples, None, None, accept_bits=bits, delta=delta)
    acc = unpack_accept_bits(words_from_tensor(bits), 16)
    ref = mh_sweeps(lpf, s0, np.arange(C), 14, T, T - 1, proposal="flip", replay_accepts=acc, tau=10.0,
                    record_deltas=True)
    d = delta.cpu().numpy().astype(np.float64)
    sig = (2.0 * (d - ref["deltas"])).std()
    assert sig < 0.05, sig
    mh_sweeps(lpf, s0, np.arange(C), 14, T, T - 1, proposal="flip", replay_accepts=acc, tau=max(10 * sig, 1e-4))
    np.testing.assert_array_equal(unpack_np(words_from_tensor(state), 16), ref["spins"])
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), 16), ref["samples"])
    assert acc.mean() > 0.05


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


# ---------------------------------------------------------------------------------------
# FP8 (E4M3) sampling copy: weights W_l in E4M3 scaled by s_l = 2^floor(log2(448 / max|W_l|)),
# biases and w_out as in the BF16 copy, E4M3 activations between layers; the local energy runs
# on the BF16 copy.

def _e4m3(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.float8_e4m3fn).double().numpy()


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def fp8_copy_logpsi(params, N, widths, s):
    """log psi of the FP8 copy, written from its definition in FP64 with every quantisation
    point of the copy (E4M3 weights with the per-layer power-of-two scale, E4M3 activations
    into layers 1 .. L-1, BF16 biases and w_out)."""
    m = Dense(N, widths, params)
    Wq = []
    for W in m.Ws:
        sc = 2.0 ** np.floor(np.log2(448.0 / np.abs(W).max()))
        Wq.append(_e4m3(W * sc) / sc)
    a = np.asarray(s, dtype=np.float64)
    L = len(widths)
    for l in range(L):
        z = a @ Wq[l].T + _bf16(m.bs[l])
        a = np.logaddexp(z, -z) - np.log(2.0) if l == 0 else np.tanh(z)
        if l < L - 1:
            a = _e4m3(a)
    return a @ _bf16(m.w_out) + m.b_out


def make_fp8(Lx, Ly, widths, seed, ham="heisenberg", bias=0.1, J2=0.0):
    p = nqs()
    N = Lx * Ly
    params = dense_params(N, widths, seed, bias_sigma=bias)
    ctx = p.Context(ham, Lx, Ly, J1=1.0, J2=J2, h=1.0, marshall=(ham == "heisenberg"), model="dense",
                    widths=widths, dtype="fp8")
    ctx.set_params(torch.from_numpy(params).cuda())
    return ctx, params


@pytest.mark.parametrize("Lx,Ly,widths,n", [(10, 10, (400, 400), 1000), (4, 4, (64, 48), 1000),
                                            (6, 6, (128, 96, 64), 1000), (16, 1, (1024, 512), 1000),
                                            (16, 16, (1024, 1024, 1024), 1000), (16, 16, (1024, 1024, 1024), 20000)])
def test_dense_fp8_logpsi_matches_its_definition(Lx, Ly, widths, n):
    """The FP8 copy's log psi against its FP64 definition with the same quantisation points.
    What remains are single-ulp E4M3 flips of activations that lie within the MUFU
    tanh / log cosh error of a rounding boundary (about 1 % of them); an error anywhere in the
    quantised path (scale, byte order, K blocking) moves log psi by O(1).  20000 rows of the
    1024^3 network take the layer products' two-row-tile configuration (ragged last pair)."""
    ctx, params = make_fp8(Lx, Ly, widths, 3)
    N = Lx * Ly
    s = np.random.default_rng(1).choice([-1, 1], size=(n, N)).astype(np.int8)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.logpsi(to_words_tensor(pack_np(s)), out)
    got = out.cpu().numpy().astype(np.float64)
    d = got - fp8_copy_logpsi(params, N, widths, s)
    full = np.abs(got - Dense(N, widths, params).logpsi(s))
    assert np.abs(d).mean() < 0.02 and np.abs(d).max() < 0.15, (np.abs(d).mean(), np.abs(d).max())
    assert np.abs(d).mean() < 0.25 * full.mean(), (np.abs(d).mean(), full.mean())  # the quantisation is resolved


def test_dense_fp8_sampler_targets_its_distribution():
    """4 x 4 Heisenberg, FP8 copy: the sampled energy equals the exact expectation under the
    FP8 copy's own distribution pi~ = |psi~|^2 (enumerated through the context's log psi over
    the zero-magnetisation sector) within 4 sigma of the Monte Carlo error; each recorded
    decision follows the MH rule on the sampler's increment; magnetisation stays zero."""
    ctx, params = make_fp8(4, 4, (64, 48), 21, bias=0.2)
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
    sec = allc[allc.sum(axis=1) == 0]
    cfg = to_words_tensor(pack_np(sec.astype(np.int8)))
    lp = torch.empty(len(sec), dtype=torch.float32, device="cuda")
    ctx.logpsi(cfg, lp)
    es = torch.empty(len(sec), dtype=torch.float32, device="cuda")
    ctx.local_energy(cfg, es)
    w = 2.0 * lp.cpu().numpy().astype(np.float64)
    pi = np.exp(w - w.max())
    pi /= pi.sum()
    e_exact = pi @ es.cpu().numpy().astype(np.float64)
    assert abs(E - e_exact) <= 4 * err, (E, e_exact, err)
    assert np.all(unpack_np(words_from_tensor(state), 16).sum(axis=1) == 0)
    # decisions against the recorded increments and the Philox thresholds
    C2, T2 = 128, 2
    st2 = torch.zeros((C2, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(st2, 9)
    bits = torch.zeros((C2, T2, 1), dtype=torch.int32, device="cuda")
    delta = torch.zeros((C2, T2, 16), dtype=torch.float32, device="cuda")
    ctx.sweep(st2, T2, T2 - 1, 10, 0, torch.zeros((C2, 1), dtype=torch.int32, device="cuda"), None, None,
              accept_bits=bits, delta=delta)
    acc = unpack_accept_bits(words_from_tensor(bits), 16)
    d = delta.cpu().numpy().astype(np.float64)
    from oracle.lattice import nn_bonds
    from oracle.philox import sweep_draws
    n_checked = 0
    for t in range(T2):
        _, u = sweep_draws(10, np.arange(C2), t, 16, len(nn_bonds(4, 4)))
        with np.errstate(divide="ignore"):
            margin = 2.0 * d[:, t, :] - np.log(u)
        real = (d[:, t, :] != 0.0) & (np.abs(margin) > 1e-5)   # moved, outside FP32 rounding of log u
        np.testing.assert_array_equal(acc[:, t, :][real], margin[real] > 0)
        n_checked += int(real.sum())
    assert n_checked > 1000, n_checked
