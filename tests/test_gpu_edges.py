"""Edge cases of the RBM / TFIM path on the GPU:

* empty calls (no chains, no sweeps, no samples) change nothing and return OK; the force of
  no samples is zero;
* the largest RBM sizes: N = 256 sites (8 words per configuration) with M = 1024 hidden units
  (32 per lane), 1D and 2D, sweeps replayed in the FP64 oracle and local energies against it;
  N = 257 is rejected at creation;
* degenerate wave functions with closed forms: a uniform psi (W = 0, a = 0) accepts every
  proposal and has eps(x) = J sum s_i s_j + h N exactly; a product state (W = 0) has
  <s_i> = tanh(2 a_i); h = 0 leaves only the diagonal;
* the smallest lattice (a ring of 3 sites) and a single chain.
"""
import numpy as np
import pytest

from helpers import nqs, pack_np, unpack_np, unpack_accept_bits, to_words_tensor, words_from_tensor
from oracle.estimators import local_energy as oracle_eloc
from oracle.hamiltonian import TFIM
from oracle.models import RBM
from oracle.sampler import mh_sweeps
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ctx_with(Lx, Ly, M, params, h=1.0, J=1.0, dtype="f32"):
    c = nqs().Context("tfim", Lx, Ly, J1=J, h=h, model="rbm", n_hidden=M, dtype=dtype)
    c.set_params(torch.from_numpy(np.asarray(params, dtype=np.float64)).cuda())
    return c


def test_empty_calls_are_no_ops():
    c = ctx_with(8, 1, 8, rbm_params(8, 8, 0.2, 1))
    st = torch.zeros((5, 1), dtype=torch.int32, device="cuda")
    c.init_chains(st, 3)
    before = st.clone()
    c.sweep(st, 0, 0, 1, 0)                                    # no sweeps
    assert torch.equal(st, before)
    empty = torch.zeros((0, 1), dtype=torch.int32, device="cuda")
    c.sweep(empty, 3, 1, 1, 0)                                 # no chains
    e = torch.zeros(0, dtype=torch.float32, device="cuda")
    c.local_energy(empty, e)
    c.logpsi(empty, e)
    c.local_energy_chains(empty, 1, e)
    stats = torch.zeros(5, dtype=torch.float64, device="cuda")
    force = torch.full((c.P,), 7.0, dtype=torch.float64, device="cuda")
    c.logpsi_grad(empty, None, e, stats, force)
    assert torch.count_nonzero(force).item() == 0             # the force of no samples is zero
    c.check_status()


@pytest.mark.parametrize("Lx,Ly", [(256, 1), (16, 16)])
def test_largest_lattice_and_hidden_layer(Lx, Ly):
    N, M, C, T = Lx * Ly, 1024, 3, 2
    params = rbm_params(N, M, 0.02, 17)
    c = ctx_with(Lx, Ly, M, params, h=0.8)
    assert c.W == 8
    with pytest.raises(nqs().NQSError):
        nqs().Context("tfim", 257, 1, J1=1.0, h=1.0, model="rbm", n_hidden=M)
    model = RBM(N, M, params)
    st = torch.zeros((C, c.W), dtype=torch.int32, device="cuda")
    c.init_chains(st, 5)
    s0 = unpack_np(words_from_tensor(st), N)
    bits = torch.zeros((C, T, c.W), dtype=torch.int32, device="cuda")
    c.sweep(st, T, 0, 6, 0, accept_bits=bits)
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    ref = mh_sweeps(model.logpsi, s0, np.arange(C), 6, T, 0, replay_accepts=acc, tau=1e-4)
    np.testing.assert_array_equal(unpack_np(words_from_tensor(st), N), ref["spins"])
    e = torch.empty(C, dtype=torch.float32, device="cuda")
    c.local_energy(st, e)
    eref = oracle_eloc(TFIM(Lx, Ly, 1.0, 0.8), model.logpsi, ref["spins"])
    np.testing.assert_allclose(e.cpu().numpy(), eref, rtol=0, atol=1e-4 * (np.abs(eref).max() + N))


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_uniform_psi_accepts_everything_and_has_closed_form_energy(dtype):
    Lx, Ly, M, C, T = 6, 6, 36, 512, 5
    N = Lx * Ly
    c = ctx_with(Lx, Ly, M, np.zeros(N + M + M * N), h=1.7, J=0.6, dtype=dtype)
    st = torch.zeros((C, c.W), dtype=torch.int32, device="cuda")
    c.init_chains(st, 2)
    S = torch.zeros((T * C, c.W), dtype=torch.int32, device="cuda")
    nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
    c.sweep(st, T, 0, 3, 0, S, None, nacc)
    assert int(nacc.sum().item()) == C * T * N                 # every proposal accepted
    e = torch.empty(T * C, dtype=torch.float32, device="cuda")
    c.local_energy(S, e)
    s = unpack_np(words_from_tensor(S), N).astype(np.float64)
    ham = TFIM(Lx, Ly, 0.6, 1.7)
    exact = ham.diagonal(s) + 1.7 * N
    np.testing.assert_allclose(e.cpu().numpy(), exact, rtol=0, atol=1e-4 * N)


def test_product_state_magnetisation():
    N, M, C, T, B = 12, 12, 4096, 60, 10
    a = np.linspace(-0.4, 0.5, N)
    c = ctx_with(N, 1, M, np.concatenate([a, np.zeros(M + M * N)]))
    st = torch.zeros((C, c.W), dtype=torch.int32, device="cuda")
    c.init_chains(st, 8)
    S = torch.zeros(((T - B) * C, c.W), dtype=torch.int32, device="cuda")
    c.sweep(st, T, B, 9, 0, S)
    s = unpack_np(words_from_tensor(S), N).astype(np.float64)
    m = s.reshape(T - B, C, N).mean(axis=0)                    # per-chain magnetisation (independent chains)
    err = m.std(axis=0) / np.sqrt(C)
    np.testing.assert_array_less(np.abs(m.mean(axis=0) - np.tanh(2 * a)), 5 * err + 1e-3)


def test_zero_field_leaves_the_diagonal_and_smallest_ring():
    N, M = 3, 5
    params = rbm_params(N, M, 0.4, 4)
    c = ctx_with(N, 1, M, params, h=0.0, J=1.3)
    s = np.array([[1, 1, 1], [1, -1, 1], [-1, -1, 1], [-1, -1, -1]], dtype=np.int8)
    e = torch.empty(4, dtype=torch.float32, device="cuda")
    c.local_energy(to_words_tensor(pack_np(s)), e)
    np.testing.assert_allclose(e.cpu().numpy(), TFIM(N, 1, 1.3, 0.0).diagonal(s), rtol=0, atol=1e-6)
    # a single chain on the ring, replayed in the oracle
    st = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
    c.init_chains(st, 1)
    s0 = unpack_np(words_from_tensor(st), N)
    bits = torch.zeros((1, 40, 1), dtype=torch.int32, device="cuda")
    c.sweep(st, 40, 0, 2, 0, accept_bits=bits)
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    ref = mh_sweeps(RBM(N, M, params).logpsi, s0, np.arange(1), 2, 40, 0, replay_accepts=acc, tau=1e-4)
    np.testing.assert_array_equal(unpack_np(words_from_tensor(st), N), ref["spins"])
