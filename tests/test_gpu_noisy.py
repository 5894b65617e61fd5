"""Noisy RBM (Sec. 4.1) on the GPU against the oracle (oracle/noisy.py):

* lockstep replay: every decision of the noisy FP32 sampler agrees with the FP64 rule on
  log psi~ = log psi + zeta/2 outside tau of the threshold, and the configurations are
  identical (one and two Philox blocks of the configuration hash);
* the sampled 4 x 4 histogram matches the exact tilted distribution pi~ = pi e^zeta / Z at the
  i.i.d. noise floor, while it is far from the unperturbed pi;
* the exact TV(pi, pi~) obeys the Pinsker bound sigma/2 (Eq. tv_gaussian) at small sigma, and
  the acceptance rate falls as sigma grows large (Fig. 1(c)).
"""
import numpy as np
import pytest

from helpers import nqs, unpack_np, unpack_accept_bits, words_from_tensor
from oracle import exact
from oracle.bounds import tv_distance
from oracle.models import RBM
from oracle.noisy import noisy_logpsi
from oracle.sampler import mh_sweeps
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TAU = 1e-4


def make(Lx, Ly, M, w_sigma, seed, noise, key, h=1.0):
    ctx = nqs().Context("tfim", Lx, Ly, J1=1.0, h=h, model="rbm", n_hidden=M, dtype="f32")
    params = rbm_params(Lx * Ly, M, w_sigma, seed)
    ctx.set_params(torch.from_numpy(params).cuda())
    ctx.set_noise(noise, key)
    return ctx, RBM(Lx * Ly, M, params)


@pytest.mark.parametrize("Lx,Ly,M,noise", [(16, 1, 16, 0.3), (6, 6, 72, 2.0), (150, 1, 40, 0.7)])
def test_noisy_sweep_lockstep_with_oracle(Lx, Ly, M, noise):
    N, C, T, B, key = Lx * Ly, 200, 4, 1, 77
    ctx, model = make(Lx, Ly, M, 0.2, 5, noise, key)
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 9)
    s0 = unpack_np(words_from_tensor(state), N)
    samples = torch.zeros(((T - B) * C, ctx.W), dtype=torch.int32, device="cuda")
    bits = torch.zeros((C, T, ctx.W), dtype=torch.int32, device="cuda")
    ctx.sweep(state, T, B, 31, 0, samples, accept_bits=bits)
    acc = unpack_accept_bits(words_from_tensor(bits), N)
    ref = mh_sweeps(noisy_logpsi(model.logpsi, noise, key), s0, np.arange(C), 31, T, B,
                    replay_accepts=acc, tau=TAU)
    np.testing.assert_array_equal(unpack_np(words_from_tensor(state), N), ref["spins"])
    np.testing.assert_array_equal(unpack_np(words_from_tensor(samples), N), ref["samples"])
    assert ref["near_threshold"] <= max(2, 1e-5 * ref["checked"])


def test_noisy_histogram_matches_the_tilted_distribution_4x4():
    noise, key = 1.0, 123
    ctx, model = make(4, 4, 64, 0.25, 13, noise, key, h=3.04)
    C, T = 32768, 200
    state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
    ctx.init_chains(state, 21)
    ctx.sweep(state, T, T, 22, 0)
    idx = words_from_tensor(state)[:, 0].astype(np.int64)
    hist = np.bincount(idx, minlength=2 ** 16) / idx.size
    pit = exact.exact_pi(noisy_logpsi(model.logpsi, noise, key), 16)
    pi = exact.exact_pi(model.logpsi, 16)
    rng = np.random.default_rng(0)
    floors = [tv_distance(np.bincount(rng.choice(pit.size, C, p=pit), minlength=pit.size) / C, pit)
              for _ in range(8)]
    assert tv_distance(hist, pit) < max(floors) * 1.15, (tv_distance(hist, pit), floors)
    assert tv_distance(hist, pi) > tv_distance(pi, pit) * 0.8 > 3 * max(floors)


def test_exact_bias_and_acceptance_against_sigma_4x4():
    _, model = make(4, 4, 64, 0.25, 13, 0.0, 1, h=3.04)
    pi = exact.exact_pi(model.logpsi, 16)
    for noise in (0.01, 0.03, 0.1):
        pit = exact.exact_pi(noisy_logpsi(model.logpsi, noise, 5), 16)
        assert tv_distance(pi, pit) <= noise / 2 * 1.1, (noise, tv_distance(pi, pit))
    rates = []
    for noise in (0.0, 1.0, 4.0):
        ctx, _ = make(4, 4, 64, 0.25, 13, noise, 5, h=3.04)
        C, T = 4096, 40
        state = torch.zeros((C, 1), dtype=torch.int32, device="cuda")
        ctx.init_chains(state, 3)
        ctx.sweep(state, 10, 10, 4, 0)                       # burn in
        nacc = torch.zeros(C, dtype=torch.int64, device="cuda")
        ctx.sweep(state, T, T, 4, 10, None, None, nacc)
        rates.append(nacc.sum().item() / (C * T * 16))
    assert rates[0] > rates[1] > rates[2], rates


def test_noise_only_on_fp32_rbm_contexts():
    p = nqs()
    c = p.Context("tfim", 4, 4, J1=1.0, h=1.0, model="rbm", n_hidden=16, dtype="f16")
    with pytest.raises(p.NQSError):
        c.set_noise(0.1, 1)
    c.set_noise(0.0, 1)                                         # off is always accepted
