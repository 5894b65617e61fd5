"""Batched uneven instances: one persistent launch over many TFIM problems.

* FP32 batch, replayed in the FP64 oracle in lockstep (bit-exact proposals, decisions
  within tau of the threshold, identical configurations).
* FP32 and FP16 batches against the same chains sampled one context at a time with
  nqs_sweep at 32 lanes per chain: bit-identical states, samples, log psi, accept counts
  and accept bits (the two paths run the same per-chain arithmetic).
* The step graph (sweep -> local energy -> statistics -> O rows) against the
  single-context calls, replayed at two sweep offsets.
* The autotuner leaves the chains untouched and reports what it timed.
"""
import numpy as np
import pytest

from helpers import nqs, unpack_np, unpack_accept_bits, words_from_tensor
from oracle.models import RBM
from oracle.sampler import mh_sweeps
from workloads import rbm_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TAU = 1e-4

# (Lx, Ly, alpha, chains): 1D and 2D, several widths per lane (E = M_pad / 32), ragged chain
# counts, and (FP16) tables too large for shared memory
SHAPES_F32 = [(16, 1, 1, 300), (6, 6, 4, 257), (37, 1, 2, 64), (8, 8, 1, 130)]
SHAPES_F16 = [(36, 1, 1, 300), (6, 6, 4, 257), (10, 10, 4, 200), (16, 16, 4, 40), (14, 14, 2, 77),
              (64, 1, 2, 100)]


def _make(shapes, dtype, seed0=11, h0=0.7):
    p = nqs()
    out = []
    for k, (Lx, Ly, alpha, C) in enumerate(shapes):
        N = Lx * Ly
        M = alpha * N
        ctx = p.Context("tfim", Lx, Ly, J1=1.0, h=h0 + 0.3 * k, model="rbm", n_hidden=M, dtype=dtype)
        params = rbm_params(N, M, 0.25 / np.sqrt(alpha), seed0 + k)
        ctx.set_params(torch.from_numpy(params).cuda())
        state = torch.zeros((C, ctx.W), dtype=torch.int32, device="cuda")
        ctx.init_chains(state, seed0 + 100 + k)
        out.append(dict(ctx=ctx, state=state, seed=seed0 + 200 + k, params=params, N=N, M=M, C=C))
    return out


def _outputs(inst, T, B, eloc=False, O=False):
    c, C = inst["ctx"], inst["C"]
    K = T - B
    d = dict(samples=torch.zeros((K * C, c.W), dtype=torch.int32, device="cuda"),
             logpsi=torch.zeros(K * C, dtype=torch.float32, device="cuda"),
             n_accepted=torch.zeros(C, dtype=torch.int64, device="cuda"),
             accept_bits=torch.zeros((C, T, c.W), dtype=torch.int32, device="cuda"))
    if eloc:
        d["eloc"] = torch.zeros(K * C, dtype=torch.float32, device="cuda")
        d["stats"] = torch.zeros(5, dtype=torch.float64, device="cuda")
    if O:
        d["O"] = torch.zeros((C, c.P), dtype=torch.float32, device="cuda")
    return d


def test_fp32_batch_lockstep_with_oracle():
    T, B = 4, 1
    insts = _make(SHAPES_F32, "f32")
    s0 = [unpack_np(words_from_tensor(i["state"]), i["N"]) for i in insts]
    outs = [_outputs(i, T, B) for i in insts]
    b = nqs().Batch([dict(ctx=i["ctx"], state=i["state"], seed=i["seed"], **o) for i, o in zip(insts, outs)],
                    T, B, warps_per_cta=8)
    b.sweep(3)
    torch.cuda.synchronize()
    for i, o, s in zip(insts, outs, s0):
        N, M, C = i["N"], i["M"], i["C"]
        acc = unpack_accept_bits(words_from_tensor(o["accept_bits"]), N)
        ref = mh_sweeps(RBM(N, M, i["params"]).logpsi, s, np.arange(C), i["seed"], T, B, sweep_offset=3,
                        replay_accepts=acc, tau=TAU)
        np.testing.assert_array_equal(unpack_np(words_from_tensor(i["state"]), N), ref["spins"])
        np.testing.assert_array_equal(unpack_np(words_from_tensor(o["samples"]), N), ref["samples"])
        np.testing.assert_array_equal(o["n_accepted"].cpu().numpy(), acc.sum(axis=(1, 2)))
        np.testing.assert_allclose(o["logpsi"].cpu().numpy(), ref["logpsi"], rtol=1e-5, atol=1e-5)
        assert ref["near_threshold"] <= max(2, 1e-5 * ref["checked"])


@pytest.mark.parametrize("dtype,shapes,warps", [("f32", SHAPES_F32, 4), ("f16", SHAPES_F16, 12),
                                                ("f16", SHAPES_F16, 0)])
def test_batch_equals_single_context_sweeps(dtype, shapes, warps):
    T, B = 5, 2
    insts = _make(shapes, dtype)
    for i in insts:   # the batch runs 32 lanes per chain; pin the single-context FP32 path to it
        i["ctx"].set_option(nqs().OPT_CHAINS_PER_WARP, 1)
    twins = [i["state"].clone() for i in insts]
    outs = [_outputs(i, T, B) for i in insts]
    b = nqs().Batch([dict(ctx=i["ctx"], state=i["state"], seed=i["seed"], **o) for i, o in zip(insts, outs)],
                    T, B, warps_per_cta=warps)
    for i, tw in zip(insts, twins):   # the autotuner (warps = 0) must leave the chains untouched
        assert torch.equal(i["state"], tw)
    b.sweep(7)
    for i, o, tw in zip(insts, outs, twins):
        r = _outputs(i, T, B)
        i["ctx"].sweep(tw, T, B, i["seed"], 7, r["samples"], r["logpsi"], r["n_accepted"],
                       accept_bits=r["accept_bits"])
        torch.cuda.synchronize()
        assert torch.equal(i["state"], tw)
        for key in ("samples", "logpsi", "n_accepted", "accept_bits"):
            assert torch.equal(o[key], r[key]), key
    info = b.info()
    assert info["n_work_items"] >= len(insts)
    if warps == 0:
        assert info["tuned"] and (info["variant"], info["warps_per_cta"]) in [(v, w) for v, w, _ in info["tuned"]]
    if dtype == "f16":
        assert 0 < info["n_staged"] < len(insts)    # the 16 x 16, alpha = 4 table goes through L2


def test_batch_step_graph_matches_single_context_calls():
    T, B = 4, 1
    insts = _make(SHAPES_F16[:4], "f16", seed0=41)
    twins = [i["state"].clone() for i in insts]
    outs = [_outputs(i, T, B, eloc=True, O=True) for i in insts]
    b = nqs().Batch([dict(ctx=i["ctx"], state=i["state"], seed=i["seed"], **o) for i, o in zip(insts, outs)],
                    T, B, warps_per_cta=8)
    for offset in (0, T):                       # replay of the captured graph at a new offset
        b.step(offset)
        for i, o, tw in zip(insts, outs, twins):
            c, C = i["ctx"], i["C"]
            r = _outputs(i, T, B, eloc=True, O=True)
            c.sweep(tw, T, B, i["seed"], offset, r["samples"], r["logpsi"], r["n_accepted"],
                    accept_bits=r["accept_bits"])
            c.local_energy(r["samples"], r["eloc"])
            c.stats(r["eloc"], C, r["stats"], r["n_accepted"], T * i["N"])
            c.logpsi_grad(r["samples"][(T - B - 1) * C:], r["O"])
            torch.cuda.synchronize()
            assert torch.equal(i["state"], tw)
            for key in ("samples", "logpsi", "n_accepted", "eloc", "stats", "O"):
                assert torch.equal(o[key], r[key]), (offset, key)


def test_batch_rejects_mixed_dtypes_and_dense_contexts():
    p = nqs()
    a = _make([(16, 1, 1, 40)], "f32")[0]
    b = _make([(16, 1, 1, 40)], "f16")[0]
    with pytest.raises(p.NQSError):
        p.Batch([dict(ctx=a["ctx"], state=a["state"], seed=1), dict(ctx=b["ctx"], state=b["state"], seed=2)], 2, 0, 8)
    d = p.Context("heisenberg", 4, 4, J1=1.0, model="dense", widths=(32, 32), dtype="bf16")
    d.set_params(torch.zeros(d.P, dtype=torch.float64, device="cuda"))
    st = torch.zeros((8, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(p.NQSError):
        p.Batch([dict(ctx=d, state=st, seed=1)], 2, 0, 8)
