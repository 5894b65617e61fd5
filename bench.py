#!/usr/bin/env python
"""Benchmark of the NQS VMC hot path on one B300 (or N, one process per GPU).

Workload: 2D transverse-field Ising model on a 10 x 10 periodic lattice, h = 3.04,
RBM with alpha = 4 (400 hidden units), weights ~ N(0, 0.05^2); 16384 chains x 500
single-spin-flip sweeps (50 burn-in), i.e. 8.19e8 Metropolis-Hastings proposals and
7.37e6 kept samples per GPU.  One step = the whole hot path on that batch:
parameter downcast, chain initialisation, the sweeps, local energies of every kept
sample, FP64 statistics, the force over every kept sample, and the O_k rows of the
last sweep's samples.  Synthetic, seeded data; no datasets or trained weights.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

import workloads

METRIC = "MH proposals/sec and local-energy samples/sec on 1 B300, mixed vs FP32 at stated bias"
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch of the sweep kernel
# (16384 chains x 500 sweeps of this workload), per sampling copy, for the kernel as built;
# a copy without an entry reports None.
SWEEP_TRAFFIC_BYTES = {"f16": 77.5e6}   # 2.38 MB read + 75.11 MB written
# Warp instructions per proposal of the sweep kernel by pipe, from the ncu capture summarised in
# profiles/rbm_sweep_pipe_mix.md (10-sweep launch of 4144 chains on this workload, kernel as profiled).
SWEEP_PIPE_MIX = {
    "f32": {"total": 90.2, "fma": 32.2, "fma_fp16": 1.3, "alu": 25.3, "lsu": 9.4, "cbu": 2.9, "xu": 2.7, "adu": 2.1},
    "f16": {"total": 132.6, "fma": 57.0, "fma_fp16": 27.2, "alu": 31.3, "lsu": 13.6, "cbu": 5.8, "xu": 3.4, "adu": 3.4},
    "bf16": {"total": 142.8, "fma": 38.0, "fma_fp16": 8.1, "alu": 59.9, "lsu": 14.7, "cbu": 5.8, "xu": 3.4, "adu": 2.9},
}
WL = workloads.TFIM_2D_10x10


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def measure_alu_peaks(nqs, torch, dev, target_ms=25.0):
    """Issue rates of the instructions the RBM kernels use (nqs_probe_alu), in T lane-ops/s:
    every SM full (4 CTAs x 512 threads), 8 independent chains per thread, best of three
    launches of about target_ms each, timed with CUDA events on the launching stream.  The
    SM clock is sampled while they run."""
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = n_sm * 4, 512
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    with ClockSampler(dev.index) as clk:
        for kind in nqs.PROBE_KINDS:
            def run(iters):
                ev0.record()
                nqs.probe_alu(kind, blocks, threads, iters, sink)
                ev1.record()
                torch.cuda.synchronize()
                return ev0.elapsed_time(ev1)
            run(64)
            iters = max(64, int(2048 * target_ms / max(run(2048), 1e-3)))
            best = min(run(iters) for _ in range(3))
            ops = blocks * threads * iters * 8 * nqs.PROBE_OPS[kind]
            out[kind] = ops / (best / 1e3) / 1e12
    out["unit"] = "T lane-ops/s (FP32 / F16 / BF16 element operations, or MUFU results)"
    out["clocks"] = clk.summary()
    return out


def enumerate_bias_4x4(nqs, torch, dev, dtype):
    """The workload's 4 x 4 case (alpha = 4, the same weight distribution) by full enumeration:
    delta(x) = 2 (log psi_copy(x) - log psi_FP32(x)) over all 2^16 configurations through
    nqs_logpsi of the 16-bit and FP32 contexts, its standard deviation (Sec. 4.2, Fig. 2), the
    exact TV(pi, pi~) and KL, and min(Pinsker, Thm 3) from the single-flip increments of delta."""
    lat = WL.extra["small_case"]
    N, M = lat.n_sites, 4 * lat.n_sites
    params = torch.from_numpy(workloads.rbm_params(N, M, WL.weight_sigma, WL.seed)).to(dev)
    x = np.arange(2 ** N, dtype=np.int64)
    cfg = torch.from_numpy(x.astype(np.int32)).view(-1, 1).to(dev)
    lps = {}
    for d in (dtype, "f32"):
        ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=WL.ham.J1, h=WL.ham.h, model="rbm", n_hidden=M, dtype=d)
        ctx.set_params(params)
        out = torch.empty(x.size, dtype=torch.float32, device=dev)
        ctx.logpsi(cfg, out)
        lps[d] = out.double().cpu().numpy()
    delta = 2.0 * (lps[dtype] - lps["f32"])
    logp = 2.0 * lps["f32"]
    pi = np.exp(logp - logp.max())
    pi /= pi.sum()
    pt = pi * np.exp(delta - delta.max())
    pt /= pt.sum()
    eps = np.concatenate([delta[x ^ (1 << i)] - delta for i in range(N)])
    s = float(eps.std() / math.sqrt(2.0))
    return {"sigma_delta": float(delta.std()), "tv_exact": float(0.5 * np.abs(pi - pt).sum()),
            "kl_exact": float(np.sum(pi * np.log(pi / pt))),
            "tv_bound": min(s / 2, thm3_bound(float(eps.mean()), s)),
            "note": "16-bit copy against the FP32 copy, all 65536 configurations, log psi from scratch"}


def thm3_bound(mu, sigma):
    """Theorem 3 (Eq. avg_bound) at r = 0 for log-density increments eps ~ N(mu, 2 sigma^2)."""
    if sigma <= 0:
        return 1.0 - math.exp(-abs(mu))
    return 1.0 - 0.5 * math.exp(sigma ** 2) * (math.exp(-mu) * math.erfc(sigma - mu / (2 * sigma))
                                               + math.exp(mu) * math.erfc(sigma + mu / (2 * sigma)))


class Step:
    """Buffers and one VMC step of the workload for one sampling dtype."""

    def __init__(self, nqs, torch, dev, dtype, C, T, B, params_h, dist=None):
        ham, lat = WL.ham, WL.ham.lattice
        self.dist = dist
        self.torch, self.dev, self.dtype = torch, dev, dtype
        self.N, self.M, self.C, self.T, self.B = lat.n_sites, WL.n_hidden, C, T, B
        self.S = (T - B) * C
        self.ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=ham.J1, h=ham.h, model="rbm", n_hidden=self.M, dtype=dtype)
        P = self.ctx.P
        self.params_h = params_h
        self.params = params_h.to(dev)
        self.state = torch.zeros((C, self.ctx.W), dtype=torch.int32, device=dev)
        self.samples = torch.zeros((self.S, self.ctx.W), dtype=torch.int32, device=dev)
        self.nacc = torch.zeros(C, dtype=torch.int64, device=dev)
        self.eloc = torch.zeros(self.S, dtype=torch.float32, device=dev)
        self.stats = torch.zeros(5, dtype=torch.float64, device=dev)
        self.moments = torch.zeros(8, dtype=torch.float64, device=dev)
        self.force = torch.zeros(P, dtype=torch.float64, device=dev)
        self.O = torch.zeros((C, P), dtype=torch.float32, device=dev)
        self.ws = torch.zeros(self.ctx.logpsi_grad_workspace(self.S), dtype=torch.uint8, device=dev)
        self.out_h = torch.zeros(5 + P, dtype=torch.float64).pin_memory()
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        # set_params (prepare, colsum, bounds; a 16-bit copy adds the FP32 copy's prepare and colsum),
        # init, sweep, local energy, stats (2; 3 with the multi-rank finalize), force (tensor-core
        # kernel + reduction), O rows
        self.launches = (3 if dtype == "f32" else 5) + 1 + 1 + 1 + (3 if dist else 2) + 2 + 1

    def run(self, seed, host_io=False):
        c, ev = self.ctx, self.ev
        if host_io:
            self.params.copy_(self.params_h, non_blocking=True)
        ev[0].record()
        c.set_params(self.params)
        c.init_chains(self.state, seed)
        ev[1].record()
        c.sweep(self.state, self.T, self.B, seed + 1, 0, self.samples, None, self.nacc)
        ev[2].record()
        c.local_energy_chains(self.samples, self.C, self.eloc)
        ev[3].record()
        if self.dist:   # the one exchange of the step: pooled statistics (global E) first, then the force
            from paper_2601_20782_b300.distributed import exchange_stats, exchange_force
            c.stats_moments(self.eloc, self.C, self.moments, self.nacc, self.T * self.N)
            exchange_stats(c, self.moments, self.stats)
            c.force_share(self.samples, self.eloc, self.stats, self.force, self.ws)
            exchange_force(self.force)
        else:
            c.stats(self.eloc, self.C, self.stats, self.nacc, self.T * self.N)
            c.logpsi_grad(self.samples, None, self.eloc, self.stats, self.force, self.ws)
        ev[4].record()
        c.logpsi_grad(self.samples[self.S - self.C:], self.O)
        ev[5].record()
        if host_io:
            self.out_h[:5].copy_(self.stats, non_blocking=True)
            self.out_h[5:].copy_(self.force, non_blocking=True)

    def phases(self):
        return [self.ev[i].elapsed_time(self.ev[i + 1]) for i in range(5)]


def run_ours(args, rank, world, dist):
    import torch
    import paper_2601_20782_b300 as nqs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lat = WL.ham.lattice
    N, M, C, T, B = lat.n_sites, WL.n_hidden, WL.n_chains, WL.n_sweeps, WL.burn_in
    if args.chains or args.sweeps:   # smaller case of the same kernels, for profiler captures only
        C, T, B = args.chains or C, args.sweeps or T, args.burn_in if args.burn_in is not None else B
    params_h = torch.from_numpy(workloads.rbm_params(N, M, WL.weight_sigma, WL.seed)).pin_memory()
    dtypes = [args.dtype] + ([d for d in ("f32", "bf16", "f16") if d != args.dtype] if args.compare else [])
    steps = {d: Step(nqs, torch, dev, d, C, T, B, params_h, dist) for d in dtypes}
    if args.chains_per_warp and "f32" in steps:
        steps["f32"].ctx.set_option(nqs.OPT_CHAINS_PER_WARP, args.chains_per_warp)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    base_seed = WL.seed * 1000 + rank * 7919
    proposals_step = C * T * N
    results = {}

    for d in dtypes:
        st = steps[d]
        for w in range(args.warmup):
            st.run(base_seed + w)
        torch.cuda.synchronize()
        phase = np.zeros(5)
        step_ms, acc_total, energies = [], 0, []
        with ClockSampler(dev.index) as clk:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()                       # L2 flush between timed steps (not timed)
                st.run(base_seed + 100 + k)
                torch.cuda.synchronize()
                acc_total += int(st.nacc.sum().item())
                energies.append(st.stats[:3].cpu().numpy().copy())
                ph = st.phases()
                phase += ph
                step_ms.append(sum(ph))
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
        t_dev = sum(step_ms) / 1e3
        if dist:
            tt = torch.tensor([t_dev], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_dev = tt.item()
        en = np.array(energies)
        results[d] = {"t_dev": t_dev, "phase": phase / args.steps, "accepts": acc_total / args.steps,
                      "clocks": clk.summary(), "E": float(en[:, 0].mean()),
                      "E_err": float(np.sqrt((en[:, 2] ** 2).sum()) / len(en))}

    # end to end through the public API with host buffers (primary dtype): pinned FP64
    # parameters in, statistics and force out
    st = steps[args.dtype]
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.run(base_seed + 200 + k, host_io=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    t_e2e = sum(e2e_ms) / 1e3
    if dist:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = tt.item()

    # stated bias of each 16-bit copy: increment errors against the FP32 copy at that copy's
    # own sampled states x, y a uniform single flip (the setting of Theorem 3)
    bias = {}
    if "f32" in steps:
        ref = steps["f32"]
        for d in dtypes:
            if d == "f32":
                continue
            S = steps[d].samples[steps[d].S - C:]
            g = torch.Generator(device=dev).manual_seed(WL.seed)
            sites = torch.randint(0, N, (S.shape[0],), generator=g, dtype=torch.int32, device=dev)
            d_lp = torch.empty(S.shape[0], dtype=torch.float32, device=dev)
            d_32 = torch.empty(S.shape[0], dtype=torch.float32, device=dev)
            steps[d].ctx.flip_delta(S, sites, d_lp)
            ref.ctx.flip_delta(S, sites, d_32)
            eps = (2.0 * (d_lp.double() - d_32.double())).cpu().numpy()
            mu, sig = float(eps.mean()), float(eps.std() / math.sqrt(2.0))
            dE = results[d]["E"] - results["f32"]["E"]
            bias[d] = {"eps_mean": mu, "eps_std": float(eps.std()), "sigma_delta": sig,
                       "pinsker_tv_bound": sig / 2, "thm3_tv_bound_r0": thm3_bound(mu, sig),
                       "tv_bound": min(sig / 2, thm3_bound(mu, sig)),
                       # Theorem 2 on the same proposals (x from the copy's own chains, y a flip)
                       "thm2_one_step_bound": float(1.0 - np.mean(np.exp(-np.abs(eps)))),
                       "enumeration_4x4": enumerate_bias_4x4(nqs, torch, dev, d),
                       "energy_vs_f32": dE, "energy_err": math.hypot(results[d]["E_err"], results["f32"]["E_err"]),
                       "sweep_speed_vs_f32": (results["f32"]["phase"][1] / results[d]["phase"][1])}

    r = results[args.dtype]
    ph = r["phase"]   # ms per phase: prep+init, sweep, eloc, stats+force, O rows
    value = world * proposals_step * args.steps / r["t_dev"]
    alu = measure_alu_peaks(nqs, torch, dev)
    # Sweep roofline (arithmetic of the method per proposal): one FMA (factor) and one multiply
    # (product) per hidden unit, three multiplies per hidden unit per accepted flip, counted as
    # FP32 lane operations; peak = the measured issue rate of the paired FP32 FMA (fma.rn.f32x2)
    # in the same units, the instruction those operations are issued as.
    alg_ops = 2.0 * M * proposals_step + 3.0 * M * r["accepts"]
    achieved = alg_ops / (ph[1] / 1e3) / 1e12
    peak = alu["ffma2"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "proposals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["t_dev"] / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16 sampling (f32 caches, accept, statistics)",
                  "f16": "f16 sampling (f32 caches, accept, statistics)"}[args.dtype],
        "data": "synthetic (seeded random-init RBM, random initial spins)",
        "config": {"workload": WL.name if (C, T) == (WL.n_chains, WL.n_sweeps) else f"{WL.name} (reduced: profiling)",
                   "lattice": "10x10 periodic", "h": WL.ham.h, "n_hidden": M, "chains": C, "sweeps": T,
                   "burn_in": B, "samples": (T - B) * C, "params": steps[args.dtype].ctx.P,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"dp{world} (chains)"},
        "local_energy": {"value": world * (T - B) * C / (ph[2] / 1e3), "unit": "samples/s", "kernel_ms": ph[2]},
        "sweep": {"value": world * proposals_step / (ph[1] / 1e3), "unit": "proposals/s", "kernel_ms": ph[1],
                  "acceptance": r["accepts"] / proposals_step},
        "phases_ms": {"set_params+init": ph[0], "sweep": ph[1], "local_energy": ph[2],
                      "stats+force": ph[3], "O_rows": ph[4]},
        "energy": {"E": r["E"], "err": r["E_err"]},
        "compare": {d: {"value": world * proposals_step * args.steps / results[d]["t_dev"],
                        "sweep_proposals_per_s": world * proposals_step / (results[d]["phase"][1] / 1e3),
                        "local_energy_samples_per_s": world * (T - B) * C / (results[d]["phase"][2] / 1e3),
                        "E": results[d]["E"], "E_err": results[d]["E_err"]}
                    for d in dtypes if d != args.dtype},
        "bias": bias,
        "roofline": {"bound": "alu", "kernel": "rbm_sweep_kernel", "achieved": achieved, "peak": peak,
                     "unit": "T lane-ops/s", "frac": achieved / peak,
                     "peak_source": "measured in this run: fma.rn.f32x2 issue rate (nqs_probe_alu), FP32 ops",
                     "traffic": SWEEP_TRAFFIC_BYTES.get(args.dtype) if (C, T) == (WL.n_chains, WL.n_sweeps) else None,
                     "traffic_source": "from profile (ncu dram bytes of this kernel at this size; null when the "
                                       "kernel changed since the capture)",
                     "note": "method arithmetic per proposal (2M + 3M per accept) vs the measured paired-FP32 "
                             "issue rate"},
        "alu_peaks": alu,
        "sweep_instructions_per_proposal": {"source": "from profile (ncu per-pipe counts, profiles/rbm_sweep_pipe_mix.md)",
                                            "method_arithmetic": 12.5, **{d: SWEEP_PIPE_MIX[d] for d in dtypes
                                                                        if d in SWEEP_PIPE_MIX}},
        "e2e": {"value": world * proposals_step * args.steps / t_e2e, "unit": "proposals/s",
                "h2d_bytes_per_step": steps[args.dtype].ctx.P * 8, "d2h_bytes_per_step": (5 + steps[args.dtype].ctx.P) * 8},
        "gpu_launches": steps[args.dtype].launches * args.steps,
        "clocks": r["clocks"],
    }
    return line


# ------------------------------------------------------------------------------------------
# The other workloads (--workload): the 1D N = 16 RBM, the dense 10 x 10 Heisenberg, the 48
# batched TFIM instances, the dense 16 x 16 J1-J2 ansatz and the 10 x 10 complex-parameter RBM.
# Each step is the whole hot path
# of that workload; the line has the same keys as the default workload's.

class _Phased:
    """CUDA events around the phases of one step, on the current stream."""

    def __init__(self, torch, names):
        self.names = names
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]

    def mark(self, k):
        self.ev[k].record()

    def ms(self):
        return {n: self.ev[k].elapsed_time(self.ev[k + 1]) for k, n in enumerate(self.names)}


class RbmStep:
    """Downcast, init, sweeps, local energies, statistics, force and last-sweep O rows of one
    RBM workload (the default workload's step for another lattice / dtype)."""

    def __init__(self, nqs, torch, dev, wl, dtype, C=None, T=None, B=None):
        lat = wl.ham.lattice
        self.wl, self.torch = wl, torch
        self.N, self.M = lat.n_sites, wl.n_hidden
        self.C, self.T, self.B = C or wl.n_chains, T or wl.n_sweeps, wl.burn_in if B is None else B
        self.S = (self.T - self.B) * self.C
        self.ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=wl.ham.J1, h=wl.ham.h, model="rbm", n_hidden=self.M,
                               dtype=dtype)
        P = self.ctx.P
        self.params_h = torch.from_numpy(workloads.rbm_params(self.N, self.M, wl.weight_sigma, wl.seed)).pin_memory()
        self.params = self.params_h.to(dev)
        z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device=dev)
        self.state, self.samples = z(self.C, self.ctx.W), z(self.S, self.ctx.W)
        self.nacc, self.eloc = z(self.C, dt=torch.int64), z(self.S, dt=torch.float32)
        self.stats, self.force = z(5, dt=torch.float64), z(P, dt=torch.float64)
        self.O = z(self.C, P, dt=torch.float32)
        self.ws = z(self.ctx.logpsi_grad_workspace(self.S), dt=torch.uint8)
        self.out_h = torch.zeros(5 + P, dtype=torch.float64).pin_memory()
        self.ph = _Phased(torch, ["set_params+init", "sweep", "local_energy", "stats+force", "O_rows"])
        self.launches = (3 if dtype == "f32" else 5) + 1 + 1 + 1 + 2 + 2 + 1   # as Step
        self.h2d, self.d2h = P * 8, (5 + P) * 8

    def run(self, seed, host_io=False):
        c, ph = self.ctx, self.ph
        if host_io:
            self.params.copy_(self.params_h, non_blocking=True)
        ph.mark(0)
        c.set_params(self.params)
        c.init_chains(self.state, seed)
        ph.mark(1)
        c.sweep(self.state, self.T, self.B, seed + 1, 0, self.samples, None, self.nacc)
        ph.mark(2)
        c.local_energy_chains(self.samples, self.C, self.eloc)
        ph.mark(3)
        c.stats(self.eloc, self.C, self.stats, self.nacc, self.T * self.N)
        c.logpsi_grad(self.samples, None, self.eloc, self.stats, self.force, self.ws)
        ph.mark(4)
        c.logpsi_grad(self.samples[self.S - self.C:], self.O)
        ph.mark(5)
        if host_io:
            self.out_h[:5].copy_(self.stats, non_blocking=True)
            self.out_h[5:].copy_(self.force, non_blocking=True)

    def units(self):
        return self.C * self.T * self.N

    def describe(self, ms, accepts, peaks_, n_sm):
        alg = 2.0 * self.M * self.units() + 3.0 * self.M * accepts
        ach = alg / (ms["sweep"] / 1e3) / 1e12
        peak = peaks_["alu"]["ffma2"]
        lat = self.wl.ham.lattice
        return {
            "alu_peaks": peaks_["alu"],
            "config": {"workload": self.wl.name, "lattice": f"{lat.Lx}x{lat.Ly} periodic", "h": self.wl.ham.h,
                       "n_hidden": self.M, "chains": self.C, "sweeps": self.T, "burn_in": self.B,
                       "samples": self.S, "params": self.ctx.P},
            "local_energy": {"value": self.S / (ms["local_energy"] / 1e3), "unit": "samples/s"},
            "sweep": {"value": self.units() / (ms["sweep"] / 1e3), "unit": "proposals/s",
                      "acceptance": accepts / self.units()},
            "roofline": {"bound": "alu", "kernel": "rbm_sweep_kernel", "achieved": ach, "peak": peak,
                         "unit": "T lane-ops/s", "frac": ach / peak, "traffic": None,
                         "note": "method arithmetic per proposal (2M + 3M per accept) vs the measured "
                                 "fma.rn.f32x2 issue rate (FP32 ops)"},
        }


class ComplexRbmStep:
    """The default workload's lattice, width and sizes with complex a, b, W (App. G): set_params,
    init, sweeps on 2 Re delta, complex local energies, statistics, conjugate force and the
    last sweep's O rows."""

    def __init__(self, nqs, torch, dev, wl, C=None, T=None, B=None):
        lat = wl.ham.lattice
        self.wl, self.torch = wl, torch
        self.N, self.M = lat.n_sites, wl.n_hidden
        self.C, self.T, self.B = C or wl.n_chains, T or wl.n_sweeps, wl.burn_in if B is None else B
        self.S = (self.T - self.B) * self.C
        self.ctx = nqs.ComplexContext(lat.Lx, lat.Ly, J1=wl.ham.J1, h=wl.ham.h, n_hidden=self.M)
        P = self.ctx.P
        self.params_h = torch.from_numpy(
            workloads.complex_rbm_params(self.N, self.M, wl.weight_sigma, wl.seed)).pin_memory()
        self.params = self.params_h.to(dev)
        z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device=dev)
        self.state, self.samples = z(self.C, self.ctx.W), z(self.S, self.ctx.W)
        self.nacc = z(self.C, dt=torch.int64)
        self.eloc_re, self.eloc_im = z(self.S, dt=torch.float32), z(self.S, dt=torch.float32)
        self.stats, self.force = z(6, dt=torch.float64), z(P, dt=torch.complex128)
        self.O = z(self.C, P, dt=torch.complex64)
        self.out_h = torch.zeros(6 + 2 * P, dtype=torch.float64).pin_memory()
        self.ph = _Phased(torch, ["set_params+init", "sweep", "local_energy", "stats+force", "O_rows"])
        # prepare, init, sweep, local energy, 2 x (stats partial + final), force + scale, O rows
        self.launches = 1 + 1 + 1 + 1 + 4 + 2 + 1
        self.h2d, self.d2h = P * 16, (6 + 2 * P) * 8

    def run(self, seed, host_io=False):
        c, ph = self.ctx, self.ph
        if host_io:
            self.params.copy_(self.params_h, non_blocking=True)
        ph.mark(0)
        c.set_params(self.params)
        c.init_chains(self.state, seed)
        ph.mark(1)
        c.sweep(self.state, self.T, self.B, seed + 1, 0, self.samples, self.nacc)
        ph.mark(2)
        c.local_energy_chains(self.samples, self.C, self.eloc_re, self.eloc_im)
        ph.mark(3)
        c.stats(self.eloc_re, self.eloc_im, self.C, self.stats, self.nacc, self.T * self.N)
        c.logpsi_grad(self.samples, None, self.eloc_re, self.eloc_im, self.stats, self.force)
        ph.mark(4)
        c.logpsi_grad(self.samples[self.S - self.C:], self.O)
        ph.mark(5)
        if host_io:
            self.out_h[:6].copy_(self.stats, non_blocking=True)
            self.out_h[6:].copy_(self.torch.view_as_real(self.force).reshape(-1), non_blocking=True)

    def units(self):
        return self.C * self.T * self.N

    def describe(self, ms, accepts, peaks_, n_sm):
        # per proposal and unit: two spin-signed table factors, two FMAs for sinh x' and cos y',
        # the square sum and the running product (6); an accepted flip rewrites four values (8)
        alg = 6.0 * self.M * self.units() + 8.0 * self.M * accepts
        ach = alg / (ms["sweep"] / 1e3) / 1e12
        peak = peaks_["alu"]["ffma"]
        lat = self.wl.ham.lattice
        return {
            "alu_peaks": peaks_["alu"],
            "config": {"workload": self.wl.name + "_complex", "lattice": f"{lat.Lx}x{lat.Ly} periodic",
                       "h": self.wl.ham.h, "n_hidden": self.M, "chains": self.C, "sweeps": self.T,
                       "burn_in": self.B, "samples": self.S, "params": self.ctx.P,
                       "weights": f"complex, re and im N(0, {self.wl.weight_sigma}^2)"},
            "local_energy": {"value": self.S / (ms["local_energy"] / 1e3), "unit": "samples/s"},
            "sweep": {"value": self.units() / (ms["sweep"] / 1e3), "unit": "proposals/s",
                      "acceptance": accepts / self.units()},
            "energy": float(self.stats[0].item()),
            "roofline": {"bound": "alu", "kernel": "crbm_sweep_kernel", "achieved": ach, "peak": peak,
                         "unit": "T lane-ops/s", "frac": ach / peak, "traffic": None,
                         "note": "method arithmetic per proposal (6M + 8M per accept) vs the measured scalar "
                                 "fma.rn.f32 issue rate (the complex sweep issues scalar FP32 operations)"},
        }


class RescnnStep:
    """Downcast, init, sweeps, local energies of every kept sample and statistics of the ResCNN
    workload (App. H: 4 residual blocks x 16 filters, 3 x 3 kernels; 10 x 10 TFIM at h = 3.04)."""

    def __init__(self, nqs, torch, dev, wl, dtype, C=None, T=None, B=None):
        lat = wl.ham.lattice
        self.wl, self.torch, self.dtype = wl, torch, dtype
        self.N, self.F, self.nb = lat.n_sites, wl.extra["filters"], wl.extra["blocks"]
        self.C, self.T, self.B = C or wl.n_chains, T or wl.n_sweeps, wl.burn_in if B is None else B
        self.S = (self.T - self.B) * self.C
        self.ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=wl.ham.J1, h=wl.ham.h, model="rescnn", n_hidden=self.F,
                               n_blocks=self.nb, dtype=dtype)
        self.params_h = torch.from_numpy(workloads.rescnn_params(self.F, self.nb, wl.seed)).pin_memory()
        self.params = self.params_h.to(dev)
        z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device=dev)
        self.state, self.samples = z(self.C, self.ctx.W), z(self.S, self.ctx.W)
        self.nacc, self.eloc = z(self.C, dt=torch.int64), z(self.S, dt=torch.float32)
        self.stats = z(5, dt=torch.float64)
        self.out_h = torch.zeros(5, dtype=torch.float64).pin_memory()
        self.force = z(self.ctx.P, dt=torch.float64)
        self.n_force = self.C          # the force over the last sweep's samples (one per chain)
        self.ph = _Phased(torch, ["set_params+init", "sweep", "local_energy", "stats", "force"])
        chunks = -(-self.S * (self.N + 1) // (1 << 20))      # local-energy chunks of 2^20 configurations
        # rows of O the library evaluates per launch when the caller gives none (its scratch)
        fchunks = -(-self.n_force // max(1, min(4096, (256 << 20) // (self.ctx.P * 4))))
        # prepare (+ the 16-bit copy's prepare), init, sweep, per chunk evaluation + combine, stats (2),
        # per force chunk the O rows and the two force kernels
        self.launches = (1 if dtype == "f32" else 2) + 1 + 1 + 2 * chunks + 2 + 3 * fchunks
        self.h2d, self.d2h = self.ctx.P * 8, 5 * 8

    def run(self, seed, host_io=False):
        c, ph = self.ctx, self.ph
        if host_io:
            self.params.copy_(self.params_h, non_blocking=True)
        ph.mark(0)
        c.set_params(self.params)
        c.init_chains(self.state, seed)
        ph.mark(1)
        c.sweep(self.state, self.T, self.B, seed + 1, 0, self.samples, None, self.nacc)
        ph.mark(2)
        c.local_energy(self.samples, self.eloc)
        ph.mark(3)
        c.stats(self.eloc, self.C, self.stats, self.nacc, self.T * self.N)
        ph.mark(4)
        last = (self.T - self.B - 1) * self.C   # the last sweep's samples and their local energies
        c.logpsi_grad(self.samples[last:], None, self.eloc[last:], self.stats, self.force)
        ph.mark(5)
        if host_io:
            self.out_h.copy_(self.stats, non_blocking=True)

    def units(self):
        return self.C * self.T * self.N

    def flops_per_eval(self):
        # algorithmic FLOPs of one forward pass: 2 x 9 x 16 x 16 per site and block convolution,
        # 2 x 9 x 16 per site for the embedding
        return 2.0 * self.N * (2 * self.nb * 9 * self.F * self.F + 9 * self.F)

    def describe(self, ms, accepts, peaks_, n_sm):
        lat = self.wl.ham.lattice
        fl = self.flops_per_eval() * self.units()
        ach = fl / (ms["sweep"] / 1e3) / 1e12
        tc = self.dtype != "f32"
        peak = float(peaks_.get("bf16_tflops", 1764.5)) if tc else 2.0 * peaks_["alu"]["ffma"]
        return {
            "config": {"workload": self.wl.name, "lattice": f"{lat.Lx}x{lat.Ly} periodic", "h": self.wl.ham.h,
                       "filters": self.F, "blocks": self.nb, "chains": self.C, "sweeps": self.T, "burn_in": self.B,
                       "samples": self.S, "params": self.ctx.P},
            "local_energy": {"value": self.S / (ms["local_energy"] / 1e3), "unit": "samples/s"},
            "sweep": {"value": self.units() / (ms["sweep"] / 1e3), "unit": "proposals/s",
                      "acceptance": accepts / self.units()},
            "force": {"rows": self.n_force, "rows_per_s": self.n_force / (ms["force"] / 1e3),
                      "note": "O rows (FP32 reverse pass) and the force of the last sweep's samples; the "
                              "statistics' E is that of all samples"},
            "energy": float(self.stats[0].item()),
            "roofline": {"bound": "tensor" if tc else "alu",
                         "kernel": "rescnn_tc_sweep_kernel" if tc else "rescnn_sweep_f32_kernel",
                         "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "peak_source": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json); F16 has the same "
                                        "nominal rate" if tc else "measured fma.rn.f32 issue rate x 2 FLOP",
                         "note": "algorithmic convolution FLOPs of one forward pass per proposal "
                                 "(2 x 9 x 16 x 16 per site and block convolution)"},
        }


class DenseStep:
    """Downcast, init, sweeps (burn-in + kept), local energies of the kept samples, statistics,
    O rows and force of a dense-ansatz workload.  `T` overrides the sweep count (the 16 x 16
    workload times a bounded number of its sweeps)."""

    def __init__(self, nqs, torch, dev, wl, C=None, T=None, B=None, n_grad=None, minsr_lambda=None, dtype="bf16"):
        lat = wl.ham.lattice
        self.wl, self.torch, self.dtype = wl, torch, dtype
        self.N = lat.n_sites
        self.C, self.T = C or wl.n_chains, T or wl.n_sweeps
        self.B = min(wl.burn_in, self.T - 1) if B is None else B
        self.S = (self.T - self.B) * self.C
        self.ctx = nqs.Context("heisenberg", lat.Lx, lat.Ly, J1=wl.ham.J1, J2=wl.ham.J2, marshall=wl.ham.marshall,
                               model="dense", widths=wl.widths, dtype=dtype)
        if self.C > 262144:
            self.ctx.set_option(nqs.OPT_MAX_ROWS, self.C)
        P = self.ctx.P
        self.n_grad = min(n_grad or self.S, self.S)
        self.params_h = torch.from_numpy(workloads.dense_params(self.N, wl.widths, wl.seed)).pin_memory()
        self.params = self.params_h.to(dev)
        z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device=dev)
        self.state, self.samples = z(self.C, self.ctx.W), z(self.S, self.ctx.W)
        self.nacc, self.eloc = z(self.C, dt=torch.int64), z(self.S, dt=torch.float32)
        self.stats, self.force = z(5, dt=torch.float64), z(P, dt=torch.float64)
        self.O = z(self.n_grad, P, dt=torch.float32)
        self.out_h = torch.zeros(5 + P, dtype=torch.float64).pin_memory()
        names = ["set_params+init", "sweep", "local_energy", "stats", "O_rows+force"]
        self.lam = minsr_lambda
        if self.lam:     # minSR on the O rows: statistics of those rows, then the solve
            names.append("minsr")
            self.stats_g = z(5, dt=torch.float64)
            self.dtheta = z(P, dt=torch.float64)
            self.ws_minsr = z(self.ctx.minsr_workspace(self.n_grad), dt=torch.uint8)
        self.ph = _Phased(torch, names)
        self.launches = None
        self.h2d, self.d2h = P * 8, (5 + P) * 8

    def run(self, seed, host_io=False):
        c, ph = self.ctx, self.ph
        if host_io:
            self.params.copy_(self.params_h, non_blocking=True)
        ph.mark(0)
        c.set_params(self.params)
        c.init_chains(self.state, seed)
        ph.mark(1)
        c.sweep(self.state, self.T, self.B, seed + 1, 0, self.samples, None, self.nacc)
        ph.mark(2)
        c.local_energy(self.samples, self.eloc)
        ph.mark(3)
        c.stats(self.eloc, self.C, self.stats, self.nacc, self.T * self.N)
        ph.mark(4)
        g = self.S - self.n_grad
        c.logpsi_grad(self.samples[g:], self.O, self.eloc[g:], self.stats, self.force)
        ph.mark(5)
        out = self.force
        if self.lam:
            c.stats(self.eloc[g:], self.n_grad, self.stats_g)
            c.minsr(self.O, self.eloc[g:], self.stats_g, self.lam, self.dtheta, workspace=self.ws_minsr)
            ph.mark(6)
            out = self.dtheta
        if host_io:
            self.out_h[:5].copy_(self.stats, non_blocking=True)
            self.out_h[5:].copy_(out, non_blocking=True)

    def units(self):
        return self.C * self.T * self.N

    def describe(self, ms, accepts, peaks_, n_sm):
        w, N = list(self.wl.widths), self.N
        f8 = self.dtype == "fp8"
        # algorithmic tensor-core FLOP per row: layers >= 1, unpadded widths (the padding of K to
        # the tile is not counted)
        gemm_row = sum(2.0 * w[l - 1] * w[l] for l in range(1, len(w)))
        n_conn = self.ctx.n_bonds
        sweep_flop = gemm_row * self.units()
        ach = sweep_flop / (ms["sweep"] / 1e3) / 1e12
        # FP8 products: the measured sustained BF16 rate x 2 (nominal dense FP8 / BF16 ratio)
        peak = float(peaks_.get("bf16_tflops_sustained", 1400.0)) * (2.0 if f8 else 1.0)
        eloc_flop = gemm_row * self.S * (1 + n_conn)
        lat = self.wl.ham.lattice
        return {
            "config": {"workload": self.wl.name, "lattice": f"{lat.Lx}x{lat.Ly} periodic", "J2": self.wl.ham.J2,
                       "widths": w, "chains": self.C, "sweeps": self.T, "burn_in": self.B, "samples": self.S,
                       "grad_rows": self.n_grad, "params": self.ctx.P},
            "local_energy": {"value": self.S / (ms["local_energy"] / 1e3), "unit": "samples/s",
                             "tensor_tflops": eloc_flop / (ms["local_energy"] / 1e3) / 1e12},
            "sweep": {"value": self.units() / (ms["sweep"] / 1e3), "unit": "proposals/s",
                      "acceptance": accepts / self.units()},
            "O_rows": {"GB_per_s": self.n_grad * self.ctx.P * 4 / (ms["O_rows+force"] / 1e3) / 1e9,
                       "note": "O rows written plus the force pass over them"},
            **({"minsr": {"samples": self.n_grad, "lambda": self.lam, "ms": ms["minsr"],
                          "gram_tflops_bf16x6": 6 * 2.0 * (self.n_grad ** 2 / 2 + self.n_grad * 64) * self.ctx.P
                          / (ms["minsr"] / 1e3) / 1e12,
                          "note": "whole solve (means, split, Gram, Cholesky, solves, dtheta); Gram FLOP counted "
                                  "as 6 BF16 products over the upper triangle"}} if self.lam else {}),
            "roofline": {"bound": "tensor",
                         "kernel": ("dense_gemm_kernel (sampler steps)" if len(w) != 2 or max(w) > 448
                                    else "dense_fused_sweep_kernel"), "achieved": ach,
                         "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "note": ("FP8 (E4M3) GEMM FLOP of layers >= 2 over all proposals / sweep time, vs 2 x the "
                                  "measured sustained cuBLAS BF16" if f8 else
                                  "BF16 GEMM FLOP of layers >= 2 over all proposals / sweep time, vs measured "
                                  "sustained cuBLAS BF16")},
            "energy": {"E": float(self.stats[0].item()), "err": float(self.stats[2].item()),
                       "note": "last timed step; local energy on the BF16 copy"},
        }


class BatchStep:
    """The 48 batched TFIM instances (FP16 sampling copies): one persistent sweep launch, then
    per instance local energies, statistics and last-sweep O rows, replayed as one CUDA graph."""

    def __init__(self, nqs, torch, dev):
        self.insts = workloads.batched_tfim_instances()
        self.T, self.B = self.insts[0].n_sweeps, self.insts[0].burn_in
        self.items, self.params = [], []
        K = self.T - self.B
        z = lambda *sh, dt=torch.int32: torch.zeros(sh, dtype=dt, device=dev)
        self.work = 0.0
        for w in self.insts:
            lat = w.ham.lattice
            N, M = lat.n_sites, w.n_hidden
            ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=w.ham.J1, h=w.ham.h, model="rbm", n_hidden=M, dtype="f16")
            ph = torch.from_numpy(workloads.rbm_params(N, M, w.weight_sigma, w.seed)).pin_memory()
            C = w.n_chains
            self.params.append((ctx, ph, ph.to(dev)))
            self.items.append(dict(ctx=ctx, state=z(C, ctx.W), seed=w.seed + 1, samples=z(K * C, ctx.W),
                                   n_accepted=z(C, dt=torch.int64), eloc=z(K * C, dt=torch.float32),
                                   stats=z(5, dt=torch.float64), O=z(C, ctx.P, dt=torch.float32), N=N, M=M, C=C))
            self.work += C * self.T * N * M
        for (ctx, _, pd), it in zip(self.params, self.items):
            ctx.set_params(pd)
            ctx.init_chains(it["state"], it["seed"])
        keys = ("ctx", "state", "seed", "samples", "n_accepted", "eloc", "stats", "O")
        self.batch = nqs.Batch([{k: it[k] for k in keys} for it in self.items], self.T, self.B, warps_per_cta=0)
        self.stats_h = torch.zeros(5 * len(self.items), dtype=torch.float64).pin_memory()
        self.ph = _Phased(torch, ["set_params+init", "step_graph"])
        self.launches = None
        self.S = sum(K * it["C"] for it in self.items)
        self.h2d = sum(ph.numel() * 8 for _, ph, _ in self.params)
        self.d2h = 5 * 8 * len(self.items)
        self.k = 0

    def run(self, seed, host_io=False):
        ph = self.ph
        ph.mark(0)
        for (ctx, p_h, p_d), it in zip(self.params, self.items):
            if host_io:
                p_d.copy_(p_h, non_blocking=True)
            ctx.set_params(p_d)
            ctx.init_chains(it["state"], seed + it["seed"])
        ph.mark(1)
        self.batch.step(self.k * self.T)
        self.k += 1
        ph.mark(2)
        if host_io:
            for q, it in enumerate(self.items):
                self.stats_h[5 * q:5 * q + 5].copy_(it["stats"], non_blocking=True)

    def units(self):
        return sum(it["C"] * self.T * it["N"] for it in self.items)

    def describe(self, ms, accepts, peaks_, n_sm):
        info = self.batch.info()
        return {
            "config": {"workload": "tfim_batched_48_instances", "instances": len(self.items),
                       "N": sorted({it["N"] for it in self.items}), "sweeps": self.T, "burn_in": self.B,
                       "chains_total": sum(it["C"] for it in self.items), "samples": self.S,
                       "batch": {k: info[k] for k in ("variant", "warps_per_cta", "n_work_items", "n_staged")}},
            "note": "value: proposals/s of the whole graphed step (sweep + local energies + statistics + O rows)",
            "roofline": None,
        }


def run_noisy_study(args, rank, world):
    """Noisy RBM (Sec. 4.1, Fig. 1(b, c)) on the 10 x 10, alpha = 4 model (FP32 sampling): for each
    sigma, the acceptance rate, the energy (local energies of the unperturbed psi over samples of
    |psi~|^2) and its shift from sigma = 0 with the Monte Carlo error, against the Pinsker bound
    sigma / 2 and the Theorem 3 bound (mu = 0, r = 0) on the sampled distribution."""
    import torch
    import paper_2601_20782_b300 as nqs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lat = WL.ham.lattice
    N, M = lat.n_sites, WL.n_hidden
    C, T, B = args.chains or 16384, args.sweeps or 100, 10 if args.burn_in is None else args.burn_in
    ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=WL.ham.J1, h=WL.ham.h, model="rbm", n_hidden=M, dtype="f32")
    ctx.set_params(torch.from_numpy(workloads.rbm_params(N, M, WL.weight_sigma, WL.seed)).to(dev))
    S = (T - B) * C
    state = torch.zeros((C, ctx.W), dtype=torch.int32, device=dev)
    samples = torch.zeros((S, ctx.W), dtype=torch.int32, device=dev)
    nacc = torch.zeros(C, dtype=torch.int64, device=dev)
    eloc = torch.zeros(S, dtype=torch.float32, device=dev)
    stats = torch.zeros(5, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sigmas = [0.0, 0.01, 0.03, 0.1, 0.3, 1.0, 3.0]
    rows, rate = [], {}
    with ClockSampler(dev.index) as clk:
        for sig in sigmas:
            ctx.set_noise(sig, WL.seed + 6)
            times = []
            for k in range(args.warmup + args.steps):
                flush.zero_()
                ctx.init_chains(state, WL.seed + 7)
                torch.cuda.synchronize()
                ev[0].record()
                ctx.sweep(state, T, B, WL.seed + 8, 0, samples, None, nacc)
                ev[1].record()
                torch.cuda.synchronize()
                if k >= args.warmup:
                    times.append(ev[0].elapsed_time(ev[1]))
            ctx.local_energy(samples, eloc)
            ctx.stats(eloc, C, stats, nacc, T * N)
            st = stats.cpu().numpy()
            rate[sig] = C * T * N / (statistics.median(times) / 1e3)
            rows.append({"sigma": sig, "acceptance": float(st[3]), "E": float(st[0]), "E_err": float(st[2]),
                         "pinsker_tv_bound": sig / 2, "thm3_tv_bound_r0": thm3_bound(0.0, sig),
                         "sweep_proposals_per_s": rate[sig]})
    e0 = rows[0]
    for r in rows:
        r["E_shift"] = r["E"] - e0["E"]
        r["E_shift_err"] = math.hypot(r["E_err"], e0["E_err"])
        r["rel_shift"] = abs(r["E_shift"]) / abs(e0["E"])
    return {
        "metric": METRIC, "value": rate[0.1], "unit": "proposals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": C * T * N / rate[0.1] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (noisy RBM: configuration-keyed Gaussian zeta)",
        "data": "synthetic (seeded random-init RBM, random initial spins)",
        "config": {"workload": "tfim2d_10x10_rbm_a4_noisy", "chains": C, "sweeps": T, "burn_in": B,
                   "sigmas": sigmas, "l2": "flushed between timed sweeps (256 MiB write)", "parallelism": "dp1"},
        "note": "value: noisy-sampler proposals/s at sigma = 0.1; the study is in `noisy`",
        "noisy": rows, "roofline": None, "clocks": clk.summary(),
    }


def run_rbm_grid(args, rank, world):
    """The sampling grid of Sec. 4.2 (Fig. 4) on the 10 x 10 TFIM RBM: sweep proposals/s of the
    FP32, BF16 and F16 copies against the number of samples N_s (N_s / 4 chains, four kept
    samples per chain after four burn-in sweeps) and the hidden-unit density alpha, and the
    16-bit copies' ratio to FP32 (the paper's ratios are to an FP64 copy, which is not built)."""
    import torch
    import paper_2601_20782_b300 as nqs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    lat = WL.ham.lattice
    N = lat.n_sites
    T, B = 8, 4
    alphas = [1, 2, 4, 8]
    n_samples = [4 * 1024, 4 * 4096, 4 * 16384, 4 * 65536] if not args.chains else [4 * args.chains]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rows = []
    with ClockSampler(dev.index) as clk:
        for alpha in alphas:
            M = alpha * N
            params = torch.from_numpy(workloads.rbm_params(N, M, WL.weight_sigma, WL.seed)).to(dev)
            ctxs = {}
            for dt in ("f32", "bf16", "f16"):
                ctxs[dt] = nqs.Context("tfim", lat.Lx, lat.Ly, J1=WL.ham.J1, h=WL.ham.h, model="rbm", n_hidden=M,
                                       dtype=dt)
                ctxs[dt].set_params(params)
            for ns in n_samples:
                C = ns // 4
                row = {"alpha": alpha, "n_samples": ns, "chains": C}
                for dt, ctx in ctxs.items():
                    state = torch.zeros((C, ctx.W), dtype=torch.int32, device=dev)
                    samples = torch.zeros(((T - B) * C, ctx.W), dtype=torch.int32, device=dev)
                    times = []
                    for k in range(args.warmup + args.steps):
                        flush.zero_()
                        ctx.init_chains(state, WL.seed + 7)
                        torch.cuda.synchronize()
                        ev[0].record()
                        ctx.sweep(state, T, B, WL.seed + 8, 0, samples)
                        ev[1].record()
                        torch.cuda.synchronize()
                        if k >= args.warmup:
                            times.append(ev[0].elapsed_time(ev[1]))
                    row[dt] = C * T * N / (statistics.median(times) / 1e3)
                row["bf16_over_f32"] = row["bf16"] / row["f32"]
                row["f16_over_f32"] = row["f16"] / row["f32"]
                rows.append(row)
    top = max(rows, key=lambda r: r["f16"])
    return {
        "metric": METRIC, "value": top["f16"], "unit": "proposals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": top["chains"] * T * N / top["f16"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 sampling (f32 caches, accept); FP32 and BF16 beside it",
        "data": "synthetic (seeded random-init RBMs, random initial spins)",
        "config": {"workload": "tfim2d_10x10_rbm_grid", "lattice": "10x10 periodic", "h": WL.ham.h,
                   "alphas": alphas, "n_samples": n_samples, "samples_per_chain": T - B, "sweeps": T, "burn_in": B,
                   "l2": "flushed between timed sweeps (256 MiB write)", "parallelism": "dp1 (chains)"},
        "note": "value: the largest F16 sweep rate of the grid; the grid is in `rbm_grid`",
        "rbm_grid": rows, "roofline": None, "clocks": clk.summary(),
    }


def run_delta_study(args, rank, world):
    """App. D (the random-state panel of its sigma(delta) figure): the spread of
    delta(x) = log |psi~(x)|^2 - log |psi(x)|^2 of the BF16 and F16 RBM copies against the chain
    length N, for a randomly initialised RBM with alpha = 1 (weights N(0, 0.1^2)) on 1D TFIM
    chains, over uniform random configurations (the flat distribution such a state is close to);
    log psi through nqs_logpsi of each copy, the FP32 context as the reference (its own error is
    about 1e-6, far below the 16-bit copies')."""
    import torch
    import paper_2601_20782_b300 as nqs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sizes = [16, 32, 64, 128, 256]
    n = args.chains or 65536
    g = torch.Generator(device=dev).manual_seed(WL.seed + 9)
    rows = []
    with ClockSampler(dev.index) as clk:
        for N in sizes:
            params = torch.from_numpy(workloads.rbm_params(N, N, 0.1, WL.seed + N)).to(dev)
            lp = {}
            for dt in ("f32", "bf16", "f16"):
                ctx = nqs.Context("tfim", N, 1, J1=1.0, h=1.0, model="rbm", n_hidden=N, dtype=dt)
                ctx.set_params(params)
                if dt == "f32":  # uniform configurations: random words, bits beyond N cleared
                    W = ctx.W
                    cfg = torch.randint(-2 ** 31, 2 ** 31, (n, W), generator=g, device=dev, dtype=torch.int64)
                    cfg = cfg.to(torch.int32)
                    last = N - 32 * (W - 1)
                    if last < 32:
                        cfg[:, W - 1] &= (1 << last) - 1
                out = torch.empty(n, dtype=torch.float32, device=dev)
                ctx.logpsi(cfg, out)
                lp[dt] = out.double()
            row = {"N": N, "alpha": 1}
            for dt in ("bf16", "f16"):
                d = 2.0 * (lp[dt] - lp["f32"])
                sd = float(d.std())
                row["sigma_delta_" + dt] = sd
                row["pinsker_tv_bound_" + dt] = sd / 2
            rows.append(row)
    return {
        "metric": METRIC, "value": None, "unit": "proposals/s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 and f16 RBM copies against the fp32 context",
        "data": "synthetic (seeded random-init RBMs, uniform random configurations)",
        "config": {"workload": "tfim1d_rbm_a1_delta_study", "sizes": sizes, "configurations": n,
                   "weight_sigma": 0.1, "parallelism": "dp1"},
        "note": "the study is in `delta_study` (sigma of delta per copy against N); no rate is measured",
        "delta_study": rows, "roofline": None, "clocks": clk.summary(),
    }


def run_rescnn_study(args, rank, world):
    """App. H sampling study of the ResCNN (4 blocks x 16 filters, 3 x 3) on the 4 x 4 TFIM: the
    sweep's proposals/s for the FP32, BF16 and F16 copies against the number of chains N_s,
    and the 16-bit copies' speed-up over FP32.  The kernels have 16 channels, so the filter
    count is not varied."""
    import torch
    import paper_2601_20782_b300 as nqs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = workloads.RESCNN_2D_10x10
    lat = wl.extra["small_case"]
    F, nb = wl.extra["filters"], wl.extra["blocks"]
    T = args.sweeps or 10
    params = torch.from_numpy(workloads.rescnn_params(F, nb, wl.seed)).to(dev)
    counts = [256, 1024, 4096, 16384, 65536] if not args.chains else [args.chains]
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rows = []
    with ClockSampler(dev.index) as clk:
        for C in counts:
            row = {"chains": C}
            for dt in ("f32", "bf16", "f16"):
                ctx = nqs.Context("tfim", lat.Lx, lat.Ly, J1=wl.ham.J1, h=wl.ham.h, model="rescnn", n_hidden=F,
                                  n_blocks=nb, dtype=dt)
                ctx.set_params(params)
                state = torch.zeros((C, ctx.W), dtype=torch.int32, device=dev)
                nacc = torch.zeros(C, dtype=torch.int64, device=dev)
                times = []
                for k in range(args.warmup + args.steps):
                    flush.zero_()
                    ctx.init_chains(state, wl.seed + 7)
                    torch.cuda.synchronize()
                    ev[0].record()
                    ctx.sweep(state, T, T, wl.seed + 8, 0, None, None, nacc)
                    ev[1].record()
                    torch.cuda.synchronize()
                    if k >= args.warmup:
                        times.append(ev[0].elapsed_time(ev[1]))
                row[dt] = C * T * lat.n_sites / (statistics.median(times) / 1e3)
            row["speedup_bf16"] = row["bf16"] / row["f32"]
            row["speedup_f16"] = row["f16"] / row["f32"]
            rows.append(row)
    top = rows[-1]
    return {
        "metric": METRIC, "value": top["f16"], "unit": "proposals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": top["chains"] * T * lat.n_sites / top["f16"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 (convolutions on tcgen05, FP32 accumulation; FP32 and BF16 beside it)",
        "data": "synthetic (seeded random-init ResCNN, random initial spins)",
        "config": {"workload": "rescnn_tfim2d_4x4_4blocks_16filters_study", "lattice": "4x4 periodic",
                   "filters": F, "blocks": nb, "sweeps": T, "chains": counts,
                   "l2": "flushed between timed sweeps (256 MiB write)", "parallelism": "dp1 (chains)"},
        "note": "value: F16 sweep proposals/s at the largest chain count; the study is in `rescnn_study`",
        "rescnn_study": rows, "roofline": None, "clocks": clk.summary(),
    }


def run_workload(args, rank, world, dist):
    import torch
    import paper_2601_20782_b300 as nqs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    C, T, B = args.chains or None, args.sweeps or None, args.burn_in   # profiling overrides (smaller cases)
    if args.workload == "tfim1d":
        st = RbmStep(nqs, torch, dev, workloads.TFIM_1D_N16, "f32", C, T, B)
    elif args.workload == "heis2d-dense":
        st = DenseStep(nqs, torch, dev, workloads.HEIS_2D_10x10, C, T, B,
                       dtype="fp8" if args.dtype == "fp8" else "bf16")
    elif args.workload == "j1j2-dense":
        wl = workloads.J1J2_2D_16x16
        st = DenseStep(nqs, torch, dev, wl, C, T or 2, 1 if B is None else B,
                       n_grad=args.grad_rows or wl.extra["minsr_samples"], minsr_lambda=1e-3,
                       dtype="fp8" if args.dtype == "fp8" else "bf16")
    elif args.workload == "crbm-tfim2d":
        st = ComplexRbmStep(nqs, torch, dev, WL, C, T, B)
    elif args.workload == "rescnn-tfim2d":
        st = RescnnStep(nqs, torch, dev, workloads.RESCNN_2D_10x10, args.dtype, C, T, B)
    else:
        st = BatchStep(nqs, torch, dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    base = 1000 + rank * 7919
    for w in range(args.warmup):
        st.run(base + w)
    torch.cuda.synchronize()
    tot, acc = {}, 0
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            st.run(base + 100 + k)
            torch.cuda.synchronize()
            for n, v in st.ph.ms().items():
                tot[n] = tot.get(n, 0.0) + v
            if isinstance(st, BatchStep):
                acc += sum(int(it["n_accepted"].sum().item()) for it in st.items)
            else:
                acc += int(st.nacc.sum().item())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    t_dev = sum(tot.values()) / 1e3
    e2e = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.run(base + 200 + k, host_io=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    t_e2e = sum(e2e)
    if dist:
        tt = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = tt.tolist()
    ms = {n: v / args.steps for n, v in tot.items()}
    pk = dict(peaks())
    if isinstance(st, (RbmStep, ComplexRbmStep)) or (isinstance(st, RescnnStep) and st.dtype == "f32"):
        pk["alu"] = measure_alu_peaks(nqs, torch, dev)
    d = st.describe(ms, acc / args.steps, pk, torch.cuda.get_device_properties(dev).multi_processor_count)
    units = st.units()
    line = {"metric": METRIC, "value": world * units * args.steps / t_dev, "unit": "proposals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"tfim1d": "f32",
                      "heis2d-dense": ("fp8 e4m3 sampling (bf16 local energy, " if args.dtype == "fp8" else "bf16 (")
                      + "fp32 accumulate, fp32 layer-0 cache)",
                      "j1j2-dense": ("fp8 e4m3 sampling (bf16 local energy, " if args.dtype == "fp8" else "bf16 (")
                      + "fp32 accumulate, fp32 layer-0 cache)",
                      "batched": "f16 sampling (f32 caches, accept, statistics)",
                      "crbm-tfim2d": "complex f32 (f64 statistics and force accumulation)",
                      "rescnn-tfim2d": {"f32": "f32 (CUDA cores)", "bf16": "bf16 convolutions on tcgen05 (fp32 "
                                        "accumulate, LN, residual stream)", "f16": "f16 convolutions on tcgen05 "
                                        "(fp32 accumulate, LN, residual stream)"}.get(args.dtype, args.dtype)
                      }[args.workload],
            "data": "synthetic (seeded random-init networks, random initial spins)"}
    line.update(d)
    if args.chains or args.sweeps or args.burn_in is not None or args.grad_rows:
        line["config"]["workload"] += " (reduced: profiling)"
    line["config"]["l2"] = "flushed between timed steps (256 MiB write)"
    line["config"]["parallelism"] = f"dp{world} (chains)"
    line["phases_ms"] = ms
    line["e2e"] = {"value": world * units * args.steps / t_e2e, "unit": "proposals/s",
                   "h2d_bytes_per_step": st.h2d, "d2h_bytes_per_step": st.d2h}
    if st.launches:
        line["gpu_launches"] = st.launches * args.steps
    line["clocks"] = clk.summary()
    if isinstance(st, RescnnStep) and args.compare:   # the other sampling copies, same sizes and steps
        line["compare"] = {}
        for d in ("f32", "bf16", "f16"):
            if d == args.dtype:
                continue
            o = RescnnStep(nqs, torch, dev, workloads.RESCNN_2D_10x10, d, C, T, B)
            for w in range(args.warmup):
                o.run(base + w)
            tot2 = {}
            for k in range(args.steps):
                flush.zero_()
                o.run(base + 100 + k)
                torch.cuda.synchronize()
                for n, v in o.ph.ms().items():
                    tot2[n] = tot2.get(n, 0.0) + v
            ms2 = {n: v / args.steps for n, v in tot2.items()}
            line["compare"][d] = {"value": world * o.units() / (sum(ms2.values()) / 1e3),
                                  "sweep_proposals_per_s": world * o.units() / (ms2["sweep"] / 1e3),
                                  "local_energy_samples_per_s": world * o.S / (ms2["local_energy"] / 1e3),
                                  "E": float(o.stats[0].item()), "E_err": float(o.stats[2].item())}
        if "f32" in line["compare"]:
            f32 = line["compare"]["f32"]
            line["mixed_vs_f32"] = {"sweep": line["sweep"]["value"] / f32["sweep_proposals_per_s"],
                                    "local_energy": line["local_energy"]["value"] / f32["local_energy_samples_per_s"],
                                    "step": line["value"] / f32["value"],
                                    "energy_minus_f32": line["energy"] - f32["E"],
                                    "energy_err": math.hypot(float(st.stats[2].item()), f32["E_err"])}
    return line


def _oracle_cmd(n_chains, n_sweeps, eloc_samples, chain0=0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; print(json.dumps(bench.oracle_sample(%d, %d, %d, %d)))"
            % (n_chains, n_sweeps, eloc_samples, chain0))
    return [sys.executable, "-c", code], env


def oracle_sample_subprocess(n_chains, n_sweeps, eloc_samples):
    """oracle_sample in a fresh interpreter pinned to one BLAS / OpenMP thread."""
    cmd, env = _oracle_cmd(n_chains, n_sweeps, eloc_samples)
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_all_cores(n_chains, n_sweeps, eloc_samples, max_workers=64):
    """The oracle on every host core at once: one single-threaded interpreter per core, each on
    its own block of chains (distinct chain ids), started together.  The aggregate rate is the
    sum of the workers' own rates, each measured inside the worker over its sampling (the
    windows overlap; interpreter start-up is not counted)."""
    workers = max(1, min(os.cpu_count() or 1, max_workers))
    procs = []
    for w in range(workers):
        cmd, env = _oracle_cmd(n_chains, n_sweeps, eloc_samples, w * n_chains)
        procs.append(subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True))
    outs = []
    for pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle worker failed")
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return {"proposals_per_s": sum(o["proposals_per_s"] for o in outs),
            "eloc_samples_per_s": sum(o["eloc_samples_per_s"] for o in outs), "cores": workers,
            "sample": f"{workers} workers x ({outs[0]['sample']})"}


def oracle_sample(n_chains, n_sweeps, eloc_samples, chain0=0):
    """The FP64 oracle on a bounded sample of the same workload; returns rates."""
    from oracle.estimators import local_energy
    from oracle.hamiltonian import make_hamiltonian
    from oracle.models import RBM
    from oracle.philox import init_spins_random
    from oracle.sampler import mh_sweeps
    lat = WL.ham.lattice
    N, M = lat.n_sites, WL.n_hidden
    model = RBM(N, M, workloads.rbm_params(N, M, WL.weight_sigma, WL.seed))
    ham = make_hamiltonian(WL.ham)
    ids = chain0 + np.arange(n_chains)
    s0 = init_spins_random(WL.seed, ids, N)
    t0 = time.perf_counter()
    out = mh_sweeps(model.logpsi, s0, ids, WL.seed + 1, n_sweeps, 0)
    t_sweep = time.perf_counter() - t0
    t0 = time.perf_counter()
    local_energy(ham, model.logpsi, out["samples"][:eloc_samples])
    t_eloc = time.perf_counter() - t0
    return {"proposals_per_s": n_chains * n_sweeps * N / t_sweep,
            "eloc_samples_per_s": eloc_samples / t_eloc, "t": t_sweep + t_eloc,
            "sample": f"{n_chains} chains x {n_sweeps} sweeps of the 10x10 alpha=4 workload "
                      f"(full re-evaluation per proposal) + local energy of {eloc_samples} samples"}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on every host core at once (one
    interpreter per core, as the cpu_baseline leg), each step a bounded sample of the default
    workload; the config is the default line's."""
    per = [oracle_sample_all_cores(256, 6, 256) for _ in range(args.warmup + args.steps)][args.warmup:]
    v = statistics.median(p["proposals_per_s"] for p in per)
    lat = WL.ham.lattice
    N, M = lat.n_sites, WL.n_hidden
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-init RBM, random initial spins)",
        "config": {"workload": WL.name, "lattice": f"{lat.Lx}x{lat.Ly} periodic", "h": WL.ham.h, "n_hidden": M,
                   "chains": WL.n_chains, "sweeps": WL.n_sweeps, "burn_in": WL.burn_in,
                   "samples": (WL.n_sweeps - WL.burn_in) * WL.n_chains, "params": workloads.rbm_n_params(N, M),
                   "parallelism": "host cores (chains)", "sample_per_step": per[0]["sample"]},
        "local_energy": {"value": statistics.median(p["eloc_samples_per_s"] for p in per), "unit": "samples/s"},
        "cpu_baseline": {"value": v, "unit": "proposals/s", "cores": per[0]["cores"], "kind": "oracle",
                         "sample": per[0]["sample"]},
        "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f16", choices=["f32", "bf16", "f16", "fp8"],
                    help="sampling copy of the timed step (the mixed-precision path by default)")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the FP32 / other-dtype comparison steps and the bias statement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chains", type=int, default=0, help="profiling only: override the chain count")
    ap.add_argument("--sweeps", type=int, default=0, help="profiling only: override the sweep count")
    ap.add_argument("--burn-in", type=int, default=None, help="profiling only: override the burn-in")
    ap.add_argument("--grad-rows", type=int, default=0, help="profiling only (j1j2-dense): O rows / minSR samples")
    ap.add_argument("--chains-per-warp", type=int, default=0, choices=[0, 1, 2],
                    help="profiling only (tfim2d): RBM sweep chains per warp of the FP32 copy (0: built-in rule)")
    ap.add_argument("--workload", default="tfim2d", choices=["tfim2d", "tfim1d", "heis2d-dense", "batched",
                                                             "j1j2-dense", "noisy-rbm", "crbm-tfim2d", "rescnn-tfim2d",
                                                             "rescnn-study", "rbm-grid", "delta-study"],
                    help="tfim2d: the 10x10 alpha=4 RBM workload (default); the others measure the other "
                         "workloads' steps with the same line")
    args = ap.parse_args()
    if args.dtype == "fp8" and args.workload not in ("heis2d-dense", "j1j2-dense"):
        ap.error("--dtype fp8 is the dense ansatz's FP8 sampling copy (--workload heis2d-dense or j1j2-dense)")
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    rank = int(os.environ.get("RANK", 0))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    if args.workload == "noisy-rbm":
        if rank == 0:
            print(json.dumps(run_noisy_study(args, rank, world)), flush=True)
        return
    if args.workload == "rescnn-study":
        if rank == 0:
            print(json.dumps(run_rescnn_study(args, rank, world)), flush=True)
        return
    if args.workload == "rbm-grid":
        if rank == 0:
            print(json.dumps(run_rbm_grid(args, rank, world)), flush=True)
        return
    if args.workload == "delta-study":
        if rank == 0:
            print(json.dumps(run_delta_study(args, rank, world)), flush=True)
        return
    if args.workload != "tfim2d":
        line = run_workload(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        if not args.no_cpu_baseline:
            cb = oracle_sample_all_cores(256, 6, 256)
            one = oracle_sample_subprocess(1024, 8, 1024)
            line["cpu_baseline"] = {"value": cb["proposals_per_s"], "unit": "proposals/s", "cores": cb["cores"],
                                    "kind": "oracle", "sample": cb["sample"],
                                    "local_energy_samples_per_s": cb["eloc_samples_per_s"],
                                    "one_core": {"value": one["proposals_per_s"], "unit": "proposals/s",
                                                 "local_energy_samples_per_s": one["eloc_samples_per_s"],
                                                 "sample": one["sample"]}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
