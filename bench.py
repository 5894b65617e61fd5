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


def reduce_stats_across_ranks(stats, n_local, dist):
    """Energy statistics over all ranks' samples, in place: an FP64 all-reduce of
    (n, n * mean, n * (var + mean^2), (n * err)^2).  Afterwards stats[0] is the global E,
    so every rank's force (1/n_r) sum_x O(x) (eps(x) - E) uses the same E."""
    import torch
    n_r = float(n_local)
    buf = torch.cat([torch.tensor([n_r], dtype=torch.float64, device=stats.device),
                     stats[:1] * n_r, (stats[1:2] + stats[:1] ** 2) * n_r, (stats[2:3] * n_r) ** 2])
    dist.all_reduce(buf)
    n = buf[0]
    mean = buf[1] / n
    stats[0] = mean
    stats[1] = buf[2] / n - mean ** 2
    stats[2] = torch.sqrt(buf[3]) / n
    return n


def reduce_force_across_ranks(force, n_local, n_total, dist):
    """F = (1/n) sum over all ranks of n_r F_r, exact when every F_r was centred on the
    global E (reduce_stats_across_ranks first); in place."""
    force.mul_(float(n_local))
    dist.all_reduce(force)
    force.div_(float(n_total))


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
        self.force = torch.zeros(P, dtype=torch.float64, device=dev)
        self.O = torch.zeros((C, P), dtype=torch.float32, device=dev)
        self.ws = torch.zeros(self.ctx.logpsi_grad_workspace(self.S), dtype=torch.uint8, device=dev)
        self.out_h = torch.zeros(5 + P, dtype=torch.float64).pin_memory()
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        self.launches = 2 + 1 + 1 + 1 + 2 + 2 + 1   # set_params, init, sweep, eloc, stats, force, O rows

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
        c.local_energy(self.samples, self.eloc)
        ev[3].record()
        c.stats(self.eloc, self.C, self.stats, self.nacc, self.T * self.N)
        if self.dist:   # the one exchange of the step: global E first, then the force
            n_total = reduce_stats_across_ranks(self.stats, self.S, self.dist)
        c.logpsi_grad(self.samples, None, self.eloc, self.stats, self.force, self.ws)
        if self.dist:
            reduce_force_across_ranks(self.force, self.S, n_total, self.dist)
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
                       "energy_vs_f32": dE, "energy_err": math.hypot(results[d]["E_err"], results["f32"]["E_err"]),
                       "sweep_speed_vs_f32": (results["f32"]["phase"][1] / results[d]["phase"][1])}

    r = results[args.dtype]
    ph = r["phase"]   # ms per phase: prep+init, sweep, eloc, stats+force, O rows
    value = world * proposals_step * args.steps / r["t_dev"]
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # Sweep roofline (arithmetic of the method per proposal): one FMA (factor) and one multiply
    # (product) per hidden unit, three multiplies per hidden unit per accepted flip, counted as
    # lane operations; peak = SMs x 128 FP32 lanes x max SM clock.
    alg_ops = 2.0 * M * proposals_step + 3.0 * M * r["accepts"]
    achieved = alg_ops / (ph[1] / 1e3) / 1e12
    peak = n_sm * 128 * sm_max * 1e6 / 1e12
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
                     "unit": "T lane-ops/s", "frac": achieved / peak, "traffic": None,
                     "note": "method arithmetic per proposal (2M + 3M per accept) vs SMs x 128 FP32 lanes x max clock"},
        "e2e": {"value": world * proposals_step * args.steps / t_e2e, "unit": "proposals/s",
                "h2d_bytes_per_step": steps[args.dtype].ctx.P * 8, "d2h_bytes_per_step": (5 + steps[args.dtype].ctx.P) * 8},
        "gpu_launches": steps[args.dtype].launches * args.steps,
        "clocks": r["clocks"],
    }
    return line


def oracle_sample_subprocess(n_chains, n_sweeps, eloc_samples):
    """oracle_sample in a fresh interpreter pinned to one BLAS / OpenMP thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; print(json.dumps(bench.oracle_sample(%d, %d, %d)))"
            % (n_chains, n_sweeps, eloc_samples))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(n_chains, n_sweeps, eloc_samples):
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
    s0 = init_spins_random(WL.seed, np.arange(n_chains), N)
    t0 = time.perf_counter()
    out = mh_sweeps(model.logpsi, s0, np.arange(n_chains), WL.seed + 1, n_sweeps, 0)
    t_sweep = time.perf_counter() - t0
    t0 = time.perf_counter()
    local_energy(ham, model.logpsi, out["samples"][:eloc_samples])
    t_eloc = time.perf_counter() - t0
    return {"proposals_per_s": n_chains * n_sweeps * N / t_sweep,
            "eloc_samples_per_s": eloc_samples / t_eloc, "t": t_sweep + t_eloc,
            "sample": f"{n_chains} chains x {n_sweeps} sweeps of the 10x10 alpha=4 workload "
                      f"(full re-evaluation per proposal) + local energy of {eloc_samples} samples"}


def run_reference(args):
    per = [oracle_sample_subprocess(1024, 5, 512) for _ in range(args.warmup + args.steps)][args.warmup:]
    v = statistics.median(p["proposals_per_s"] for p in per)
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WL.name},
        "ms_per_step": statistics.median(p["t"] for p in per) * 1e3,
        "local_energy": {"value": statistics.median(p["eloc_samples_per_s"] for p in per), "unit": "samples/s"},
        "cpu_baseline": {"value": v, "unit": "proposals/s", "cores": 1, "kind": "oracle",
                         "sample": per[0]["sample"]},
        "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f16", choices=["f32", "bf16", "f16"],
                    help="sampling copy of the timed step (the mixed-precision path by default)")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the FP32 / other-dtype comparison steps and the bias statement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chains", type=int, default=0, help="profiling only: override the chain count")
    ap.add_argument("--sweeps", type=int, default=0, help="profiling only: override the sweep count")
    ap.add_argument("--burn-in", type=int, default=None, help="profiling only: override the burn-in")
    args = ap.parse_args()
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
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        if not args.no_cpu_baseline:
            cb = oracle_sample_subprocess(1024, 8, 1024)
            line["cpu_baseline"] = {"value": cb["proposals_per_s"], "unit": "proposals/s", "cores": 1,
                                    "kind": "oracle", "sample": cb["sample"],
                                    "local_energy_samples_per_s": cb["eloc_samples_per_s"]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
