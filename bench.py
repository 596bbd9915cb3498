#!/usr/bin/env python
"""Benchmark: Lanczos steps/s of the Liouville-Lanczos hot path on one GB300.

Workload (default): the C2 CrI3-shaped synthetic crystal -- hexagonal a = 13 bohr,
c = 30 bohr (vacuum slab), FFT 36x36x96, ~5000 plane waves per spinor component,
4x4 k grid (16 k), 40 occupied spinor bands, 8 atoms x 8 KB projectors with
spin-orbit, q = (1/8, 0, 0) 2pi/a.  A step is one pseudo-Hermitian Lanczos
iteration of one chain (one Liouvillian application + the FP64 scalar update).

Reported (one JSON line on rank 0):
  value          mixed-precision steps/s (FP32 vectors and arithmetic, FP64 scalars)
  fp64           the FP64 path's steps/s
  chi_rel_err    ||chi_mixed - chi_fp64|| / ||chi_fp64|| at eta = 10 meV on 0-100 meV
  roofline       dominant stage of the mixed step against the measured HBM peak
  cpu_baseline   the FP64 CPU oracle on a one-k-point sample of the same workload
  e2e            host ground state in -> coefficients out, through the C ABI

--impl reference runs the oracle (CPU) as the reference arm.
Multi-GPU: replicas only (independent chains, no collective): value sums ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lanczos steps/s and %HBM roofline, mixed vs FP64 at rel chi(w) err <=1e-4"
WORKLOAD = ("C2: hexagonal a=13 c=30 bohr, FFT 36x36x96, ~5000 PW/component, 4x4 k, "
            "Nocc=40, 8 atoms x 8 KB projectors with SOC, q=(1/8,0,0) 2pi/a, PH Lanczos")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tdlz", choices=["tdlz", "reference"])
    ap.add_argument("--config", default="C2")
    ap.add_argument("--flavor", default="phm", choices=["ph", "phm", "nh"])
    ap.add_argument("--chi-steps", type=int, default=60)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.samples = []
        self.stop = threading.Event()
        self.th = None

    def start(self):
        def run():
            while not self.stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.idx),
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits"],
                                         capture_output=True, text=True, timeout=5).stdout
                    self.samples.append([v.strip() for v in out.strip().split(",")])
                except Exception:
                    pass
                self.stop.wait(0.2)
        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()

    def finish(self):
        self.stop.set()
        if self.th:
            self.th.join(timeout=10)
        sm = [float(s[0]) for s in self.samples if s and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) > 1 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, n in enumerate(names):
                if len(s) > 3 + i and s[3 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def make_workload(cfg, tol):
    from synth import make_ground_state
    t = time.time()
    gs = make_ground_state(cfg, tol=tol, log=log)
    log(f"[bench] ground state {cfg}: npwx={gs.npwx} nk={gs.nk} nocc={gs.nocc} "
        f"gap={gs.meta['gap_min']:.3e} resid={gs.meta['resid_max']:.2e} "
        f"({time.time() - t:.1f} s)")
    return gs


def sample_bundle(gs, nk_sample=1):
    """The first nk_sample k points of a bundle (weights kept at 1/Nk)."""
    import dataclasses
    s = slice(0, nk_sample)
    return dataclasses.replace(
        gs, nk=nk_sample, kpts=gs.kpts[s], wk=gs.wk[s], npw_k=gs.npw_k[s], npw_kq=gs.npw_kq[s],
        miller_k=gs.miller_k[s], miller_kq=gs.miller_kq[s], evals=gs.evals[:, s],
        evals_kq=gs.evals_kq[:, s], coeff_k=gs.coeff_k[:, s], coeff_kq=gs.coeff_kq[:, s],
        beta_kq=gs.beta_kq[s])


def oracle_step_time(gs, nsteps=1, flavor="phm"):
    """Seconds per Lanczos step of the FP64 oracle on a one-k-point sample, scaled by nk."""
    from oracle.liouvillian import Liouvillian
    from oracle.lanczos import lanczos_nh, lanczos_ph, lanczos_phm
    sub = sample_bundle(gs, 1)
    lv = Liouvillian(sub)
    v = lv.start_vector(0)
    u = [lv.left_vector(l) for l in range(3)]
    t = time.perf_counter()
    if flavor == "nh":
        lanczos_nh(lv.apply, lv.apply_adjoint, v, u, nsteps)
    elif flavor == "ph":
        lanczos_ph(lv.apply, v, u, nsteps)
    else:
        lanczos_phm(lv.apply, v, u, nsteps)
    el = time.perf_counter() - t
    # phm spends one extra L product before its first step; count it as a step
    per = el / (nsteps + (1 if flavor == "phm" else 0))
    return per * gs.nk, el


def cpu_info():
    cores = len(os.sched_getaffinity(0))
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    gs = make_workload(args.config, args.tol)
    cores, model = cpu_info()
    times = []
    for i in range(args.warmup + args.steps):
        per, _ = oracle_step_time(gs, 1, args.flavor)
        if i >= args.warmup:
            times.append(per)
    t = sum(times)
    value = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "flavor": args.flavor},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: one oracle Lanczos step restricted to k point 0 "
                                   f"of {gs.nk}, time x {gs.nk} (cost is linear in k)",
                         "cpu": model},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def chain_steps_per_s(ctx, q, mu, flavor, precision, warmup, steps, profile=False):
    import torch  # noqa: F401
    ch = ctx.chain_create([q], [mu], warmup + steps + 1, flavor, precision)
    try:
        ch.advance(warmup)
        ctx.synchronize()
        if profile:
            ctx.profile(True)
        l0 = ctx.launch_count()
        start = __import__("torch").cuda.Event(enable_timing=True)
        end = __import__("torch").cuda.Event(enable_timing=True)
        # the library runs on its own stream; bracket with device syncs + events on it
        ctx.synchronize()
        t0 = time.perf_counter()
        ch.advance(steps)
        ctx.synchronize()
        wall = time.perf_counter() - t0
        launches = ctx.launch_count() - l0
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(False)
        res = ch.read()
        del start, end
        return steps / wall, wall, launches, prof, res
    finally:
        ch.close()


def run_tdlz(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2203_01120_gb300 import TDLZ_FP64, TDLZ_MIXED, Context, build_ext
    build_ext.build()
    gs = make_workload(args.config, args.tol)
    mu = rank % 3  # replicas: each rank runs its own column of chi
    ctx = Context(local)
    # ------------------------------------------------------------ e2e (host in/out)
    t0 = time.perf_counter()
    q = ctx.load_ground_state(gs)
    ch = ctx.chain_create([q], [mu], args.steps, args.flavor, TDLZ_MIXED)
    ch.advance(args.steps)
    res_e2e = ch.read()
    e2e_wall = time.perf_counter() - t0
    ch.close()
    bundle_bytes = sum(int(np.asarray(getattr(gs, k)).nbytes) for k in (
        "kpts", "wk", "npw_k", "npw_kq", "miller_k", "miller_kq", "evals", "coeff_k", "coeff_kq",
        "vloc", "bfield", "n0", "m0", "beta_kq", "dnl"))
    coef_bytes = args.steps * (16 * 2 + 8 + 16 * 3)
    # ------------------------------------------------------------ device-resident timing
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    sps_mixed, wall_mixed, launches, _, _ = chain_steps_per_s(
        ctx, q, mu, args.flavor, TDLZ_MIXED, args.warmup, args.steps)
    clocks = clk.finish()
    if world > 1:
        t = torch.tensor([wall_mixed], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        wall_mixed = float(t.item())
    # profiled pass (per-stage CUDA events on the library stream) for the roofline
    _, _, _, prof, _ = chain_steps_per_s(ctx, q, mu, args.flavor, TDLZ_MIXED, 1, args.steps,
                                         profile=True)
    fp64_steps = max(3, args.steps // 4)
    sps_fp64, wall_fp64, _, prof64, _ = chain_steps_per_s(ctx, q, mu, args.flavor, TDLZ_FP64, 1,
                                                          fp64_steps, profile=True)
    # ------------------------------------------------------------ chi error mixed vs FP64
    m = args.chi_steps
    r64 = ctx.lanczos_run([q], [mu], m, args.flavor, TDLZ_FP64)
    r32 = ctx.lanczos_run([q], [mu], m, args.flavor, TDLZ_MIXED)
    c64 = ctx.spectrum(r64, 0.0, 100.0, 0.1, 10.0, units=1)[0]
    c32 = ctx.spectrum(r32, 0.0, 100.0, 0.1, 10.0, units=1)[0]
    chi_err = float(np.linalg.norm(c32 - c64) / np.linalg.norm(c64[mu]))
    ctx.close()
    if rank != 0:
        return
    hbm, peak_src = measured_peaks()
    # dominant stage of the mixed step
    stages = {k: v for k, v in prof.items() if v["launches"] > 0 and v["ms"] > 0}
    top = max(stages, key=lambda k: stages[k]["ms"])
    st = stages[top]
    nl = st["launches"]
    per_launch_s = st["ms"] / 1000.0 / nl
    bytes_launch = st["bytes"] / nl
    achieved = bytes_launch / per_launch_s / 1e9
    step_bytes = sum(v["bytes"] for v in stages.values()) / args.steps
    step_ms = sum(v["ms"] for v in stages.values()) / args.steps
    cores, model = cpu_info()
    cpu = None
    if not args.no_cpu_baseline:
        per, el = oracle_step_time(gs, 1, args.flavor)
        cpu = {"value": 1.0 / per, "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle Lanczos step ({args.flavor}) restricted to k point 0 of "
                         f"{gs.nk}, {el:.1f} s, scaled x{gs.nk} (cost linear in k)",
               "cpu": model}
    line = {
        "metric": METRIC, "value": world * args.steps / wall_mixed if world > 1 else sps_mixed,
        "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * wall_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "flavor": args.flavor, "precision": "mixed",
                   "chains_per_gpu": 1, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (per-step working set > 5 GB)"},
        "fp64": {"value": sps_fp64, "unit": "steps/s", "steps": fp64_steps,
                 "ms_per_step": 1000 * wall_fp64 / fp64_steps},
        "chi_rel_err": chi_err, "chi_steps": m, "chi_tolerance": 1e-4,
        "roofline": {"bound": "hbm", "stage": top, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "peak_source": peak_src},
        "step_roofline": {"alg_bytes_per_step": step_bytes, "ms_per_step_profiled": step_ms,
                          "achieved_gbs": step_bytes / (step_ms / 1000) / 1e9,
                          "frac_hbm": step_bytes / (step_ms / 1000) / 1e9 / hbm},
        "stages_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in stages.items()},
        "stages_fp64_ms_per_step": {k: round(v["ms"] / fp64_steps, 4) for k, v in prof64.items()
                                    if v["launches"]},
        "clocks": clocks, "gpu_launches": launches,
        "e2e": {"value": args.steps / e2e_wall, "unit": "steps/s",
                "h2d_bytes_per_step": bundle_bytes / args.steps,
                "d2h_bytes_per_step": coef_bytes / args.steps,
                "what": "load_ground_state(host bundle) + chain of K mixed steps + coefficients "
                        "to host, through the C ABI"},
        "cpu_baseline": cpu,
        "status": int(res_e2e["status"][0]),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_tdlz(args)


if __name__ == "__main__":
    main()
