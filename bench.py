#!/usr/bin/env python
"""Benchmark: Lanczos steps/s of the Liouville-Lanczos hot path on one GB300.

Workload (default): the C2 CrI3-shaped synthetic crystal -- hexagonal a = 13 bohr,
c = 30 bohr (vacuum slab), FFT 36x36x96, ~5000 plane waves per spinor component,
4x4 k grid (16 k), 40 occupied spinor bands, 8 atoms x 8 KB projectors with
spin-orbit, q = (1/8, 0, 0) 2pi/a.  A step is one Lanczos iteration of one chain
and its FP64 scalar update: two Liouvillian applications (L q and L^H p) for the
non-Hermitian flavour used by default, one for the pseudo-Hermitian flavours.

Reported (one JSON line on rank 0):
  value          mixed-precision steps/s (FP32 vectors and arithmetic, FP64 scalars)
  fp64           the FP64 path's steps/s
  flavors        steps/s of the mixed path for each Lanczos flavour (NH: two Liouvillian
                 applications per step, PH: one)
  chi            mixed vs FP64 chi(omega) at eta = 10 meV on 0-100 meV, per column
  roofline       the step against its algorithmic work (bytes and flops of one step from
                 the per-application counts of the method) and the FP32 / HBM peaks, with
                 the dominant kernel's own figures beside it
  cpu_baseline   the FP64 CPU oracle: one full step of the same workload (C2), or a
                 one-k-point sample scaled by the k count where a full step takes too long
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
            "Nocc=40, 8 atoms x 8 KB projectors with SOC, q=(1/8,0,0) 2pi/a")


def workload(name):
    """The workload label of the JSON line: the C2 description, or the config's own shape."""
    if name == "C2":
        return WORKLOAD
    from synth.configs import CONFIGS
    c = CONFIGS[name]
    return (f"{name}: {c.kind} cell, FFT {'x'.join(map(str, c.fft))}, ecut {c.ecut} Ha, "
            f"{c.kgrid[0]}x{c.kgrid[1]}x{c.kgrid[2]} k, Nocc={c.nocc}, q={tuple(c.q_2pi_a)} 2pi/a")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tdlz", choices=["tdlz", "reference"])
    ap.add_argument("--config", default="C2")
    # NH by default: on the synthetic C2 model D + K is indefinite (the positive-definite
    # metric does not exist) and the J-metric start vector has a J-norm ~1e-3 of its norm
    ap.add_argument("--flavor", default=None, choices=["ph", "phm", "nh"],
                    help="default: nh on C2 (its D + K is indefinite), ph on C3")
    ap.add_argument("--chi-steps", type=int, default=500,
                    help="length of the mixed and FP64 chains of the chi error (C4: 500)")
    ap.add_argument("--states", default="auto", choices=["auto", "random"],
                    help="occupied states: auto = diagonalised on C0-C2, random orthonormal "
                         "on larger cells (the cost of a step does not depend on them)")
    ap.add_argument("--chains", type=int, default=3, choices=[1, 2, 3],
                    help="chi columns per GPU (x, y, z), advanced together")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-only", action="store_true",
                    help="profiling runs: time the mixed chains only (no FP64 chains, no chi error)")
    ap.add_argument("--bundle", default=None, help="cache file for the generated ground state")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="run N Liouvillian applications on a shape-only bundle (for profilers)")
    ap.add_argument("--precision", default="both", choices=["mixed", "fp64", "both"])
    ap.add_argument("--batched", type=int, default=0,
                    help="also time the batched form: this many q-points (|q| = m/16 2pi/a) x "
                         "3 NH chains in one chain set (not part of the default run)")
    ap.add_argument("--kpoints", type=int, default=0,
                    help="profiling runs only: keep the first N k points (smaller device footprint)")
    a = ap.parse_args()
    if a.flavor is None:
        a.flavor = "ph" if a.config in ("C3", "C5") else "nh"
    return a


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


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """Largest value over the ranks of the default process group (the value itself
    without one).  The bench times every rank and reports the slowest."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, chains: int, steps: int, max_wall: float) -> float:
    """Chain-steps per second of the whole job: every rank advances its own chains
    (replicas, weak scaling), the job lasts as long as its slowest rank."""
    return world * chains * steps / max_wall


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def random_states(cfg, states):
    """Shape-only bundles (random orthonormal occupied states) on the large cells, where
    the eigensolver would take tens of minutes and a step costs the same either way."""
    return states == "random" or (states == "auto" and cfg in ("C3", "C5"))


def make_workload(cfg, tol, bundle=None, states="auto"):
    from synth import GroundState, make_ground_state
    t = time.time()
    if bundle and os.path.exists(bundle):
        gs = GroundState.load(bundle)
        gs.meta = {"gap_min": float("nan"), "resid_max": float("nan")}
        log(f"[bench] ground state {cfg} loaded from {bundle}")
        return gs
    if random_states(cfg, states):
        gs = make_ground_state(cfg, solver="random")
        log(f"[bench] shape-only ground state {cfg}: npwx={gs.npwx} nk={gs.nk} "
            f"nocc={gs.nocc} ({time.time() - t:.1f} s)")
        return gs
    gs = make_ground_state(cfg, tol=tol, log=log)
    if bundle:
        gs.save(bundle)
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


def oracle_step_time(gs, nsteps=1, flavor="phm", nk_sample=None):
    """Seconds per Lanczos step of the FP64 oracle: the whole bundle (nk_sample None), or
    its first nk_sample k points with the time scaled by nk / nk_sample (the cost is
    linear in k).  Returns (seconds per full step, measured seconds, k points run)."""
    from oracle.liouvillian import Liouvillian
    from oracle.lanczos import lanczos_nh, lanczos_ph, lanczos_phm
    nks = gs.nk if nk_sample is None else min(nk_sample, gs.nk)
    sub = gs if nks == gs.nk else sample_bundle(gs, nks)
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
    return per * gs.nk / nks, el, nks


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
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, rank 0
    only.  Each step is a bounded sample of the workload (one Lanczos step restricted to
    k point 0); value is that time scaled to steps/s of the whole workload (cost linear
    in k), ms_per_step the sample's measured time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    gs = make_workload(args.config, args.tol, args.bundle, args.states)
    cores, model = cpu_info()
    sample_s, full_s = [], []
    for i in range(args.warmup + args.steps):
        per_full, el, _ = oracle_step_time(gs, 1, args.flavor, nk_sample=1)
        if i >= args.warmup:
            sample_s.append(el)
            full_s.append(per_full)
    value = args.steps / sum(full_s)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * sum(sample_s) / args.steps,
        "ms_per_step_is": "measured time of one sampled step (k point 0 only); value scales "
                          f"it by the {gs.nk} k points of the workload",
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.config), "flavor": args.flavor},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: one oracle Lanczos step restricted to k point 0 "
                                   f"of {gs.nk}, time x {gs.nk} (cost is linear in k)",
                         "cpu": model},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes per launch of a stage's kernel, from one ncu capture of the same build
# (dram__bytes_read.sum + dram__bytes_write.sum): the product kernel of the C2 step
# (6 stacked vectors) captured at 4 of the 16 k points, scaled by 4 (its traffic is
# linear in the number of k points).  Summary: profiles/kernels_C2_k4_full.md.
NCU_TRAFFIC = {("C2", "product"): 4 * 8.837e9}


# GB300's FP64 vector rate (nominal, dense): the binding roof of the FP64 path, whose
# FFT, pointwise and GEMM stages all run on the FP64 pipe.
FP64_PEAK_TFLOPS = 1.25


def fp64_roofline(prof64):
    """Nominal flops of the profiled FP64 steps (per stage: 5 N log2 N per line transform,
    8 per complex multiply-add of the contractions, the pointwise products) over their
    CUDA-event time, against the FP64 rate."""
    ms = sum(v["ms"] for v in prof64.values())
    fl = sum(v["flops"] for v in prof64.values())
    if ms <= 0:
        return None
    achieved = fl / (ms / 1000) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64 rate"}


def ncu_traffic(args, stage):
    if args.kpoints or args.flavor != "nh" or args.chains != 3:
        return None
    return NCU_TRAFFIC.get((args.config, stage))


def algorithmic_work(gs, flavor, chains, elem):
    """Algorithmic bytes and flops of one Lanczos step of `chains` chains of one q-point,
    from the per-application counts of the method: V = 2 sides x Nk x Nb x 2 spinor
    components x Np complex numbers per response vector (Np the mean k+q sphere), elem
    bytes per complex number.
      bytes  NH: 6V per chain (q, p in; L q, L^H p out; q, p of the previous step) + the
             occupied orbitals U_k, U_k+q (2V) shared by the chains of one q + the
             projector table Nk Nbeta Np; PH: 3V per chain instead of 6V.
      flops  per application: FFTs 2 Nk Nb 4 x 5 Nr log2 Nr x 0.56 (pruned to the sphere),
             contractions 2 Nk (16 Nb^2 2 Np + 16 Nbeta Nb 2 Np), pointwise 110 per grid
             point and band-side; NH applies L twice per chain and step, PH once."""
    import math
    import numpy as np
    s_, ns = 2, 2
    nk, nb, nproj = gs.nk, gs.nocc, gs.nproj
    npw = float(np.mean(gs.npw_kq))
    nr = int(np.prod(gs.fft))
    v = s_ * nk * nb * ns * npw
    nvec_terms, apps = (6, 2) if flavor == "nh" else (3, 1)
    bytes_ = chains * nvec_terms * v * elem + 2 * v * elem + nk * nproj * npw * elem
    fft = s_ * nk * nb * 4 * (5 * nr * math.log2(nr) * 0.56)
    gemm = s_ * nk * (16 * nb * nb * ns * npw + 16 * nproj * nb * ns * npw)
    point = 110 * s_ * nk * nb * nr
    return bytes_, chains * apps * (fft + gemm + point)


def fp32_peak_tflops(device=0):
    """FP32 vector peak derived from unit counts: SMs x 128 FP32 lanes x 2 flop (FMA) x
    the maximum SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"


def chain_steps_per_s(ctx, q, mus, flavor, precision, warmup, steps, stream, profile=False):
    """Chain-steps per second summed over the chains mus (one group on one q-slot).
    The library runs on `stream` (handed to it at context creation); the timed
    region is bracketed by CUDA events recorded on that stream, with the stream
    synchronised on both sides."""
    import torch
    ch = ctx.chain_create([q] * len(mus), mus, warmup + steps + 1, flavor, precision)
    try:
        ch.advance(warmup)
        ctx.synchronize()
        if profile:
            ctx.profile(True)
        l0 = ctx.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ctx.synchronize()
        ev0.record(stream)
        ch.advance(steps)
        ev1.record(stream)
        ctx.synchronize()
        wall = ev0.elapsed_time(ev1) / 1000.0
        launches = ctx.launch_count() - l0
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(False)
        res = ch.read()
        return len(mus) * steps / wall, wall, launches, prof, res
    finally:
        ch.close()


def cufft_baseline(rows, fft, device, reps=3):
    """cuFFT (through torch.fft) on the batch of one Liouvillian pass: `rows` full-box 3D
    transforms of the FFT grid in FP32 complex, inverse and forward, out of place, timed
    with CUDA events after one warm-up.  The library's passes transform only the sticks and
    planes of the spheres and include the sphere scatter and gather; cuFFT transforms the
    whole box.  Returns milliseconds per batch, or the error."""
    import torch
    try:
        dims = (1, 2, 3)
        x = torch.randn(rows, *fft, dtype=torch.complex64, device=device)
        out = {}
        for name, f in (("inverse_ms", torch.fft.ifftn), ("forward_ms", torch.fft.fftn)):
            y = f(x, dim=dims)
            torch.cuda.synchronize(device)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(reps):
                y = f(x, dim=dims)
            ev1.record()
            torch.cuda.synchronize(device)
            out[name] = ev0.elapsed_time(ev1) / reps
            del y
        del x
        torch.cuda.empty_cache()
        return {"rows": rows, "grid": list(fft), **out,
                "what": "torch.fft (cuFFT) full-box batched 3D FFT, complex64, out of place"}
    except Exception as e:  # reported, never fatal to the bench line
        return {"rows": rows, "grid": list(fft), "error": f"{type(e).__name__}: {e}"[:200]}


def cufft_pruned_baseline(rows, fft, nsm, npm, device, reps=3):
    """cuFFT (torch.fft) driven the same pruned way as the library's passes, on the batch
    of one pass: batched 1D transforms along the sphere's sticks (rows x nsm lines of
    n3), along y on its planes (rows x npm x n3 lines of n2), along x over the box
    (rows x n2 x n3 lines of n1), complex64, out of place.  The gathers and scatters
    between the stages (done by the library's passes) are not included.  Returns
    milliseconds per batch for each direction, or the error."""
    import torch
    try:
        n1, n2, n3 = fft
        out = {}
        for name, f in (("inverse_ms", torch.fft.ifft), ("forward_ms", torch.fft.fft)):
            total = 0.0
            for shape, dim in (((rows, nsm, n3), 2), ((rows, npm, n2, n3), 2),
                               ((rows, n1, n2 * n3), 1)):
                x = torch.randn(*shape, dtype=torch.complex64, device=device)
                y = f(x, dim=dim)
                torch.cuda.synchronize(device)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record()
                for _ in range(reps):
                    y = f(x, dim=dim)
                ev1.record()
                torch.cuda.synchronize(device)
                total += ev0.elapsed_time(ev1) / reps
                del x, y
                torch.cuda.empty_cache()
            out[name] = total
        return {"rows": rows, "grid": list(fft), "sticks": nsm, "planes": npm, **out,
                "what": "torch.fft (cuFFT) batched 1D passes on the sticks, the planes and the "
                        "box, complex64, out of place, without the gathers between passes"}
    except Exception as e:  # reported, never fatal to the bench line
        return {"rows": rows, "grid": list(fft), "error": f"{type(e).__name__}: {e}"[:200]}


def run_batched(args, local, stream):
    """The batched form: q-points m = 1..NQ along x (|q| = m/16 2pi/a) of the same crystal,
    three NH chains (mu = x, y, z) on each, all in one chain set -- one group per q-slot,
    each with its own k+q plane-wave counts, advanced together and replayed from one
    captured graph, mixed precision.  The occupied states are random orthonormal spinors
    on the crystal's spheres (the cost of a Liouvillian pass does not depend on them)."""
    import torch
    from paper_2203_01120_gb300 import TDLZ_MIXED, Context
    from synth import make_ground_state
    ctx = Context(local, stream=stream.cuda_stream)
    try:
        qs, npw = [], []
        for m in range(1, args.batched + 1):
            gs = make_ground_state(args.config, q_2pi_a=(m / 16.0, 0.0, 0.0), solver="random")
            npw.append([int(gs.npw_kq.min()), int(gs.npw_kq.max())])
            qs.append(ctx.load_ground_state(gs))
            del gs
        slots = [q for q in qs for _ in range(3)]
        mus = [mu for _ in qs for mu in range(3)]
        ch = ctx.chain_create(slots, mus, args.warmup + args.steps + 1, "nh", TDLZ_MIXED)
        try:
            ch.advance(args.warmup)
            ctx.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            ch.advance(args.steps)
            ev1.record(stream)
            ctx.synchronize()
            wall = ev0.elapsed_time(ev1) / 1000.0
            res = ch.read()
        finally:
            ch.close()
        log(f"[bench] batched: {len(mus)} chains on {len(qs)} q-slots, "
            f"{1000 * wall / args.steps:.2f} ms per step")
        return {"q_points": len(qs), "chains": len(mus), "value": len(mus) * args.steps / wall,
                "unit": "steps/s", "steps": args.steps, "ms_per_step": 1000 * wall / args.steps,
                "npw_kq_range_per_q": npw, "status": [int(v) for v in res["status"]],
                "what": "chain-steps/s of all chains of the set; occupied states random "
                        "orthonormal on the crystal's spheres"}
    finally:
        ctx.close()


def sphere_sticks_planes(gs):
    """Largest number of (m1, m2) sticks and of m1 planes over the k+q spheres."""
    import numpy as np
    nsm = npm = 0
    for k in range(gs.nk):
        m = np.asarray(gs.miller_kq[k][:int(gs.npw_kq[k])])
        nsm = max(nsm, len({(int(a), int(b)) for a, b in m[:, :2]}))
        npm = max(npm, len(set(int(a) for a in m[:, 0])))
    return nsm, npm


def chi_column_errors(c32, c64, mus=None):
    """Per chi column mu: max over lambda of ||chi32 - chi64||_2 / ||chi64[mu][mu]||_2
    (row i of the arrays is the chain of column mus[i], default i)."""
    import numpy as np
    mus = list(range(len(c64))) if mus is None else mus
    return [float(np.linalg.norm(c32[i] - c64[i], axis=1).max() / np.linalg.norm(c64[i][mu]))
            for i, mu in enumerate(mus)]


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
    gs = make_workload(args.config, args.tol, args.bundle, args.states)
    if args.kpoints:  # profiling captures only: the first k points of the workload
        gs = sample_bundle(gs, args.kpoints)
    chi_steps = args.chi_steps if args.config in ("C1", "C2") else min(args.chi_steps, 10)
    # replicas: every rank runs the chi columns mus (the paper's ipol = 4: x, y, z)
    mus = list(range(args.chains))
    stream = torch.cuda.Stream(device=local)
    ctx = Context(local, stream=stream.cuda_stream)
    # the CrI3-shaped cells: mixed work on a q-slot holding FP32 data only, FP64 work on a
    # second context afterwards (both sets of real-space orbitals and workspaces together
    # would fill most of the device)
    split = args.config not in ("C1", "C2")
    # ------------------------------------------------------------ e2e (host in/out)
    t0 = time.perf_counter()
    if split:
        os.environ["TDLZ_MIXED_ONLY"] = "1"
    try:
        q = ctx.load_ground_state(gs)
    finally:
        os.environ.pop("TDLZ_MIXED_ONLY", None)
    t1 = time.perf_counter()
    ch = ctx.chain_create([q] * len(mus), mus, args.steps, args.flavor, TDLZ_MIXED)
    ctx.synchronize()
    t2 = time.perf_counter()
    ch.advance(args.steps)
    res_e2e = ch.read()
    e2e_wall = time.perf_counter() - t0
    e2e_parts = {"load_s": t1 - t0, "chain_start_s": t2 - t1,
                 "steps_and_read_s": e2e_wall - (t2 - t0)}
    ch.close()
    bundle_bytes = sum(int(np.asarray(getattr(gs, k)).nbytes) for k in (
        "kpts", "wk", "npw_k", "npw_kq", "miller_k", "miller_kq", "evals", "coeff_k", "coeff_kq",
        "vloc", "bfield", "n0", "m0", "beta_kq", "dnl"))
    coef_bytes = len(mus) * args.steps * (16 * 2 + 8 + 16 * 3)
    # ------------------------------------------------------------ device-resident timing
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    sps_mixed, wall_mixed, launches, _, _ = chain_steps_per_s(
        ctx, q, mus, args.flavor, TDLZ_MIXED, args.warmup, args.steps, stream)
    clocks = clk.finish()
    wall_mixed = max_over_ranks(wall_mixed, "cuda")
    # profiled pass (per-stage CUDA events on the library stream) for the roofline
    _, _, _, prof, _ = chain_steps_per_s(ctx, q, mus, args.flavor, TDLZ_MIXED, 1, args.steps,
                                         stream, profile=True)
    flavors = {args.flavor: {"value": len(mus) * args.steps / wall_mixed, "unit": "steps/s",
                             "ms_per_step": 1000 * wall_mixed / args.steps,
                             "l_applications_per_step": len(mus) * (2 if args.flavor == "nh" else 1)}}
    if not args.mixed_only and args.config in ("C1", "C2"):
        for fl in ("nh", "ph"):
            if fl in flavors:
                continue
            sps, wall, _, _, res = chain_steps_per_s(ctx, q, mus, fl, TDLZ_MIXED, args.warmup,
                                                     args.steps, stream)
            flavors[fl] = {"value": sps, "unit": "steps/s", "ms_per_step": 1000 * wall / args.steps,
                           "l_applications_per_step": len(mus) * (2 if fl == "nh" else 1),
                           "status": [int(v) for v in res["status"]]}
    fp64_steps = max(3, args.steps // 4)
    m = chi_steps
    chi = None
    autotune = {k: v[0] for k, v in ctx.autotune_report().items()}
    if args.mixed_only:  # profiling runs: the mixed chains above are the whole workload
        sps_fp64, wall_fp64, prof64 = None, None, {}
    else:
        # ------------------------------------------------ chi error mixed vs FP64
        # C2: the timed chains; larger cells (shape-only occupied states, where the
        # J-metric start vector has a J-norm ~1e-3 of its norm and the PH recursion is
        # ill-conditioned from its first steps) one NH chain over a short prefix
        chi_fl, chi_mus = (args.flavor, mus) if args.config in ("C1", "C2") else ("nh", [0])
        r32 = ctx.lanczos_run([q] * len(chi_mus), chi_mus, m, chi_fl, TDLZ_MIXED)
        if split:
            ctx.close()
            ctx = Context(local, stream=stream.cuda_stream)
            q = ctx.load_ground_state(gs)
        sps_fp64, wall_fp64, _, prof64, _ = chain_steps_per_s(
            ctx, q, mus, args.flavor, TDLZ_FP64, 1, fp64_steps, stream, profile=True)
        r64 = ctx.lanczos_run([q] * len(chi_mus), chi_mus, m, chi_fl, TDLZ_FP64)
        chi = {"steps": m, "flavor": chi_fl, "chains": chi_mus, "omega_mev": [0.0, 100.0, 0.1],
               "eta_mev": 10.0, "tolerance": 1e-4,
               "norm": "per column mu: max over lambda ||chi_mixed - chi_fp64|| / ||chi_fp64[mu][mu]||"}
        for mm in sorted({m, min(m, 100)}):
            c64 = ctx.spectrum(r64, 0.0, 100.0, 0.1, 10.0, units=1, itermax0=mm)
            c32 = ctx.spectrum(r32, 0.0, 100.0, 0.1, 10.0, units=1, itermax0=mm)
            chi[f"rel_err_{mm}"] = chi_column_errors(c32, c64, chi_mus)
        chi["status"] = [int(v) for v in r32["status"]] + [int(v) for v in r64["status"]]
        # conditioning probe: the same mixed chains through the other real-space path
        # (same operator and precision, different rounding order); where the two FP32
        # results differ by as much as FP32 differs from FP64, the chi of that chain
        # length is not determined to that precision by any FP32 computation
        if args.config in ("C2", "C4"):
            os.environ["TDLZ_PLANES"] = "1"
            try:
                q2 = ctx.load_ground_state(gs)
            finally:
                del os.environ["TDLZ_PLANES"]
            r32b = ctx.lanczos_run([q2] * len(mus), mus, m, args.flavor, TDLZ_MIXED)
            for mm in sorted({m, min(m, 100)}):
                ca = ctx.spectrum(r32, 0.0, 100.0, 0.1, 10.0, units=1, itermax0=mm)
                cb = ctx.spectrum(r32b, 0.0, 100.0, 0.1, 10.0, units=1, itermax0=mm)
                chi[f"fp32_rounding_spread_{mm}"] = chi_column_errors(cb, ca)
    ctx.close()
    # cuFFT on the same batch as one pass: full box, and driven the same pruned way
    cufft = None
    if not args.kpoints and not args.mixed_only and args.config in ("C1", "C2"):
        rows = len(mus) * (2 if args.flavor == "nh" else 1) * 4 * gs.nk * gs.nocc
        fft = tuple(int(n) for n in gs.fft)
        cufft = {"full_box": cufft_baseline(rows, fft, local)}
        nsm, npm = sphere_sticks_planes(gs)
        cufft["pruned"] = cufft_pruned_baseline(rows, fft, nsm, npm, local)
        st_ms = {k: v["ms"] / args.steps for k, v in prof.items()}
        cufft["tdlz_inverse_ms"] = st_ms.get("scatter", 0.0) + st_ms.get("fft_inv", 0.0)
        cufft["tdlz_forward_ms"] = st_ms.get("fft_fwd", 0.0) + st_ms.get("gather", 0.0)
    batched = run_batched(args, local, stream) if args.batched else None
    if rank != 0:
        return
    hbm, peak_src = measured_peaks()
    # dominant stage of the mixed step, against its own design traffic
    stages = {k: v for k, v in prof.items() if v["launches"] > 0 and v["ms"] > 0}
    top = max(stages, key=lambda k: stages[k]["ms"])
    st = stages[top]
    nl = st["launches"]
    per_launch_s = st["ms"] / 1000.0 / nl
    bytes_launch = st["bytes"] / nl
    design_bytes_step = sum(v["bytes"] for v in stages.values()) / args.steps
    # the step against the algorithmic work of the method
    alg_bytes, alg_flops = algorithmic_work(gs, args.flavor, len(mus), 8)
    step_s = wall_mixed / args.steps
    peak32, src32 = fp32_peak_tflops(local)
    achieved_tf = alg_flops / step_s / 1e12
    cores, model = cpu_info()
    cpu = None
    if not args.no_cpu_baseline:
        full = args.config in ("C1", "C2")  # one full step is ~40 s of oracle on C2
        per, el, nks = oracle_step_time(gs, 1, args.flavor, nk_sample=None if full else 1)
        cpu = {"value": 1.0 / per, "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": (f"one full FP64 oracle Lanczos step ({args.flavor}, one chain, all "
                          f"{gs.nk} k points), {el:.1f} s" if nks == gs.nk else
                          f"one FP64 oracle Lanczos step ({args.flavor}) restricted to k point 0 "
                          f"of {gs.nk}, {el:.1f} s, scaled x{gs.nk} (cost linear in k)"),
               "cpu": model}
    line = {
        "metric": METRIC,
        "value": whole_job_rate(world, len(mus), args.steps, wall_mixed),
        "l_applications_per_s": whole_job_rate(world, len(mus), args.steps, wall_mixed)
        * (2 if args.flavor == "nh" else 1),
        "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * wall_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload(args.config), "flavor": args.flavor, "precision": "mixed",
                   "chains_per_gpu": len(mus), "parallelism": f"replicas{world}",
                   "occupied_states": "random orthonormal (shape only)"
                   if random_states(args.config, args.states) else "diagonalised",
                   "ms_per_step_is": "one step of every chain of the GPU (advanced together)",
                   "l2": "inputs larger than L2 (per-step working set > 5 GB)"},
        "flavors": flavors,
        "fp64": None if sps_fp64 is None else {
            "value": sps_fp64, "unit": "steps/s", "steps": fp64_steps,
            "ms_per_step": 1000 * wall_fp64 / fp64_steps,
            "roofline": fp64_roofline(prof64)},
        "chi": chi,
        "roofline": {
            "bound": "alu", "achieved": achieved_tf, "peak": peak32, "unit": "TFLOP/s",
            "frac": achieved_tf / peak32, "peak_source": src32,
            "scope": "the whole mixed step against the algorithmic flops and bytes of the "
                     "method's Liouvillian applications (pruned FFTs, contractions, pointwise "
                     "products; response vectors, orbitals, projectors)",
            "flops_per_step": alg_flops, "alg_bytes_per_step": alg_bytes,
            "achieved_gbs": alg_bytes / step_s / 1e9, "hbm_peak_gbs": hbm,
            "frac_hbm": alg_bytes / step_s / 1e9 / hbm, "hbm_peak_source": peak_src,
            "design_bytes_per_step": design_bytes_step,
            "design_over_alg_bytes": design_bytes_step / alg_bytes,
            "traffic": None,
            "dominant_kernel": {
                "stage": top, "bound": "hbm",
                "achieved_gbs": bytes_launch / per_launch_s / 1e9,
                "frac": bytes_launch / per_launch_s / 1e9 / hbm,
                "design_bytes_per_launch": bytes_launch, "launches": nl,
                "traffic": ncu_traffic(args, top), "traffic_unit": "bytes per launch"}},
        "stages_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in stages.items()},
        "stages_fp64_ms_per_step": {k: round(v["ms"] / fp64_steps, 4) for k, v in prof64.items()
                                    if v["launches"]},
        "clocks": clocks, "gpu_launches": launches, "autotune": autotune,
        "e2e": {"value": len(mus) * args.steps / e2e_wall, "unit": "steps/s",
                "h2d_bytes_per_step": bundle_bytes / args.steps,
                "d2h_bytes_per_step": coef_bytes / args.steps,
                "what": "load_ground_state(host bundle) + chain of K mixed steps + coefficients "
                        "to host, through the C ABI", **e2e_parts},
        "cpu_baseline": cpu,
        "status": [int(v) for v in res_e2e["status"]],
    }
    if cufft:
        line["cufft_baseline"] = cufft
    if batched:
        line["batched"] = batched
    print(json.dumps(line), flush=True)


def run_c5(args):
    """The batched form (C5): six q-points m/16 (2pi/a), m = 1..6, along x of the
    CrI3-shaped cell on a 4x4 k grid, each with its own cutoff (10000-13000 plane waves per
    spinor component), three chains (mu = x, y, z) on each: 18 chains in one chain set,
    one group per q-slot, advanced together and replayed from one captured graph, mixed
    precision.  Occupied states random orthonormal (the cost of a step does not depend
    on them); q-slots loaded for mixed precision only (the FP64 orbitals released)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2203_01120_gb300 import TDLZ_MIXED, Context, build_ext
    from synth import make_ground_state
    from synth.configs import c5_ecut
    build_ext.build()
    nq = 6
    t = time.time()
    bundles = [make_ground_state("C5", q_2pi_a=(m / 16.0, 0.0, 0.0), ecut=c5_ecut(m, nq),
                                 solver="random") for m in range(1, nq + 1)]
    log(f"[bench] C5: {nq} shape-only bundles ({time.time() - t:.1f} s), npw_kq "
        f"{[int(b.npw_kq.mean()) for b in bundles]}")
    stream = torch.cuda.Stream(device=local)
    ctx = Context(local, stream=stream.cuda_stream)
    os.environ["TDLZ_MIXED_ONLY"] = "1"
    try:
        t0 = time.perf_counter()
        qs = [ctx.load_ground_state(b) for b in bundles]
        t1 = time.perf_counter()
    finally:
        del os.environ["TDLZ_MIXED_ONLY"]
    slots = [q for q in qs for _ in range(3)]
    mus = [mu for _ in qs for mu in range(3)]
    nch = len(mus)
    # e2e: the loads above + chain start + K steps + coefficients to the host
    ch = ctx.chain_create(slots, mus, args.steps, args.flavor, TDLZ_MIXED)
    ctx.synchronize()
    t2 = time.perf_counter()
    ch.advance(args.steps)
    res_e2e = ch.read()
    e2e_wall = time.perf_counter() - t0
    ch.close()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    ch = ctx.chain_create(slots, mus, args.warmup + args.steps + 1, args.flavor, TDLZ_MIXED)
    ch.advance(args.warmup)
    ctx.synchronize()
    l0 = ctx.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ch.advance(args.steps)
    ev1.record(stream)
    ctx.synchronize()
    wall = ev0.elapsed_time(ev1) / 1000.0
    launches = ctx.launch_count() - l0
    clocks = clk.finish()
    wall = max_over_ranks(wall, "cuda")
    res = ch.read()
    ch.close()
    ctx.profile(True)
    chp = ctx.chain_create(slots, mus, args.steps + 2, args.flavor, TDLZ_MIXED)
    chp.advance(1)
    ctx.profile(False)
    ctx.profile(True)
    chp.advance(args.steps)
    ctx.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    chp.close()
    ctx.close()
    if rank != 0:
        return
    step_s = wall / args.steps
    alg_b = alg_f = 0.0
    for b in bundles:
        bb, ff = algorithmic_work(b, args.flavor, 3, 8)
        alg_b, alg_f = alg_b + bb, alg_f + ff
    peak32, src32 = fp32_peak_tflops(local)
    hbm, peak_src = measured_peaks()
    stages = {k: v for k, v in prof.items() if v["launches"] > 0 and v["ms"] > 0}
    cores, model = cpu_info()
    cpu = None
    if not args.no_cpu_baseline:
        per, el, nks = oracle_step_time(bundles[0], 1, args.flavor, nk_sample=1)
        cpu = {"value": 1.0 / per, "unit": "chain-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle Lanczos step ({args.flavor}) of the q = 1/16 chain "
                         f"restricted to k point 0 of 16, {el:.1f} s, scaled x16 (cost linear "
                         "in k; the other q-points have 0.9-1.2 times its plane waves)",
               "cpu": model}
    bundle_bytes = sum(sum(int(np.asarray(getattr(b, k)).nbytes) for k in (
        "kpts", "wk", "npw_k", "npw_kq", "miller_k", "miller_kq", "evals", "coeff_k", "coeff_kq",
        "vloc", "bfield", "n0", "m0", "beta_kq", "dnl")) for b in bundles)
    line = {
        "metric": METRIC, "value": whole_job_rate(world, nch, args.steps, wall),
        "l_applications_per_s": whole_job_rate(world, nch, args.steps, wall)
        * (2 if args.flavor == "nh" else 1),
        "unit": "chain-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "C5: batched form, hexagonal a=13 c=38 bohr, FFT 45x45x144, 4x4 k, "
                               "Nocc=70, 8 atoms x 8 KB projectors with SOC, q = m/16 2pi/a "
                               "(m = 1..6) with 10000-13000 PW per component, 3 chains per q",
                   "flavor": args.flavor, "precision": "mixed", "chains_per_gpu": nch,
                   "q_points": nq, "parallelism": f"replicas{world}",
                   "npw_kq_mean_per_q": [int(b.npw_kq.mean()) for b in bundles],
                   "occupied_states": "random orthonormal (shape only)",
                   "ms_per_step_is": "one step of all 18 chains (6 q-slot groups, one graph)",
                   "l2": "inputs larger than L2"},
        "roofline": {
            "bound": "alu", "achieved": alg_f / step_s / 1e12, "peak": peak32, "unit": "TFLOP/s",
            "frac": alg_f / step_s / 1e12 / peak32, "peak_source": src32,
            "scope": "the whole batched step against the algorithmic flops and bytes of its "
                     "Liouvillian applications",
            "flops_per_step": alg_f, "alg_bytes_per_step": alg_b,
            "achieved_gbs": alg_b / step_s / 1e9, "hbm_peak_gbs": hbm,
            "frac_hbm": alg_b / step_s / 1e9 / hbm, "hbm_peak_source": peak_src, "traffic": None},
        "stages_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in stages.items()},
        "clocks": clocks, "gpu_launches": launches,
        "e2e": {"value": nch * args.steps / e2e_wall, "unit": "chain-steps/s",
                "h2d_bytes_per_step": bundle_bytes / args.steps,
                "d2h_bytes_per_step": nch * args.steps * (16 * 2 + 8 + 16 * 3) / args.steps,
                "what": "load_ground_state of the 6 host bundles + chain set of K mixed steps + "
                        "coefficients to host, through the C ABI",
                "load_s": t1 - t0, "chain_start_s": t2 - t1},
        "cpu_baseline": cpu,
        "status": [int(v) for v in res["status"]],
    }
    print(json.dumps(line), flush=True)


def run_profile_apply(args):
    """Small, self-contained case for profilers: a shape-only bundle of the config
    (random orthonormal occupied states, no diagonalisation) and a few Liouvillian
    applications per precision.  Used by the ncu summaries under profiles/."""
    import numpy as np
    import torch
    from paper_2203_01120_gb300 import TDLZ_FP64, TDLZ_MIXED, Context, build_ext
    from synth import make_ground_state, random_br_vector
    build_ext.build()
    gs = make_ground_state(args.config, solver="random")
    if args.kpoints:
        gs = sample_bundle(gs, args.kpoints)
    ctx = Context(0)
    q = ctx.load_ground_state(gs)
    x = random_br_vector(gs, seed=7)
    precs = {"mixed": [TDLZ_MIXED], "fp64": [TDLZ_FP64], "both": [TDLZ_MIXED, TDLZ_FP64]}
    for prec in precs[args.precision]:
        dt = torch.complex64 if prec == TDLZ_MIXED else torch.complex128
        xt = torch.as_tensor(x, dtype=dt, device="cuda")
        yt = torch.zeros_like(xt)
        ctx.synchronize()
        t = time.perf_counter()
        for _ in range(args.profile_apply):
            ctx.apply_liouvillian(q, xt, yt, False, prec)
        ctx.synchronize()
        dt_ms = 1000 * (time.perf_counter() - t) / args.profile_apply
        log(f"[profile-apply] {args.config} {'mixed' if prec else 'fp64'}: {dt_ms:.3f} ms per L "
            f"(|y| = {float(torch.linalg.vector_norm(yt)):.4e})")
    ctx.close()
    del np


def main():
    args = parse()
    if args.profile_apply:
        run_profile_apply(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "C5":
        run_c5(args)
    else:
        run_tdlz(args)


if __name__ == "__main__":
    main()
