"""Benchmark of the GB300 CGKS-5th / GKS-2nd hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full time step of the hot path (dt on the device,
reconstruction, gas-kinetic flux, cell update; two stages for CGKS-5th).
Default workload: CGKS-5th, FP64, nonlinear, on decaying isotropic
turbulence at 512^3 (Mt 0.5, k0 8, seed 103, mu 1e-3; gamma 1.4, Pr 0.72,
CFL 0.3) with synthetic cell-averaged initial data, inputs resident in HBM;
the mixed-precision and mixed + learned-indicator paths of the same
workload are reported under "variants" with their kinetic-energy error
against FP64 after the same steps. --workload tgv runs the Taylor-Green
vortex instead (Sec. 4.1; Ma 0.1, Re 1600; 128^3 by default).
Metric: cell-stage updates/s (cells x stages x steps / device time).

Multi-GPU: replicas only (the path does not shard on one box): every rank
advances its own grid, no data-path collective; value = sum over ranks.
--impl reference times the FP64 CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
# Work per unit of the hot kernels, from ncu's SASS op counters
# (sm__sass_thread_inst_executed_op_{dfma,dadd,dmul,ffma,fadd,fmul}_pred_on,
# an FMA counted as 2 FLOP) and dram__bytes_{read,write} of one launch on
# the 64^3 stand-in of the 512^3 turbulence (the same cells per wavelength
# and dt/tau, so the flux takes the same branches; profiles/opcount_*.md):
# FP64 and FP32 FLOP, algorithmic bytes
# (state and face-state buffers read and written once) and measured DRAM
# bytes. A unit is one reconstructed cell for a reconstruction, one face
# Gauss point for a flux kernel (12 per cell for CGKS-5th: 3 faces x 4
# points; 3 per cell for GKS-2nd).
_DRAM_NOTE = ("ncu dram__bytes_read+write per unit of one launch on a 64^3 grid, times "
              "this launch's units (the traffic grows with the units: one pass over state "
              "and face buffers that exceed L2)")
KERNEL_OPS = {
    "recon5": {"fp64": 15708.5, "fp32": 130.0, "bytes": 160 + 3840, "dram": 3832.4,
               "dram_note": _DRAM_NOTE},
    "flux_cgks5": {"fp64": 4006.5, "fp32": 16.0, "bytes": (3840 + 720) / 12, "dram": 377.4,
                   "dram_note": _DRAM_NOTE},
    "recon5_mixed": {"fp64": 0.0, "fp32": 14676.2, "bytes": 40 + 60 + 1920, "dram": 1787.8,
                     "dram_note": _DRAM_NOTE},
    "flux_cgks5_mixed": {"fp64": 21.5, "fp32": 6380.4, "bytes": (1920 + 40 + 720) / 12,
                         "dram": 225.2, "dram_note": _DRAM_NOTE},
}
KERNEL_OPS["recon5_learned"] = KERNEL_OPS["recon5_mixed"]
KERNEL_OPS["flux_cgks5_learned"] = KERNEL_OPS["flux_cgks5_mixed"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="cells per axis (default 512; --workload tgv 128; --c2 64, --c3 256, "
                         "--c5 512)")
    ap.add_argument("--scheme", default="cgks5", choices=["cgks5", "gks2"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--indicator", action="store_true",
                    help="mixed precision with the learned smoothness indicator (CGKS-5th)")
    ap.add_argument("--workload", default="hit", choices=["tgv", "hit"],
                    help="hit: decaying isotropic turbulence (Mt 0.5, k0 8, seed 103, mu 1e-3); "
                         "tgv: Taylor-Green vortex (Ma 0.1, Re 1600)")
    ap.add_argument("--proxy-of", type=int, default=None,
                    help="hit: a small grid standing in for this larger one (k0 and mu scaled "
                         "so that cells per wavelength and dt/tau match; for op counts)")
    ap.add_argument("--slab-planes", type=int, default=0,
                    help="z-planes per reconstruction/flux slab (0: automatic)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host round trip (very large grids)")
    ap.add_argument("--c5", action="store_true",
                    help="FP64 vs mixed vs mixed + learned indicator on one isotropic-turbulence "
                         "state (default 512^3, z-slabs), with the KE error against FP64")
    ap.add_argument("--c4", action="store_true",
                    help="batched ensemble of 64 uneven 2D instances (double shear layers, "
                         "four-quadrant Riemann problems), autotuned tiles, graph-replayed steps")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="--c5: FP64 steps (an FP64 step at 512^3 takes ~23 s)")
    ap.add_argument("--c2", action="store_true",
                    help="Taylor-Green vortex to t_end with E_k, eps_S, eps_D histories, FP64 "
                         "and mixed on one grid (default 64^3)")
    ap.add_argument("--t-end", type=float, default=10.0, help="--c2: final time (U0 = L = 1)")
    ap.add_argument("--every", type=float, default=0.1, help="--c2: sampling interval")
    ap.add_argument("--precisions", default="fp64,mixed",
                    help="--c2: paths to run (fp64, mixed, fp64p: FP64 from the initial "
                         "state perturbed by 1e-14 relative, the FP64 path's own sensitivity)")
    ap.add_argument("--ma2", action="store_true",
                    help="--c2: the supersonic Taylor-Green vortex of Sec. 4.2 (Ma 2, Re 1600, "
                         "Pr 0.7, Sutherland viscosity) instead of the Ma 0.1 one")
    ap.add_argument("--linear", action="store_true",
                    help="--c2: the linear scheme (chi = 1 / no limiter), as the paper runs the "
                         "subsonic Taylor-Green vortex")
    ap.add_argument("--c3", action="store_true",
                    help="isotropic turbulence Mt 0.5 and 1.0 (Re_lambda 72), FP64 vs mixed vs "
                         "mixed + learned indicator, per-step E_k, eps_S, eps_D (default 256^3)")
    ap.add_argument("--general", action="store_true",
                    help="general-grid kernels: the Taylor-Green octant [0, pi]^3 bounded by six "
                         "symmetry planes on a stretched mesh (cells 0.7-1.3 times the mean), "
                         "FP64 and mixed, against the periodic uniform kernels on the same cell "
                         "count (default 256^3)")
    ap.add_argument("--lines", action="store_true",
                    help="CGKS-5th FP64 with the line-averaged derivatives as the cell's own data "
                         "(gks_step_lines) against the averaged-gradient form on the same "
                         "Taylor-Green grid (default 128^3)")
    ap.add_argument("--history", default=None,
                    help="--c2/--c3: write the sampled histories to this JSON file")
    args = ap.parse_args()
    if args.n is None:
        args.n = (64 if args.c2 else 128 if args.lines else 256 if (args.c3 or args.general)
                  else 512 if args.c5
                  else 128 if args.workload == "tgv" else 512)
    return args


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
def sample_workload(args, n):
    """The benchmark's workload at a size the CPU oracle finishes in seconds
    (the same generator and parameters; only the grid is smaller)."""
    from paper_2508_19911_gb300 import workloads as wl
    if getattr(args, "workload", "hit") == "tgv":
        Q, G, grid = wl.taylor_green(n)
        return Q, G, grid, 1.0 / 1600, "taylor_green"
    Q, G, grid, _ = wl.isotropic_turbulence(n, Mt=0.5, k0=8.0, seed=103)
    return Q, G, grid, 1e-3, "isotropic_turbulence"


def cpu_baseline(args):
    """The FP64 oracle as it stands, OpenMP over cells on all host cores,
    on a bounded sample (about 15 s on 16 cores): the benchmark's workload
    on a 48^3 grid (CGKS-5th; 96^3 for GKS-2nd), 2 time steps."""
    import oracle
    cg = args.scheme == "cgks5"
    n = 48 if cg else 96
    steps = 2
    Q, G, grid, mu, name = sample_workload(args, n)
    cores = os.cpu_count() or 1
    P = oracle.params(n=grid.n, L=grid.L, scheme=1 if cg else 0, nonlinear=1, mu0=mu,
                      threads=cores)
    oracle.run(P, Q.copy(), G.copy() if cg else None, nsteps=1)  # warm
    t0 = time.perf_counter()
    oracle.run(P, Q, G if cg else None, nsteps=steps)
    el = time.perf_counter() - t0
    stages = 2 if cg else 1
    return {"value": n ** 3 * stages * steps / el, "unit": METRIC, "cores": cores,
            "kind": "oracle",
            "sample": f"{name} {n}^3 {args.scheme} FP64 nonlinear, {steps} steps ({el:.1f} s)"}


def reference_arm(args, rank):
    """The oracle timed on the host cores, each step a bounded sample of the
    benchmark's workload (24^3 CGKS-5th, 48^3 GKS-2nd)."""
    if rank != 0:
        return None
    import oracle
    cg = args.scheme == "cgks5"
    n = 24 if cg else 48
    Q, G, grid, mu, name = sample_workload(args, n)
    cores = os.cpu_count() or 1
    P = oracle.params(n=grid.n, L=grid.L, scheme=1 if cg else 0, nonlinear=1, mu0=mu,
                      threads=cores)
    for _ in range(args.warmup):
        oracle.run(P, Q, G if cg else None, nsteps=1)
    t0 = time.perf_counter()
    oracle.run(P, Q, G if cg else None, nsteps=args.steps)
    el = time.perf_counter() - t0
    stages = 2 if cg else 1
    val = n ** 3 * stages * args.steps / el
    full_n = getattr(args, "n", None) or 512
    tag = "learned" if getattr(args, "indicator", False) else getattr(args, "precision", "fp64")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "cell-stage/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the GPU arm's config (same workload name and physics); each timed
        # step is a bounded sample of it, described in cpu_baseline.sample
        "config": {"workload": f"{name}_{full_n}^3_{args.scheme}_{tag}_nonlinear",
                   "cells": full_n ** 3, "scheme": args.scheme, "stages_per_step": stages,
                   "gamma": 1.4, "Pr": 0.72, "cfl": 0.3, "parallelism": "host cores",
                   "sample": f"{name} {n}^3 per timed step (same generator and physics)"},
        "cpu_baseline": {"value": val, "unit": "cell-stage/s", "cores": cores, "kind": "oracle",
                         "sample": f"{name} {n}^3 {args.scheme} FP64, {args.steps} steps"},
        "e2e": {"value": val, "unit": "cell-stage/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    return line


# ---------------------------------------------------------------------------
def trained_indicator(torch, dev):
    """Train the smoothness-indicator network on the GPU (library kernels:
    dumps of the solver's own data vectors and chi, loss/gradient/Adam)."""
    from paper_2508_19911_gb300 import indicator as ind
    t0 = time.time()
    x, y, stats = ind.training_set(dev, n=32)
    params, hist = ind.train(x, y, epochs=6, seed=1)
    info = {"theta": ind.THETA, "label_eps": ind.LABEL_EPS, "samples": int(y.numel()),
            "label_1_fraction": float(y.mean().item()), "final_loss": float(hist[-1]),
            "train_s": time.time() - t0}
    del x, y
    torch.cuda.empty_cache()
    return params.cpu().numpy(), info


def _dist_ready():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier_ranks():
    """Barrier over the ranks (no-op in a single process)."""
    if _dist_ready():
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(torch, x):
    """The largest value of a host float over the ranks: the slowest rank
    sets a replica run's time (NCCL: reduced on this rank's GPU; gloo: on
    the host)."""
    if not _dist_ready():
        return float(x)
    import torch.distributed as dist
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kinetic_energy(Q):
    """per-cell rho |U|^2 / 2 of a state [5][...] (device tensor)"""
    return 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]


def rel_l2(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def replica_throughput(world, cells, stages, steps, ms):
    """Whole-job cell-stage updates per second of `world` independent
    replicas, each advancing `cells` cells `steps` steps, timed by the
    slowest rank (ms)."""
    return world * cells * stages * steps / (ms / 1e3)


def time_steps(torch, solver, Q, G, steps, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        solver.step(Q, G, nsteps=1, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)  # ms


def time_kernel(torch, fn, reps, stream):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps  # ms per launch


def make_workload(args):
    """Initial cell averages and gradients of the benchmark workload (host,
    numpy; setup only) with its physics and a description."""
    from paper_2508_19911_gb300 import workloads as wl
    n = args.n
    if args.workload == "tgv":
        Qh, Gh, grid = wl.taylor_green(n)
        return dict(Q=Qh, G=Gh, grid=grid, phys=dict(mu=1.0 / 1600), name="taylor_green",
                    data="synthetic (Taylor-Green cell averages)",
                    cfg={"Ma": 0.1, "Re": 1600})
    k0 = 8.0 if args.proxy_of is None else 8.0 * n / args.proxy_of
    mu = 1e-3 if args.proxy_of is None else 1e-3 * args.proxy_of / n
    Qh, Gh, grid, info = wl.isotropic_turbulence(n, Mt=0.5, k0=k0, seed=103)
    cfg = {"Mt": 0.5, "k0": k0, "seed": 103, "mu": mu,
           "taylor_lambda": float(info["taylor_lambda"])}
    if args.proxy_of is not None:
        cfg["proxy_of"] = f"{args.proxy_of}^3 (same cells per wavelength and dt/tau)"
    return dict(Q=Qh, G=Gh, grid=grid, phys=dict(mu=mu), name="isotropic_turbulence",
                data="synthetic (seeded isotropic turbulence, E(k) ~ k^4 exp(-2 (k/k0)^2))",
                cfg=cfg)


def timed_steps(torch, solver, Q, G, warmup, steps, stream, clock_index):
    """W untimed steps, then K steps timed with CUDA events on the solver's
    stream, with the per-kernel launch times recorded inside the timed
    region and the SM clocks sampled during it."""
    for _ in range(warmup):
        solver.step(Q, G, nsteps=1, sync=False)
    torch.cuda.synchronize()
    barrier_ranks()
    solver.kernel_timing(True)
    with ClockSampler(clock_index) as clk:
        ms = time_steps(torch, solver, Q, G, steps, stream)
    solver.kernel_timing(False)
    kt = solver.kernel_times()
    return ms, kt, clk.summary()


def alu_peaks(torch, stream):
    """Measured FMA throughput of this GPU (TFLOP/s), FP64 and FP32."""
    from paper_2508_19911_gb300 import gks
    f64, _ = gks.fma_rate("fp64", stream)
    f32, _ = gks.fma_rate("fp32", stream)
    return f64 / 1e12, f32 / 1e12


def kernel_roofline(kind, ops, kt, units_total, peaks, hbm_peak, hbm_src, clocks):
    """Roofline of one kernel from the launches recorded in the timed
    region: achieved = work per unit x units processed / summed launch
    time (the average launch's work over its average duration)."""
    ms, launches = kt[kind]
    sec = ms / 1e3
    p64, p32 = peaks
    a64 = ops["fp64"] * units_total / sec / 1e12
    a32 = ops["fp32"] * units_total / sec / 1e12
    hbm = ops["bytes"] * units_total / sec / 1e9
    f64, f32 = a64 / p64, a32 / p32
    r = {"kernel": ops["name"], "launches": launches, "ms_per_launch": ms / launches,
         "units_per_launch": units_total / launches}
    if f64 >= f32:  # the binding unit: the FP64 pipe unless the FP32 one is busier
        r.update({"bound": "alu", "achieved": a64, "peak": p64, "unit": "TFLOP/s (FP64)",
                  "frac": f64})
    else:
        r.update({"bound": "alu", "achieved": a32, "peak": p32, "unit": "TFLOP/s (FP32)",
                  "frac": f32})
    r.update({
        "traffic": ops["dram"] * units_total / launches if ops.get("dram") else None,
        "traffic_note": ops.get("dram_note"),
        "fp64": {"achieved_tflops": a64, "peak_tflops": p64, "frac": f64},
        "fp32": {"achieved_tflops": a32, "peak_tflops": p32, "frac": f32},
        "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak, "frac": hbm / hbm_peak,
                "peak_source": hbm_src},
        "peak_note": "ALU peaks of measured: gks_fma_rate (independent FMA chains on every SM) "
                     f"during this run, SM clock {clocks.get('sm_mhz')} MHz; HBM peak of measured "
                     "copy bandwidth (MEASURED_PEAKS.json)"})
    return r


def path_rooflines(kt, scheme, prec, cells, nxy, slab, stages, steps, peaks, clocks):
    """Rooflines of the reconstruction and flux kernels of one path and the
    dominant one of the two (the larger share of the recorded time)."""
    pk = measured_peaks()
    hbm_peak = pk.get("hbm_gbs") or HBM_FALLBACK_GBS
    hbm_src = "MEASURED_PEAKS.json" if pk.get("hbm_gbs") else "fallback"
    cg = scheme == "cgks5"
    K = 4 if cg else 1
    sfx = {"fp64": "", "mixed": "_mixed", "learned": "_learned"}[prec]
    out = {}
    # flux: every stage computes the faces of every cell (3 axes x K points)
    # reconstruction: every stage reconstructs every cell, and each z-slab
    # also the plane below it
    nslabs = 0 if not slab else -(-(cells // nxy) // slab)
    units = {"flux": 3 * K * cells * stages * steps,
             "recon": (cells + nslabs * nxy) * stages * steps}
    names = {"flux": ("flux_cgks5" if cg else "flux_gks2") + sfx,
             "recon": ("recon5" if cg else "recon2") + sfx}
    for kind in ("recon", "flux"):
        ops = KERNEL_OPS.get(names[kind])
        if ops is None or kt[kind][1] == 0:
            continue
        out[kind] = kernel_roofline(kind, dict(ops, name=names[kind]), kt, units[kind], peaks,
                                    hbm_peak, hbm_src, clocks)
    dom = max(("recon", "flux"), key=lambda k: kt[k][0])
    total = sum(v[0] for v in kt.values())
    share = {k: kt[k][0] / total for k in kt}
    return out.get(dom), out, share


def launches_in(kt, cg, prec, stages, steps):
    """Kernels of this library launched in a timed region: the recorded
    reconstruction, flux and update launches, two per time step (reduction
    + finalisation), and the mixed path's views of the state (the float-float
    split of Q, and for CGKS-5th the FP32 gradient copy) once per stage."""
    n = kt["recon"][1] + kt["flux"][1] + kt["update"][1] + 2 * kt["dt"][1]
    if prec != "fp64":
        n += (2 if cg else 1) * stages * steps
    return n


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2508_19911_gb300 import gks

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    t0 = time.time()
    wk = make_workload(args)
    Qh, Gh, grid = wk["Q"], wk["G"], wk["grid"]
    n = args.n
    scheme = args.scheme
    cg = scheme == "cgks5"
    stages = 2 if cg else 1
    cells, nxy = n ** 3, n * n
    prec = "mixed" if args.indicator else args.precision
    tag = "learned" if args.indicator else prec
    if args.indicator and not cg:
        raise SystemExit("--indicator needs --scheme cgks5")
    want_variants = cg and not args.no_variants and rank == 0
    params, ind_info = None, None
    if args.indicator:
        params, ind_info = trained_indicator(torch, dev)
    setup_s = time.time() - t0

    def new_solver(p, learned):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme=scheme, nonlinear=True,
                                  precision="mixed" if learned else p, indicator=learned,
                                  slab_planes=args.slab_planes, **wk["phys"]), stream)
        if learned:
            s.set_indicator(params, theta=ind_info["theta"])
        return s

    solver = new_solver(prec, args.indicator)
    slab = solver.slab_planes
    Q = torch.tensor(Qh, device=dev)
    G = torch.tensor(Gh, device=dev) if cg else None
    ms, kt, clocks = timed_steps(torch, solver, Q, G, args.warmup, args.steps, stream, local_rank)
    ms = max_over_ranks(torch, ms)
    if args.indicator:
        ind_info["skip_fraction"] = solver.indicator_skips() / (
            5 * (cells + (-(-n // slab) * nxy if slab else 0)) * stages * (args.steps + args.warmup))
    if solver.status():
        raise RuntimeError("non-physical state during the benchmark")
    value = replica_throughput(world, cells, stages, args.steps, ms)
    peaks = alu_peaks(torch, stream)
    roofline, rooflines, share = path_rooflines(kt, scheme, tag, cells, nxy, slab, stages,
                                                args.steps, peaks, clocks)
    # per-cell kinetic energy after the warm-up and timed steps: the FP64
    # reference for the mixed variants' error (same initial state and steps)
    ke_ref = kinetic_energy(Q) if prec == "fp64" else None
    del Q, G
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        # end to end through the C-ABI with host buffers (gks_step_host):
        # every step the library copies the state from pinned host memory
        # to the device, advances it one step and copies it back; all the
        # timed steps of the device leg, from the same initial state
        Qp = torch.from_numpy(Qh).pin_memory()
        Gp = torch.from_numpy(Gh).pin_memory() if cg else None
        solver.step_host(Qp, Gp, nsteps=0)  # first call allocates the device copy
        torch.cuda.synchronize()
        barrier_ranks()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            solver.step_host(Qp, Gp, nsteps=1)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(torch, e0.elapsed_time(e1))
        state_bytes = Qh.nbytes + (Gh.nbytes if cg else 0)
        e2e = {"value": replica_throughput(world, cells, stages, args.steps, e2e_ms),
               "unit": "cell-stage/s", "h2d_bytes_per_step": state_bytes,
               "d2h_bytes_per_step": state_bytes, "ms_per_step": e2e_ms / args.steps,
               "steps": args.steps}
        del Qp, Gp
    solver.close()
    torch.cuda.empty_cache()

    variants = {}
    if want_variants:
        # the learned indicator is not among them: its gain is bounded by
        # GENO's share of the mixed reconstruction (a few percent of the
        # step) and the network costs about what it skips (--indicator runs
        # it as the main path)
        for vtag in ("fp64", "mixed"):
            if vtag == tag:
                continue
            s2 = new_solver("fp64" if vtag == "fp64" else "mixed", vtag == "learned")
            Q2 = torch.tensor(Qh, device=dev)
            G2 = torch.tensor(Gh, device=dev)
            ms2, kt2, clk2 = timed_steps(torch, s2, Q2, G2, args.warmup, args.steps, stream, 0)
            v = {"value": cells * stages * args.steps / (ms2 / 1e3), "unit": "cell-stage/s",
                 "ms_per_step": ms2 / args.steps, "slab_planes": s2.slab_planes,
                 "steps": args.steps, "warmup": args.warmup}
            if vtag == "learned":
                sl = s2.slab_planes
                v["skip_fraction"] = s2.indicator_skips() / (
                    5 * (cells + (-(-n // sl) * nxy if sl else 0)) * stages *
                    (args.steps + args.warmup))
            if s2.status():
                raise RuntimeError(f"non-physical state in the {vtag} variant")
            r2, rs2, sh2 = path_rooflines(kt2, scheme, vtag, cells, nxy, s2.slab_planes, stages,
                                          args.steps, peaks, clk2)
            v.update({"roofline": r2, "rooflines": rs2, "time_share": sh2,
                      "gpu_launches": launches_in(kt2, cg, vtag, stages, args.steps),
                      "clocks": clk2})
            if ke_ref is not None and vtag != "fp64":
                # the stated error: per-cell KE against FP64 after the same steps
                v["ke_rel_l2_vs_fp64"] = rel_l2(kinetic_energy(Q2), ke_ref)
                v["ke_steps"] = args.warmup + args.steps
            variants[f"{scheme}_{vtag}_{n}^3"] = v
            s2.close()
            del Q2, G2
            torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": "cell-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "cell_steps_per_s": value / stages,
        "dtype": "f64" if prec == "fp64" else "f32+f64",
        "indicator": ind_info if args.indicator else None,
        "data": wk["data"],
        "config": dict({"workload": f"{wk['name']}_{n}^3_{scheme}_{tag}_nonlinear",
                        "cells": cells, "scheme": scheme, "stages_per_step": stages,
                        "gamma": 1.4, "Pr": 0.72, "cfl": 0.3, "parallelism": f"replicas{world}",
                        "slab_planes": slab,
                        "l2": "working set larger than L2 (state + face buffers > 129 MB)"},
                       **wk["cfg"]),
        "roofline": roofline, "rooflines": rooflines, "time_share": share,
        "measured_peaks": {"fp64_tflops": peaks[0], "fp32_tflops": peaks[1],
                           "how": "gks_fma_rate, after the timed steps"},
        "e2e": e2e, "gpu_launches": launches_in(kt, cg, prec, stages, args.steps),
        "clocks": clocks, "setup_s": setup_s, "variants": variants,
    }
    return line


def run_c5(args):
    """FP64 and mixed(+learned) CGKS-5th on one seeded isotropic-turbulence
    state (Mt 0.5, k0 8, seed 103; 512^3 by default, z-slabs chosen by the
    library): throughput of each path, its slab size and peak device memory,
    and the relative L2 error of the per-cell kinetic energy of the mixed
    paths against FP64 after the same steps."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n = args.n
    t0 = time.time()
    Qh, Gh, grid, info = wl.isotropic_turbulence(n, Mt=0.5, k0=8.0, seed=103)
    gen_s = time.time() - t0
    cells = n ** 3
    params, ind_info = trained_indicator(torch, dev)

    def ke(Q):
        return 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]

    paths, ke_ref, results = [("fp64", False), ("mixed", False), ("mixed", True)], None, {}
    for prec, learned in paths:
        tag = "learned" if learned else prec
        steps = args.fp64_steps if prec == "fp64" else args.steps
        warm = 1 if prec == "fp64" else args.warmup
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=prec,
                                  indicator=learned, mu=1e-3, slab_planes=args.slab_planes),
                       stream)
        if learned:
            s.set_indicator(params, theta=ind_info["theta"])
        Q = torch.tensor(Qh, device=dev)
        G = torch.tensor(Gh, device=dev)
        torch.cuda.reset_peak_memory_stats(dev)
        free0, total = torch.cuda.mem_get_info(dev)
        for _ in range(warm):
            s.step(Q, G, nsteps=1, sync=False)
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            ms = time_steps(torch, s, Q, G, steps, stream)
        if s.status():
            raise RuntimeError(f"non-physical state in the {tag} run")
        free1, _ = torch.cuda.mem_get_info(dev)
        # KE after the first min(warm + steps) steps of each path: rerun from
        # the initial state for the comparison step count
        results[tag] = {"value": cells * 2 * steps / (ms / 1e3), "unit": "cell-stage/s",
                        "ms_per_step": ms / steps, "steps": steps, "warmup": warm,
                        "slab_planes": s.slab_planes,
                        "device_bytes_in_use": int(total - free1), "clocks": clk.summary()}
        s.close()
        del Q, G
        torch.cuda.empty_cache()
    # accuracy: the same number of steps (the FP64 count) on every path
    k = args.fp64_steps + 1
    kes = {}
    for prec, learned in paths:
        tag = "learned" if learned else prec
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=prec,
                                  indicator=learned, mu=1e-3, slab_planes=args.slab_planes),
                       stream)
        if learned:
            s.set_indicator(params, theta=ind_info["theta"])
        Q = torch.tensor(Qh, device=dev)
        G = torch.tensor(Gh, device=dev)
        s.step(Q, G, nsteps=k)
        if learned:
            results[tag]["skip_fraction"] = s.indicator_skips() / (5 * cells * 2 * k)
        kes[tag] = ke(Q)
        s.close()
        del Q, G
        torch.cuda.empty_cache()
    for tag in ("mixed", "learned"):
        d = kes[tag] - kes["fp64"]
        results[tag]["ke_rel_l2_vs_fp64"] = float(torch.linalg.vector_norm(d) /
                                                  torch.linalg.vector_norm(kes["fp64"]))
        results[tag]["ke_steps"] = k
    line = {
        "metric": METRIC, "value": results["learned"]["value"], "unit": "cell-stage/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": results["learned"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded isotropic turbulence)",
        "config": {"workload": f"isotropic_turbulence_{n}^3_cgks5_fp64_vs_mixed_learned",
                   "cells": cells, "Mt": 0.5, "k0": 8, "seed": 103, "mu": 1e-3,
                   "taylor_lambda": float(info["taylor_lambda"]), "generation_s": gen_s,
                   "indicator": ind_info},
        "paths": results,
    }
    return line


def _dump_history(path, obj):
    if path:
        with open(path, "w") as f:
            json.dump(obj, f)


def run_c2(args):
    """Taylor-Green vortex (Ma 0.1, Re 1600, U0 = L = 1; with --ma2 the
    supersonic one of Sec. 4.2: Ma 2, U0 = sqrt(gamma) Ma, Pr 0.7,
    Sutherland viscosity mu0 = U0/1600), CGKS-5th or GKS-2nd nonlinear, from
    t = 0 to t_end: the kinetic energy E_k and the solenoidal and
    dilatational dissipation eps_S, eps_D sampled every `every` time units
    on each path (FP64, mixed); -dE_k/dt from centred differences of the
    samples; the mixed history's largest deviation from FP64 and the
    relative L2 difference of the per-cell kinetic energy at t_end. Each
    sample time is hit exactly (the last step before it is clamped on the
    device); steps past it are no-ops."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n = args.n
    scheme = args.scheme
    cg = scheme == "cgks5"
    stages = 2 if cg else 1
    if args.ma2:
        Qh, Gh, grid = wl.taylor_green_supersonic(n)
        U0 = math.sqrt(1.4) * 2.0
        phys = dict(mu=U0 / 1600, mu_law=1, Pr=0.7)
    else:
        Qh, Gh, grid = wl.taylor_green(n)
        phys = dict(mu=1.0 / 1600)
    nsamp = int(round(args.t_end / args.every))
    times = [args.every * j for j in range(nsamp + 1)]
    hist, paths, kes = {"times": times}, {}, {}
    for prec in args.precisions.split(","):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme=scheme,
                                  precision="fp64" if prec == "fp64p" else prec,
                                  nonlinear=not args.linear, **phys), stream)
        Q0 = Qh
        if prec == "fp64p":
            rng = np.random.default_rng(2024)
            Q0 = Qh * (1.0 + 1e-14 * rng.uniform(-1.0, 1.0, Qh.shape))
        Q = torch.tensor(Q0, device=dev)
        G = torch.tensor(Gh, device=dev) if cg else None
        t = torch.zeros(1, dtype=torch.float64, device=dev)
        diag = [s.diagnostics(Q, G)]
        steps, ms = 0, 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            for ts in times[1:]:
                while True:
                    t_now = float(t.item())
                    if ts - t_now <= 1e-9 * ts:
                        break
                    dt_est = float(s.compute_dt(Q).item())
                    k = max(1, math.ceil((ts - t_now) / dt_est - 1e-6))
                    e0.record(stream)
                    s.step(Q, G, nsteps=k, t_stop=ts, t=t, sync=False)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                    steps += k
                diag.append(s.diagnostics(Q, G))  # raises on a non-physical state
        kes[prec] = 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]
        s.close()
        del Q, G
        torch.cuda.empty_cache()
        d = np.array(diag)
        ek, es, ed = d[:, 0], d[:, 1], d[:, 2]
        rate = -(ek[2:] - ek[:-2]) / (2 * args.every)
        j = int(np.argmax(rate))
        hist[prec] = {"E_k": ek.tolist(), "eps_S": es.tolist(), "eps_D": ed.tolist()}
        paths[prec] = {
            "steps": steps, "ms_per_step": ms / steps,
            "value": n ** 3 * stages * steps / (ms / 1e3), "unit": "cell-stage/s",
            "E_k_end_over_E_k0": float(ek[-1] / ek[0]),
            "peak_minus_dEk_dt": float(rate[j]), "peak_time": times[j + 1],
            "eps_S_at_peak": float(es[j + 1]), "eps_D_at_peak": float(ed[j + 1]),
            "peak_eps_S": float(es.max()), "peak_eps_S_time": times[int(np.argmax(es))],
            "clocks": clk.summary()}
    if "fp64" in hist:
        ref = hist["fp64"]
        for prec in paths:
            if prec == "fp64":
                continue
            h = hist[prec]
            paths[prec]["max_dev_E_k_vs_fp64"] = float(
                np.max(np.abs(np.array(h["E_k"]) - ref["E_k"])) / ref["E_k"][0])
            paths[prec]["max_dev_eps_S_vs_fp64"] = float(
                np.max(np.abs(np.array(h["eps_S"]) - ref["eps_S"])) / np.max(ref["eps_S"]))
            paths[prec]["ke_rel_l2_vs_fp64_at_end"] = float(
                torch.linalg.vector_norm(kes[prec] - kes["fp64"]) /
                torch.linalg.vector_norm(kes["fp64"]))
    _dump_history(args.history, hist)
    first = paths[next(iter(paths))]
    return {
        "metric": METRIC, "value": first["value"], "unit": "cell-stage/s", "n_gpus": 1,
        "steps": first["steps"], "warmup": 0, "ms_per_step": first["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if "fp64" in paths else "f32+f64",
        "data": "synthetic (Taylor-Green cell averages)",
        "config": {"workload": f"taylor_green{'_supersonic' if args.ma2 else ''}_{n}^3_{scheme}_"
                               f"{'linear' if args.linear else 'nonlinear'}_to_t{args.t_end:g}",
                   "cells": n ** 3,
                   "Ma": 2.0 if args.ma2 else 0.1, "Re": 1600, "sample_every": args.every},
        "paths": paths,
    }


def run_c3(args):
    """Decaying isotropic turbulence on [0, 2 pi]^3 (k0 = 8; mu = rho0
    u_rms lambda/Re_lambda with Re_lambda = 72 and lambda the Taylor
    microscale of the discrete initial field): Mt 0.5 (seed 101) and Mt 1.0
    (seed 102), CGKS-5th nonlinear on three paths (FP64, mixed, mixed +
    learned indicator) for the same steps; E_k, eps_S and eps_D after every
    step, the device time of each path, the indicator's skip fraction, and
    the mixed paths' deviations from FP64 (per-cell kinetic energy, relative
    L2, at the end; dissipation histories)."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n = args.n
    cells = n ** 3
    params, ind_info = trained_indicator(torch, dev)
    steps = args.steps
    hist, cases = {}, {}
    for Mt, seed in ((0.5, 101), (1.0, 102)):
        Qh, Gh, grid, info = wl.isotropic_turbulence(n, Mt=Mt, k0=8.0, seed=seed)
        mu = info["u_rms"] * info["taylor_lambda"] / 72.0
        key = f"Mt{Mt:g}"
        hist[key], res, kes = {}, {}, {}
        for prec, learned in (("fp64", False), ("mixed", False), ("mixed", True)):
            tag = "learned" if learned else prec
            s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=prec,
                                      indicator=learned, mu=mu), stream)
            if learned:
                s.set_indicator(params, theta=ind_info["theta"])
            Q = torch.tensor(Qh, device=dev)
            G = torch.tensor(Gh, device=dev)
            diag = [s.diagnostics(Q, G)]
            ms = 0.0
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            for _ in range(steps):
                e0.record(stream)
                s.step(Q, G, nsteps=1, sync=False)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                diag.append(s.diagnostics(Q, G))  # raises on a non-physical state
            d = np.array(diag)
            hist[key][tag] = {"E_k": d[:, 0].tolist(), "eps_S": d[:, 1].tolist(),
                              "eps_D": d[:, 2].tolist(), "min_p": d[:, 4].tolist()}
            res[tag] = {"ms_per_step": ms / steps, "value": cells * 2 * steps / (ms / 1e3),
                        "unit": "cell-stage/s", "E_k_end_over_E_k0": float(d[-1, 0] / d[0, 0]),
                        "eps_D_over_eps_S_end": float(d[-1, 2] / d[-1, 1])}
            if learned:
                res[tag]["skip_fraction"] = s.indicator_skips() / (5 * cells * 2 * steps)
            kes[tag] = 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]
            s.close()
            del Q, G
            torch.cuda.empty_cache()
        ref = hist[key]["fp64"]
        for tag in ("mixed", "learned"):
            dk = kes[tag] - kes["fp64"]
            res[tag]["ke_rel_l2_vs_fp64"] = float(torch.linalg.vector_norm(dk) /
                                                  torch.linalg.vector_norm(kes["fp64"]))
            for q in ("eps_S", "eps_D"):
                r = np.array(ref[q])
                res[tag][f"max_dev_{q}_vs_fp64"] = float(
                    np.max(np.abs(np.array(hist[key][tag][q]) - r)) / np.max(np.abs(r)))
        del kes
        torch.cuda.empty_cache()
        cases[key] = {"seed": seed, "mu": mu, "u_rms": info["u_rms"],
                      "taylor_lambda": info["taylor_lambda"], "paths": res}
    _dump_history(args.history, hist)
    lead = cases["Mt0.5"]["paths"]["learned"]
    return {
        "metric": METRIC, "value": lead["value"], "unit": "cell-stage/s", "n_gpus": 1,
        "steps": steps, "warmup": 0, "ms_per_step": lead["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded isotropic turbulence)",
        "config": {"workload": f"isotropic_turbulence_{n}^3_cgks5_Mt0.5_Mt1.0", "cells": cells,
                   "k0": 8, "Re_lambda": 72, "indicator": ind_info},
        "cases": cases,
    }


def run_c4(args):
    """The batched ensemble (row a9): 64 seeded 2D instances of 64^2..512^2
    cells advanced together, a step as one persistent launch over one work
    list (mode 1; mode 0: one persistent launch per phase, for
    comparison), captured in a CUDA graph, tile size from the autotuner;
    cell-stage updates per second over all instances."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    insts = wl.ensemble_instances(64, seed0=2000)
    spec = [dict(n=g.n, L=g.L, **ph) for _, _, g, ph in insts]
    cells = sum(g.n[0] * g.n[1] * g.n[2] for _, _, g, _ in insts)
    out = {}
    for prec in ("fp64", "mixed"):
        for mode in (1, 0):
            e = gks.Ensemble(spec, precision=prec)
            e.set_mode(mode)
            for i, (Q, G, _, _) in enumerate(insts):
                q, gg = e.views(i)
                q.copy_(torch.tensor(Q, device=dev))
                gg.copy_(torch.tensor(G, device=dev))
            tile, tune_ms = e.autotune()
            e.step(args.warmup, graph=True)
            torch.cuda.synchronize()
            with ClockSampler(0) as clk:
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(torch.cuda.current_stream(dev))
                e.step(args.steps, graph=True)
                t1.record(torch.cuda.current_stream(dev))
                torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            e.times()  # raises if an instance became non-physical or a wait ran out
            launches = 1 if mode == 1 else (8 if prec == "fp64" else 12)
            out[f"{prec}_mode{mode}"] = {
                "value": cells * 2 * args.steps / (ms / 1e3), "unit": "cell-stage/s",
                "ms_per_step": ms / args.steps, "tile": tile, "autotune_ms_per_step": tune_ms,
                "launches_per_step": launches, "clocks": clk.summary()}
            e.close()
            torch.cuda.empty_cache()
    return {
        "metric": METRIC, "value": out["fp64_mode1"]["value"], "unit": "cell-stage/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": out["fp64_mode1"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded 2D double shear layers and four-quadrant Riemann problems)",
        "config": {"workload": "ensemble_64x2d_64..512", "instances": 64, "cells": cells,
                   "launches_per_step": 1},
        "paths": out,
    }


def run_general(args):
    """Row N3 measured: CGKS-5th nonlinear on the Taylor-Green octant with
    six symmetry planes (mirror ghosts) on a stretched mesh, through the
    general-grid kernels, FP64 and mixed; the same cell count on the
    periodic uniform kernels beside it (the cost of the general gathers and
    the boundary faces). Cell-stage updates per second."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n = args.n
    e = wl.stretched_edges(2 * n, 2 * np.pi, 0.3)[:n + 1]
    Qo, Go, go = wl.taylor_green(edges=(e, e, e))
    Qp, Gp, gp = wl.taylor_green(n)
    out = {}
    for prec in ("fp64", "mixed"):
        for name, (Q, G, grid, kw) in {
                "octant_symmetry_stretched": (Qo, Go, go, dict(bc=("symmetry",) * 3,
                                                              spacing=go.spacing)),
                "periodic_uniform": (Qp, Gp, gp, {})}.items():
            s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision=prec,
                                      mu=1.0 / 1600, **kw), stream)
            Qd, Gd = torch.tensor(Q, device=dev), torch.tensor(G, device=dev)
            ms, kt, clk = timed_steps(torch, s, Qd, Gd, args.warmup, args.steps, stream, 0)
            if s.status():
                raise RuntimeError(f"non-physical state ({name}, {prec})")
            out[f"{name}_{prec}"] = {
                "value": n ** 3 * 2 * args.steps / (ms / 1e3), "unit": "cell-stage/s",
                "ms_per_step": ms / args.steps,
                "recon_ms": kt["recon"][0] / max(kt["recon"][1], 1),
                "flux_ms": kt["flux"][0] / max(kt["flux"][1], 1), "clocks": clk}
            s.close()
            del Qd, Gd
            torch.cuda.empty_cache()
    for prec in ("fp64", "mixed"):
        out[f"general_over_periodic_{prec}"] = (out[f"octant_symmetry_stretched_{prec}"]["value"] /
                                                out[f"periodic_uniform_{prec}"]["value"])
    return {
        "metric": METRIC, "value": out["octant_symmetry_stretched_fp64"]["value"],
        "unit": "cell-stage/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": out["octant_symmetry_stretched_fp64"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Taylor-Green cell averages)",
        "config": {"workload": f"taylor_green_octant_{n}^3_symmetry_stretched_cgks5",
                   "cells": n ** 3, "stretch": "0.7-1.3 of the mean cell"},
        "paths": out,
    }


# FP64 work per unit of the line-form kernels (ncu op counts on the
# Taylor-Green 32^3 case of --lines; an FMA counts 2): the reconstruction
# per cell, the flux per face Gauss point (12 per cell)
LINES_OPS = {
    "recon": {"name": "recon5_lines_kernel", "unit": "cell", "per_cell": 1, "fp64": 19289.0},
    "flux": {"name": "flux_faces_lines_kernel", "unit": "Gauss point", "per_cell": 12,
             "fp64": 3756.5},
}


def lines_cpu_baseline():
    """The oracle's line form as it stands, all host cores, on a bounded
    sample: Taylor-Green 32^3, one step."""
    import oracle
    from paper_2508_19911_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    Q, _, grid, L = wl.taylor_green(8, lines=True)
    oracle.run_b(oracle.params(n=grid.n, L=grid.L, threads=cores), Q, L, nsteps=1)  # tables
    n = 32
    Q, _, grid, L = wl.taylor_green(n, lines=True)
    P = oracle.params(n=grid.n, L=grid.L, mu0=1.0 / 1600, threads=cores)
    t0 = time.perf_counter()
    oracle.run_b(P, Q, L, nsteps=1)
    el = time.perf_counter() - t0
    return {"value": n ** 3 * 2 / el, "unit": "cell-stage/s", "cores": cores, "kind": "oracle",
            "sample": f"taylor_green {n}^3 cgks5 lines FP64 nonlinear, 1 step ({el:.1f} s)"}


def run_lines(args):
    """Row N2 measured: CGKS-5th nonlinear FP64 with the 12 line-averaged
    derivatives per variable as the cell's own data (a dense 34 x 72
    reconstruction, per-Gauss-point interface values, every line advanced)
    against the averaged-gradient form, Taylor-Green n^3. Cell-stage
    updates per second, CUDA events on the solver's stream."""
    import torch

    from paper_2508_19911_gb300 import gks
    from paper_2508_19911_gb300 import workloads as wl

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n = args.n
    Q, G, grid, L = wl.taylor_green(n, lines=True)
    out = {}
    for form in ("lines", "gradients"):
        s = gks.Solver(gks.Config(n=grid.n, L=grid.L, scheme="cgks5", precision="fp64",
                                  mu=1.0 / 1600), stream)
        Qd = torch.tensor(Q, device=dev)
        Xd = torch.tensor(L if form == "lines" else G, device=dev)
        step = s.step_lines if form == "lines" else s.step
        for _ in range(args.warmup):
            step(Qd, Xd, nsteps=1, sync=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            step(Qd, Xd, nsteps=args.steps, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # the per-kernel split from a second timed pass with launch events
        s.kernel_timing(True)
        step(Qd, Xd, nsteps=args.steps, sync=False)
        torch.cuda.synchronize()
        s.kernel_timing(False)
        kt = s.kernel_times()
        if s.status():
            raise RuntimeError(f"non-physical state ({form})")
        out[form] = {"value": n ** 3 * 2 * args.steps / (ms / 1e3), "unit": "cell-stage/s",
                     "ms_per_step": ms / args.steps, "clocks": clk.summary(),
                     "kernel_ms_per_launch": {k: (v[0] / v[1] if v[1] else None)
                                              for k, v in kt.items()}}
        if form == "lines":
            p64, _ = alu_peaks(torch, stream)
            roof = {}
            for kind, ops in LINES_OPS.items():
                ms_l = kt[kind][0] / max(kt[kind][1], 1)
                units = n ** 3 * ops["per_cell"]
                r = {"kernel": ops["name"], "unit": ops["unit"], "ms_per_launch": ms_l,
                     "fp64_flop_per_unit": ops["fp64"]}
                if ops["fp64"]:
                    a = ops["fp64"] * units / (ms_l / 1e3) / 1e12
                    r.update({"bound": "alu", "achieved": a, "peak": p64,
                              "unit_rate": "TFLOP/s (FP64)", "frac": a / p64,
                              "peak_note": "measured FP64 FMA rate (gks_fma_rate)"})
                roof[kind] = r
            out[form]["roofline"] = roof
        s.close()
        del Qd, Xd
        torch.cuda.empty_cache()
    out["lines_over_gradients"] = out["lines"]["value"] / out["gradients"]["value"]
    cpu = None if args.no_cpu else lines_cpu_baseline()
    return {
        "metric": METRIC, "value": out["lines"]["value"], "unit": "cell-stage/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["lines"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Taylor-Green cell averages and line-averaged derivatives)",
        "config": {"workload": f"taylor_green_{n}^3_cgks5_lines", "cells": n ** 3},
        "roofline": out["lines"]["roofline"], "cpu_baseline": cpu,
        "paths": out,
    }


def main():
    args = parse()
    if args.lines:
        print(json.dumps(run_lines(args)))
        return
    if args.general:
        print(json.dumps(run_general(args)))
        return
    if args.c4:
        print(json.dumps(run_c4(args)))
        return
    if args.c5:
        print(json.dumps(run_c5(args)))
        return
    if args.c2:
        print(json.dumps(run_c2(args)))
        return
    if args.c3:
        print(json.dumps(run_c3(args)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = reference_arm(args, rank)
        if line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
