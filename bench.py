#!/usr/bin/env python
"""Throughput of the direction-splitting step (arXiv 2004.13887, Section 2.2) on GB300.

Workload: the rising thermal bubble of Section 3.2 on the regional sector
r in [6371, 6381] km, 20 km x 20 km, 128 x 256 x 256 cells, dry air, Gaussian
potential-temperature perturbation (seeded), dt = 1 s.  One "step" is one time
step t^n -> t^{n+1}: K = 2 Picard iterations, each the right-hand side of
eq. (spl1) and the three line sweeps of eqs. (spl1)-(spl3).

Metric: grid-point updates/s = cells x steps / time (whole job: summed over
ranks for N > 1, each rank advancing its own replica; no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GRID = (128, 256, 256)
K_ITER = 2
DT = 1.0
WORKLOAD = ("rising thermal bubble, regional sector r=[6371,6381] km x 20 km x 20 km, "
            "128x256x256 cells, K=2 Picard iterations/step, dt=1 s")
METRIC = "grid-point updates/s"
UNIT = "points/s"

# FP64 operations (DADD + DMUL + 2 DFMA, counted from the kernels' SASS
# instruction mix with ncu, profiles/fp64_counts_bubble_64cubed.md) per grid
# point of one K = 2 step of the FP64 mode: 2 x (1000 right-hand side, which
# also stores the line rows + 158 coefficients + 834 sweeps, which read them)
# + 15 (the second iteration's average).
FP64_FLOP_PER_POINT_STEP = 4000.0
# FP64 FMA throughput of GB300 measured on this machine with independent FMA
# chains (152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz); MEASURED_PEAKS.json has no
# FP64 figure, so this is the library's own measurement.
FP64_PEAK_TFLOPS = 1.257


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth in MEASURED_PEAKS.json, else
    the profiling recipe's fallback figure"""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = hbm_peak()

# Algorithmic bytes per grid point of each mixed-precision kernel launch: the
# information it must move once -- no coefficient planes, no elimination
# scratch, no halo re-reads (those are what ncu's DRAM traffic adds on top):
#   sweep_r/theta : rhs in (5 x 4 B) + Ubar in (5 x 4) + increment out (5 x 4)        =  60
#   sweep_phi     : rhs in (5 x 4) + Ubar in (5 x 4) + U^k in and out (2 x 5 x 8)     = 120
#   rhs           : U^n and U^k in (2 x 5 x 8) + R out (5 x 4)                         = 100
#   coef          : Ubar in (5 x 4) + 17 coefficient planes out (17 x 4)               =  88
#   avg           : U^n and U^k in (2 x 5 x 8) + Ubar out (5 x 4)                      = 100
MIXED_BYTES_PER_POINT = {"sweep_r": 60, "sweep_theta": 60, "sweep_phi": 120, "rhs": 100, "coef": 88, "avg": 100}

# DRAM traffic of each mixed stage measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over the stage's launches, per grid point, the mean of
# the two Picard iterations of a step; profiles/traffic_bubble_64x256x256_mixed.md),
# measured on the 64 x 256 x 256 window of the same sector (the ncu capture
# stays small; its FP64 state, 168 MB, still exceeds L2), and the hash of the
# kernel sources it was measured on: reported only while the sources match.
# The stencil stages (avg, coef, rhs) move the same bytes per point on any
# grid of the sector, so their figures scale to the workload by the point
# count; the sweeps only where their line layouts are the same (theta and phi
# lines of 256 cells; the window's r lines are 64 cells, the workload's 128).
TRAFFIC_GRID = (64, 256, 256)
MEASURED_TRAFFIC = {"avg": 92.6, "coef": 75.4, "rhs": 199.0, "sweep_theta": 68.6, "sweep_phi": 130.6}
PER_POINT_STAGES = ("avg", "coef", "rhs", "sweep_theta", "sweep_phi")
TRAFFIC_SOURCE_HASH = "8343889b4a6ba17a"


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the CUDA sources and the C header"""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(root, "paper_2004_13887_gb300", "csrc")
    h = hashlib.sha256()
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    for f in files + [os.path.join(root, "include", "sph.h")]:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        """start sampling every 20 ms and return once the first sample is in,
        so that the timed region that follows is covered"""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.f.name) == 0 and self.proc.poll() is None:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle

def oracle_grid(steps: int):
    """The oracle's sample of the workload for a run of `steps` steps: the whole
    128 x 256 x 256 sector up to 60 steps (about 3 s per step on the GPU host's
    16 cores, so the default 20 + 3 steps take about a minute), else its
    central 128 x w x w columns (same cells, same bubble)."""
    from inputs import cases
    if steps <= 60:
        return cases.bubble_grid(GRID)
    w = 128 if steps <= 240 else 64
    return cases.bubble_window(GRID, (w, w))


def oracle_sample(steps: int):
    """The oracle on a bounded sample of the workload (about 10-15 s of host
    time at the default 4 steps of the whole sector), K = 2."""
    import oracle
    from inputs import cases
    grid = oracle_grid(steps)
    c = cases.bubble(GRID, seed=1, dt=DT, grid=grid)
    oracle.build()
    U = c.init
    U, _ = oracle.step(grid, c.par, U, c.dt, K_ITER, bg=c.bg)   # untimed warm-up (page-in)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = oracle.step(grid, c.par, U, c.dt, K_ITER, bg=c.bg)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": grid.npoints * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{grid.nr}x{grid.nt}x{grid.np} cells of the same sector and bubble (central columns "
                      f"when narrower than the workload), {steps} step(s) of K={K_ITER} after one untimed step, "
                      f"FP64 C oracle with OpenMP over lines",
            "seconds": dt}


# ------------------------------------------------------------- our arm

def max_over_ranks(ms, dist, device="cuda"):
    """The job's time is the slowest replica's: an all-reduce MAX of each rank's
    CUDA-event time (the only collective of the benchmark; replicas exchange no
    data)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank, steps, world, t_max_ms):
    """grid-point updates/s of the whole job: every rank advances its own copy
    of the workload (weak scaling), timed by the slowest rank"""
    return points_per_rank * steps * world / (t_max_ms / 1e3)


def time_path(solver, args, dist, local):
    """warm-up, then the timed steps (CUDA events on the library's stream, no
    per-stage timing inside the timed region), then a separate pass of the
    same number of steps with the library's per-stage CUDA events on, for the
    stage shares and the dominant stage's launch time.  The timed steps replay
    a CUDA graph of two steps recorded on the solver's own stream (the
    library's sph_batch_capture of one context): no host launch or per-step
    status read between kernels; the status (non-finite values, zero pivots)
    is read once after the timed steps."""
    import torch
    from paper_2004_13887_gb300 import Batch
    for _ in range(args.warmup):
        solver.step(DT, K_ITER)
    torch.cuda.synchronize()
    graph = Batch([solver], stream=solver.stream)
    graph.capture(DT, K_ITER, 2)
    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = solver.launches
    e0.record(solver.stream)
    graph.launch(args.steps // 2)
    if args.steps % 2:
        solver.step_async(DT, K_ITER)
    e1.record(solver.stream)
    torch.cuda.synchronize()
    solver.status()
    graph.close()
    launches = solver.launches - l0
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    t_max = max_over_ranks(e0.elapsed_time(e1), dist)
    # stage profile: a separate pass (its events would perturb the headline)
    solver.profile(True)
    for _ in range(max(2, min(args.steps, 10))):
        solver.step(DT, K_ITER)
    kern = solver.profile_read()
    solver.profile(False)
    return t_max, kern, launches, clocks


def field_errors(Um, Ud, c):
    """relative L2 error of the mixed state against FP64, per physical field"""
    import numpy as np
    bgp, bgT = c.bg
    par = c.par
    Rg = par.cv * (par.gamma - 1.0)
    out = {}
    P = [U[0] + bgp[1:-1][:, None, None] for U in (Um, Ud)]
    T = [U[4] + bgT[1:-1][:, None, None] for U in (Um, Ud)]
    rho = [(p + par.pinf) / (Rg * t) for p, t in zip(P, T)]
    th = [t * (bgp[1] / p) ** (Rg / (par.gamma * par.cv)) for p, t in zip(P, T)]
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    out["p"], out["rho"], out["theta"], out["T"] = rel(*P), rel(*rho), rel(*th), rel(*T)
    num = sum(float(np.linalg.norm(Um[q] - Ud[q])) ** 2 for q in (1, 2, 3))
    den = sum(float(np.linalg.norm(Ud[q])) ** 2 for q in (1, 2, 3))
    out["u"] = math.sqrt(num / max(den, 1e-300))
    return out


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    import paper_2004_13887_gb300 as sph
    from inputs import cases

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        sph.build()
    if dist is not None:
        dist.barrier()
    c = cases.bubble(GRID, seed=1, dt=DT)
    g = c.grid
    N = g.npoints
    dev = [torch.from_numpy(f.copy()).cuda() for f in c.init]

    # FP64 path, timed first (the reference point of the mixed path's error)
    U64 = None
    if args.only in ("both", "fp64"):
        s64 = sph.Solver(g, c.par, precision=sph.SPH_PREC_FP64, stream=torch.cuda.Stream())
        s64.set_background(*c.bg)
        s64.set_state(dev)
        t64, kern64, _, _ = time_path(s64, args, dist, local)
        U64 = [f.cpu().numpy() for f in s64.get_state()]
        s64.close()
        del s64
        torch.cuda.empty_cache()
    if args.only == "fp64":
        return {"metric": METRIC, "value": job_throughput(N, args.steps, world, t64), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t64 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64"}}

    solver = sph.Solver(g, c.par, precision=sph.SPH_PREC_MIXED, stream=torch.cuda.Stream())
    solver.set_background(*c.bg)
    solver.set_state(dev)
    stream = solver.stream

    t_max, kern, launches, clocks = time_path(solver, args, dist, local)
    value = job_throughput(N, args.steps, world, t_max)
    Um = [f.cpu().numpy() for f in solver.get_state()]
    errors, fp64 = None, None
    if U64 is not None:
        errors = {"metric": "relative L2 after warmup+steps steps", **field_errors(Um, U64, c)}
        ach64 = FP64_FLOP_PER_POINT_STEP * N * args.steps / (t64 * 1e-3) / 1e12
        fp64 = {"value": job_throughput(N, args.steps, world, t64), "ms_per_step": t64 / args.steps,
                "kernel_shares": {k: round(v[0] / max(sum(x[0] for x in kern64.values()), 1e-30), 4)
                                  for k, v in kern64.items() if v[1]},
                "roofline": {"bound": "fp64", "kernel": "whole FP64 step (all stages)", "unit": "TFLOP/s",
                             "flop_per_point_step": FP64_FLOP_PER_POINT_STEP, "achieved": ach64,
                             "peak": FP64_PEAK_TFLOPS, "frac": ach64 / FP64_PEAK_TFLOPS,
                             "peak_source": "FP64 FMA rate measured by this library on the pool's GB300 "
                                            "(MEASURED_PEAKS.json has no FP64 figure)",
                             "hbm_note": "the FP64 step does ~4000 FP64 flop per point against ~2.5 KB of traffic: "
                                         "bound by the FP64 pipe, not HBM"}}

    # dominant kernel of the mixed step and its HBM roofline
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_n = kern[dom]
    per_launch_ms = dom_ms / max(dom_n, 1)
    bpp = MIXED_BYTES_PER_POINT.get(dom)
    traffic = None
    if dom in MEASURED_TRAFFIC and TRAFFIC_SOURCE_HASH == kernel_source_hash() and \
            (tuple(GRID) == TRAFFIC_GRID or dom in PER_POINT_STAGES):
        traffic = MEASURED_TRAFFIC[dom] * N   # bytes per stage launch (all its kernels), scaled by the points
    roof = {"bound": "hbm", "kernel": dom, "unit": "GB/s", "peak": HBM_PEAK_GBS,
            "peak_source": HBM_PEAK_SOURCE, "timing": "CUDA events around each stage, separate pass of the same steps",
            "launch_ms": per_launch_ms, "traffic": traffic, "bytes_per_point": bpp}
    if bpp:
        achieved = bpp * N / (per_launch_ms * 1e-3) / 1e9
        roof.update(achieved=achieved, frac=achieved / HBM_PEAK_GBS)
    else:
        roof.update(achieved=None, frac=None)
    shares = {k: round(v[0] / max(sum(x[0] for x in kern.values()), 1e-30), 4) for k, v in kern.items() if v[1]}

    # end to end through the C ABI with host buffers (pinned), copies timed
    pinned = [torch.empty(s, dtype=torch.float64).pin_memory() for s in solver.shapes]
    for p, f in zip(pinned, c.init):
        p.numpy()[...] = f
    host = [p.numpy() for p in pinned]
    nb = sum(int(np.prod(s)) * 8 for s in solver.shapes)
    out_pinned = [torch.empty(s, dtype=torch.float64).pin_memory() for s in solver.shapes]
    out = [p.numpy() for p in out_pinned]
    e2e_steps = max(3, min(args.steps, 10))
    solver.set_state(host)
    solver.step(DT, K_ITER)
    solver.get_state(device=False, out=out)
    torch.cuda.synchronize()
    # one context: copy in, step, copy out, one after the other
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(host)
        solver.step(DT, K_ITER)
        solver.get_state(device=False, out=out)
    torch.cuda.synchronize()
    e2e_serial_s = time.perf_counter() - t0
    # two contexts on two host threads (each on its own stream), each stepping
    # problems whose state lives in pinned host memory: one context's copies
    # (host link) overlap the other's step (GPU); every step still copies its
    # whole state in and out
    solver2 = sph.Solver(g, c.par, precision=sph.SPH_PREC_MIXED, stream=torch.cuda.Stream())
    solver2.set_background(*c.bg)
    out2 = [torch.empty(s_, dtype=torch.float64).pin_memory().numpy() for s_ in solver.shapes]
    solver2.set_state(host)
    solver2.step(DT, K_ITER)
    solver2.get_state(device=False, out=out2)
    torch.cuda.synchronize()
    e2e_pipe_steps = 2 * e2e_steps

    def e2e_worker(sv, o, n):
        torch.cuda.set_device(local)
        for _ in range(n):
            sv.set_state(host)
            sv.step(DT, K_ITER)
            sv.get_state(device=False, out=o)

    import threading
    th = [threading.Thread(target=e2e_worker, args=(sv, o, e2e_steps)) for sv, o in ((solver, out), (solver2, out2))]
    t0 = time.perf_counter()
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = job_throughput(N, e2e_pipe_steps, world, e2e_s * 1e3)
    e2e_serial = job_throughput(N, e2e_steps, world, e2e_serial_s * 1e3)
    solver2.close()
    solver.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "K": K_ITER, "dt_s": DT,
                   "precision": "mixed: FP32 stencils and line solves; FP64 state, update, div u, cyclic corrections",
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch": "CUDA graph of two steps on the solver's stream (sph_batch_capture), status read "
                             "after the timed steps",
                   "l2": (f"no flush: the state (5 FP64 fields, {nb / 1e6:.0f} MB) and per-iteration buffers "
                          f"exceed the 129 MB L2" if nb > 129e6 else
                          f"no flush: the state ({nb / 1e6:.0f} MB) fits the 129 MB L2 (small case)")},
        "roofline": roof,
        "kernel_shares": shares,
        "error_vs_fp64": errors,
        "fp64_plain": fp64,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
                "steps": e2e_pipe_steps,
                "how": "C ABI with pinned host buffers: per step sph_set_state (host in), sph_step, sph_get_state "
                       "(host out); two contexts on two host threads, so one's copies overlap the other's step",
                "one_context_in_sequence": e2e_serial},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    return line


def run_reference(args, rank, world):
    """The oracle (FP64 C, OpenMP over lines) on the host cores; rank 0 only."""
    if rank != 0:
        return None
    import numpy as np   # noqa: F401
    import oracle
    from inputs import cases
    grid = oracle_grid(args.steps + args.warmup)
    c = cases.bubble(GRID, seed=1, dt=DT, grid=grid)
    oracle.build()
    U = c.init
    for _ in range(args.warmup):
        U, _ = oracle.step(grid, c.par, U, c.dt, K_ITER, bg=c.bg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _ = oracle.step(grid, c.par, U, c.dt, K_ITER, bg=c.bg)
    dt = time.perf_counter() - t0
    value = grid.npoints * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{grid.nr}x{grid.nt}x{grid.np} cells of the same sector and bubble per step, "
              f"K={K_ITER}, FP64 C oracle, OpenMP over lines")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "K": K_ITER, "dt_s": DT, "precision": "fp64",
                       "sample_grid": [grid.nr, grid.nt, grid.np],
                       "same_config": [grid.nr, grid.nt, grid.np] == list(GRID)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ensemble(args, rank, world, dist):
    """The batched ensemble (64 bubbles on uneven grids, mixed precision, one
    CUDA graph per two steps, line solver autotuned per grid shape): grid-point
    updates/s summed over the instances.  Not the default workload."""
    import numpy as np
    import torch
    from paper_2004_13887_gb300 import ensemble
    from inputs import cases
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    specs = cases.ensemble_specs()
    # the instances are partitioned across the ranks by points (level 1 of the
    # multi-GPU design: independent problems, no data-path collective)
    share = ensemble.partition([int(np.prod(sp["n"])) for sp in specs], world)[rank]
    cs = [cases.bubble(specs[q]["n"], seed=specs[q]["seed"], dt=DT, amplitude=specs[q]["amplitude"],
                       radius=specs[q]["radius"]) for q in share]
    ens = ensemble.Ensemble(cs, dt=DT, n_iter=K_ITER)
    steps = args.steps + (args.steps & 1)
    warm = max(args.warmup + (args.warmup & 1), 4)
    ens.run(warm)
    ens.status()
    l0 = sum(s.launches for s in ens.solvers)
    sampler = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0.record(ens.batch.stream)
    ens.run(steps)
    e1.record(ens.batch.stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ens.status()
    t_max = max_over_ranks(e0.elapsed_time(e1), dist)
    pts = ens.points
    total_pts = sum(int(np.prod(sp["n"])) for sp in specs)   # every rank's share together
    value = total_pts * steps / (t_max * 1e-3)
    bpp = K_ITER * sum(MIXED_BYTES_PER_POINT.values())
    achieved = bpp * pts * steps / (t_max * 1e-3) / 1e9   # this rank's share on this rank's GPU
    shapes = {}
    for c in cs:
        k = f"{c.grid.nr}x{c.grid.nt}x{c.grid.np}"
        shapes[k] = shapes.get(k, 0) + 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": t_max / steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batched ensemble: 64 independent thermal bubbles on the 20 km sector, uneven grids "
                                   "nr in {16,32,48,64}, n_theta and n_phi in {64,128,192,256}, amplitude 0.2-1 K, "
                                   "radius 1-3 km, K=2, dt=1 s, one CUDA graph per two steps",
                       "launch": ("batched: one kernel per stage and line layout over all instances (instance "
                                  "descriptor tables in device memory)") if ens.fused else "one graph branch per instance",
                       "launch_ms_per_step": {("batched" if k else "graph_branches"): v for k, v in ens.mode_ms.items()},
                       "instances": len(specs), "instances_rank0": len(cs), "points": total_pts,
                       "points_rank0": pts, "shapes": shapes,
                       "line_solver": {f"{k[0]}x{k[1]}x{k[2]}": ({0: "thomas", 1: "partitioned", 2: "partitioned_warp", 3: "partitioned_narrow"}[v[0]])
                                       for k, v in ens.choice.items()},
                       "tile": {f"{k[0]}x{k[1]}x{k[2]}": f"{128 // (v[1][0] * v[1][1])}x{v[1][0]}x{v[1][1]}"
                                for k, v in ens.choice.items()},
                       "parallelism": "instances partitioned by points across ranks" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": "whole step (all stages)", "unit": "GB/s", "peak": HBM_PEAK_GBS,
                         "achieved": achieved, "frac": achieved / HBM_PEAK_GBS, "traffic": None,
                         "bytes_per_point": bpp},
            "gpu_launches": sum(s.launches for s in ens.solvers) - l0, "clocks": clocks}
    ens.close()
    return line


def run_adjoint(args, rank, world, dist):
    """The gradient workload: d(final kinetic energy)/d(initial potential-
    temperature perturbation) over 20 steps of a 96 x 192 x 192 bubble (plus 1e-3
    white noise), FP64, through the autograd Function with checkpoints every
    ceil(sqrt(20)) = 5 steps; the gradient checked against central differences
    along 2 seeded directions.  Metric: grid-point updates/s of the forward
    steps, the adjoint steps and the recomputation together."""
    import numpy as np
    import torch
    import paper_2004_13887_gb300 as sph
    from paper_2004_13887_gb300 import adjoint
    from inputs import cases
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        sph.build()
    c = cases.adjoint_bubble()
    g, par, bg = c.grid, c.par, c.bg
    nsteps = 20
    s = sph.Solver(g, par)
    s.set_background(*bg)
    Pi = torch.as_tensor(c.info["Pi"], device="cuda")
    base = [torch.as_tensor(f, device="cuda") for f in c.init]
    th0 = torch.as_tensor(c.info["theta0"], device="cuda")

    def J_of(theta):
        U0 = [base[0], base[1], base[2], base[3], Pi * theta]
        return adjoint.kinetic_energy(adjoint.steps(s, c.dt, K_ITER, nsteps, U0), g, bg, par)

    # warm-up (allocates the adjoint's workspace), then the timed gradient
    th = th0.clone().requires_grad_(True)
    J_of(th).backward()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = s.launches
    t0 = time.perf_counter()
    th = th0.clone().requires_grad_(True)
    J = J_of(th)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    clocks = sampler.stop()
    launches = s.launches - l0
    grad = th.grad.detach()
    rng = np.random.default_rng(7)
    checks = []
    with torch.no_grad():
        for _ in range(2):
            v = torch.as_tensor(rng.standard_normal(g.shapes()[4]), device="cuda")
            eps = 1e-4
            fd = (float(J_of(th0 + eps * v)) - float(J_of(th0 - eps * v))) / (2 * eps)
            ad = float(torch.sum(grad * v))
            checks.append(abs(fd - ad) / max(abs(fd), 1e-300))
    longest, cap = s.tape_use()
    s.close()
    # forward 20 steps + backward (20 recomputed steps + 20 adjoint steps)
    N = g.npoints
    total = t2 - t0
    line = {"metric": "grid-point updates/s of the gradient (forward + recompute + adjoint steps)",
            "value": N * nsteps / total, "unit": UNIT, "n_gpus": world, "steps": nsteps, "warmup": 1,
            "ms_per_step": 1e3 * total / nsteps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "adjoint: gradient of the final kinetic energy after 20 steps w.r.t. the initial "
                                   "potential-temperature perturbation, bubble 96x192x192 + 1e-3 white noise, K=2, "
                                   "dt=1 s, checkpoints every 5 steps", "grid": [g.nr, g.nt, g.np]},
            "forward_s": t1 - t0, "backward_s": t2 - t1, "kinetic_energy": float(J),
            "fd_check_rel_diff": checks, "tape_longest": longest, "tape_capacity": cap,
            "gpu_launches": launches, "clocks": clocks}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default=None, help="nr,nt,np of a smaller sector (profiling of small cases)")
    ap.add_argument("--workload", choices=["bubble", "ensemble", "adjoint"], default="bubble",
                    help="ensemble: the 64-instance batched ensemble; adjoint: the gradient workload "
                         "(instead of the benchmark workload)")
    ap.add_argument("--only", choices=["both", "mixed", "fp64"], default="both",
                    help="profiling: run one path only (the JSON line then lacks the other)")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the ensemble and gradient workloads the default line also carries")
    args = ap.parse_args()
    if args.grid:
        global GRID, WORKLOAD
        GRID = tuple(int(v) for v in args.grid.split(","))
        WORKLOAD = WORKLOAD.replace("128x256x256", "x".join(map(str, GRID)))
    if args.warmup < 3:
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch.distributed as dist_
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist_.init_process_group("nccl")
        dist = dist_
    if args.workload in ("ensemble", "adjoint"):
        line = (run_ensemble if args.workload == "ensemble" else run_adjoint)(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    line = run_ours(args, rank, world, dist)
    if world == 1 and not args.no_extras and args.only == "both" and not args.grid:
        # the other two workloads, each in its own key (their own metrics; the
        # headline stays the benchmark workload's)
        import torch
        torch.cuda.empty_cache()
        ea = argparse.Namespace(**vars(args))
        ea.steps, ea.warmup = 10, 4
        try:
            e = run_ensemble(ea, rank, world, dist)
            line["ensemble"] = {k: e[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "roofline",
                                                  "gpu_launches", "clocks")}
            line["ensemble"]["workload"] = e["config"]["workload"]
            line["ensemble"]["line_solver"] = e["config"]["line_solver"]
            line["ensemble"]["tile"] = e["config"]["tile"]
            line["ensemble"]["launch"] = e["config"]["launch"]
            line["ensemble"]["launch_ms_per_step"] = e["config"]["launch_ms_per_step"]
        except Exception as ex:   # the headline stands without it
            line["ensemble"] = {"error": str(ex)}
        torch.cuda.empty_cache()
        try:
            a = run_adjoint(args, rank, world, dist)
            line["adjoint"] = {k: a[k] for k in ("metric", "value", "unit", "ms_per_step", "forward_s", "backward_s",
                                                 "fd_check_rel_diff", "tape_longest", "gpu_launches", "clocks")}
            line["adjoint"]["workload"] = a["config"]["workload"]
        except Exception as ex:
            line["adjoint"] = {"error": str(ex)}
    if rank == 0:
        if not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = oracle_sample(4)
            except Exception as e:   # the GPU number stands without it
                line["cpu_baseline"] = {"error": str(e)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
