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

# FP64 operations (DADD + DMUL + 2 DFMA, counted from the kernel's SASS
# instruction mix with ncu) per line point of each kernel; None = not measured.
FP64_FLOP_PER_POINT = {"rhs": None, "coef": None, "sweep_r": None, "sweep_theta": None, "sweep_phi": None}
FP64_PEAK_TFLOPS = 1.26   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25)


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
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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

def oracle_sample(steps: int):
    """The oracle on a bounded sample of the workload: the central 128 x w x w
    columns of the same sector (same cells, same bubble), K = 2."""
    import numpy as np
    import oracle
    from inputs import cases
    w = 64 if steps <= 30 else 32
    grid = cases.bubble_window(GRID, (w, w))
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
            "sample": f"central {grid.nr}x{grid.nt}x{grid.np} columns of the same sector and bubble, "
                      f"{steps} step(s) of K={K_ITER}, FP64 C oracle with OpenMP over lines",
            "seconds": dt}


# ------------------------------------------------------------- our arm

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
    solver = sph.Solver(g, c.par, precision=sph.SPH_PREC_FP64)
    solver.set_background(*c.bg)
    dev = [torch.from_numpy(f.copy()).cuda() for f in c.init]
    solver.set_state(dev)
    stream = solver.stream

    for _ in range(args.warmup):
        solver.step(DT, K_ITER)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = solver.launches
    solver.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.step(DT, K_ITER)
    e1.record(stream)
    torch.cuda.synchronize()
    kern = solver.profile_read()
    solver.profile(False)
    launches = solver.launches - l0
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = N * args.steps * world / (t_max / 1e3)

    # dominant kernel and its roofline
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_n = kern[dom]
    per_launch_ms = dom_ms / max(dom_n, 1)
    units = N   # every kernel processes each cell once per launch
    fpp = FP64_FLOP_PER_POINT.get(dom)
    roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
            "peak_source": "FP64 nominal from unit counts and clocks (no measured FP64 peak on file)",
            "launch_ms": per_launch_ms, "traffic": None}
    if fpp:
        achieved = fpp * units / (per_launch_ms * 1e-3) / 1e12
        roof.update(achieved=achieved, frac=achieved / FP64_PEAK_TFLOPS, flop_per_point=fpp)
    else:
        roof.update(achieved=None, frac=None)
    shares = {k: round(v[0] / max(sum(x[0] for x in kern.values()), 1e-30), 4) for k, v in kern.items() if v[1]}

    # end to end through the C ABI with host buffers (pinned), copies timed
    pinned = [torch.empty(s, dtype=torch.float64).pin_memory() for s in solver.shapes]
    for p, f in zip(pinned, c.init):
        p.numpy()[...] = f
    host = [p.numpy() for p in pinned]
    nb = sum(int(np.prod(s)) * 8 for s in solver.shapes)
    e2e_steps = max(3, min(args.steps, 10))
    solver.set_state(host)
    solver.step(DT, K_ITER)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state(host)
        solver.step(DT, K_ITER)
        out = solver.get_state(device=False)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = N * e2e_steps * world / e2e_s
    solver.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "K": K_ITER, "dt_s": DT, "precision": "fp64",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: the state (5 FP64 fields, 336 MB) and per-iteration buffers exceed the 129 MB L2"},
        "roofline": roof,
        "kernel_shares": shares,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
                "steps": e2e_steps},
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
    w = 64 if args.steps + args.warmup <= 30 else 32
    grid = cases.bubble_window(GRID, (w, w))
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
    sample = (f"central {grid.nr}x{grid.nt}x{grid.np} columns of the same sector and bubble per step, "
              f"K={K_ITER}, FP64 C oracle, OpenMP over lines")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "K": K_ITER, "dt_s": DT, "precision": "fp64",
                       "sample_grid": [grid.nr, grid.nt, grid.np]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default=None, help="nr,nt,np of a smaller sector (profiling of small cases)")
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
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        if not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = oracle_sample(2)
            except Exception as e:   # the GPU number stands without it
                line["cpu_baseline"] = {"error": str(e)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
