"""Batched ensembles of independent problems of different sizes: one solver
per instance (mixed precision), stepped together by a CUDA graph (Batch),
with the line solver of each grid shape chosen by timing (autotune)."""
from __future__ import annotations

import numpy as np

from . import (SPH_LINES_PARTITIONED, SPH_LINES_PARTITIONED_NARROW, SPH_LINES_PARTITIONED_WARP, SPH_LINES_THOMAS,
               SPH_PREC_MIXED, Batch, Solver)


def _partitioned_applies(grid) -> bool:
    return any(n in (16, 32, 48, 64, 128, 192, 256) for n in (grid.nr, grid.nt, grid.np)) or grid.np in (512, 1024)


def _candidates(grid, fused=False):
    """the line solvers worth timing on a grid: the narrow layout only where a
    direction has lines of 16 to 64 cells, the one-warp layout only where one
    has 64 or 128; block Thomas unless the grid goes into batched launches,
    which take partitioned layouts only"""
    if not _partitioned_applies(grid):
        return () if fused else (SPH_LINES_THOMAS,)
    ns = (grid.nr, grid.nt, grid.np)
    out = [SPH_LINES_PARTITIONED]
    if any(n in (64, 128) for n in ns):
        out.append(SPH_LINES_PARTITIONED_WARP)
    if any(n in (16, 32, 48, 64) for n in ns):
        out.append(SPH_LINES_PARTITIONED_NARROW)
    if not fused:
        out.append(SPH_LINES_THOMAS)
    return tuple(out)


def partition(points, world: int):
    """Split instances of the given sizes (grid points) over `world` ranks,
    balanced by points: largest first, each to the rank with the fewest points
    so far (ties to the lower rank).  Returns one sorted list of instance
    indices per rank; every index appears exactly once.  The instances are
    independent, so each rank steps its share alone -- no data-path
    collective."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for q in sorted(range(len(points)), key=lambda q: (-points[q], q)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(q)
        load[r] += points[q]
    return [sorted(p) for p in parts]


def time_steps(solver, dt, n_iter, steps=2, warmup=1):
    """milliseconds per step on the solver's stream (CUDA events)"""
    import torch
    for _ in range(warmup):
        solver.step_async(dt, n_iter)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(solver.stream)
    for _ in range(steps):
        solver.step_async(dt, n_iter)
    e1.record(solver.stream)
    solver.status()
    return e0.elapsed_time(e1) / steps


TILES = ((1, 1), (2, 1), (4, 1), (2, 2), (8, 1), (4, 2))


def autotune(cases, dt, n_iter, tiles=TILES, fused=False):
    """For every distinct grid shape among the cases: the fastest line solver of
    the mixed mode (partitioned, partitioned with a warp per line, partitioned
    with few lanes per short line, or block Thomas), then with it the fastest stencil tile shape among `tiles`, each
    timed on one scratch solver started from that shape's first case.
    Returns {shape: (SPH_LINES_*, (tj, ti))}."""
    import torch
    choice = {}
    for c in cases:
        shape = (c.grid.nr, c.grid.nt, c.grid.np)
        if shape in choice:
            continue
        s = Solver(c.grid, c.par, precision=SPH_PREC_MIXED, stream=torch.cuda.Stream())
        s.set_background(*c.bg)
        init = [torch.from_numpy(np.array(f, dtype=np.float64, copy=True)).cuda() for f in c.init]
        solvers = _candidates(c.grid, fused)
        if not solvers:
            raise ValueError(f"grid {shape}: no partitioned layout for batched launches")
        best, best_ms = None, None
        for which in solvers:
            s.set_state(init)
            s.set_line_solver(which)
            ms = time_steps(s, dt, n_iter)
            if best_ms is None or ms < best_ms:
                best, best_ms = which, ms
        s.set_line_solver(best)
        tile, tile_ms = tiles[0], None
        for tj, ti in tiles:
            s.set_state(init)
            s.set_tile(tj, ti)
            ms = time_steps(s, dt, n_iter)
            if tile_ms is None or ms < tile_ms:
                tile, tile_ms = (tj, ti), ms
        s.close()
        choice[shape] = (best, tile)
    return choice


def _batchable(grid) -> bool:
    """whether batched launches take the grid: partitioned layouts in all three
    directions"""
    ok = (16, 32, 48, 64, 128, 192, 256)
    return grid.nr in ok and grid.nt in ok and (grid.np in ok or grid.np in (512, 1024))


class Ensemble:
    """cases: objects with grid, par, bg, init (inputs.cases.Case).  Each gets
    a mixed-precision solver on its own stream; step() replays a graph of
    `graph_steps` steps of all of them.  fused: record the graph from batched
    launches (one kernel per stage and line layout over every instance,
    sph_batch_capture_fused) rather than one branch of launches per instance;
    None: when every grid allows batched launches, both graphs are timed on
    the ensemble (a few steps each, then every state is put back to its
    initial value) and the faster is kept (mode_ms holds the two timings)."""

    def __init__(self, cases, dt, n_iter=2, tune=True, graph_steps=2, fused=None):
        import torch
        self.cases = list(cases)
        self.dt, self.n_iter = dt, n_iter
        modes = [bool(fused)] if fused is not None else \
            ([True, False] if all(_batchable(c.grid) for c in self.cases) else [False])
        self.fused = modes[0]
        self.mode_ms = {}
        self.choice = autotune(self.cases, dt, n_iter, fused=self.fused) if tune else {}
        self.solvers = []
        for c in self.cases:
            s = Solver(c.grid, c.par, precision=SPH_PREC_MIXED, stream=torch.cuda.Stream())
            s.set_background(*c.bg)
            s.set_state([torch.from_numpy(np.array(f, dtype=np.float64, copy=True)).cuda() for f in c.init])
            shape = (c.grid.nr, c.grid.nt, c.grid.np)
            if shape in self.choice:
                which, (tj, ti) = self.choice[shape]
                s.set_line_solver(which)
                s.set_tile(tj, ti)
            self.solvers.append(s)
        torch.cuda.synchronize()
        self.batch = Batch(self.solvers)
        self.graph_steps = graph_steps
        if len(modes) > 1:
            for m in modes:
                self.batch.capture(dt, n_iter, graph_steps, fused=m)
                self.mode_ms[m] = self._time_replays()
            for s, c in zip(self.solvers, self.cases):
                s.set_state([torch.from_numpy(np.array(f, dtype=np.float64, copy=True)).cuda() for f in c.init])
            torch.cuda.synchronize()
            self.fused = min(self.mode_ms, key=self.mode_ms.get)
        self.batch.capture(dt, n_iter, graph_steps, fused=self.fused)

    def _time_replays(self, replays=2):
        """milliseconds per step of the captured graph (one warm-up replay)"""
        import torch
        self.batch.launch(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.batch.stream)
        self.batch.launch(replays)
        e1.record(self.batch.stream)
        self.batch.status()
        return e0.elapsed_time(e1) / (replays * self.graph_steps)

    @property
    def points(self) -> int:
        return sum(c.grid.nr * c.grid.nt * c.grid.np for c in self.cases)

    def run(self, steps):
        """advance every instance by `steps` (a multiple of graph_steps) steps"""
        if steps % self.graph_steps:
            raise ValueError(f"steps must be a multiple of {self.graph_steps}")
        self.batch.launch(steps // self.graph_steps)

    def status(self):
        self.batch.status()

    def close(self):
        self.batch.close()
        for s in self.solvers:
            s.close()
