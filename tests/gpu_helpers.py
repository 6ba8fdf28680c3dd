"""Shared helpers of the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs and compare."""
import numpy as np

import oracle
import paper_2004_13887_gb300 as sph
from inputs import Grid


def rel_err(a, b):
    """max-norm error of a against b, relative to max |b| (per field)."""
    s = float(np.max(np.abs(b)))
    d = float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
    return d / s if s > 0 else d


def to_host(fields):
    return [f.detach().cpu().numpy() for f in fields]


def to_dev(fields):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(f)).to("cuda") for f in fields]


def solver_for(grid, par, bg=None, state=None, precision=0):
    s = sph.Solver(grid, par, precision=precision)
    if bg is not None:
        s.set_background(bg[0], bg[1])
    if state is not None:
        s.set_state(state)
    return s


def perturbed(fields, scale, seed, grid):
    """fields + scale*noise with the wall-face normal velocity left unchanged"""
    rng = np.random.default_rng(seed)
    out = []
    for q, f in enumerate(fields):
        n = rng.standard_normal(f.shape) * scale[q]
        if q == 1:
            n[0] = n[-1] = 0
        if q == 2:
            n[:, 0] = n[:, -1] = 0
        if q == 3 and not grid.periodic:
            n[:, :, 0] = n[:, :, -1] = 0
        out.append(f + n)
    return out


def subgrid(grid, i0, i1, j0, j1, k0, k1):
    """The sub-sector of cells [i0,i1) x [j0,j1) x [k0,k1) (full phi range if periodic)."""
    if grid.periodic:
        k0, k1 = 0, grid.np
    return Grid(i1 - i0, j1 - j0, k1 - k0, grid.r1 + i0 * grid.dr, grid.r1 + i1 * grid.dr,
                grid.t1 + j0 * grid.dth, grid.t1 + j1 * grid.dth, grid.p1 + k0 * grid.dph,
                grid.p1 + k1 * grid.dph, periodic=grid.periodic)


def cut(grid, fields, i0, i1, j0, j1, k0, k1):
    if grid.periodic:
        k0, k1 = 0, grid.np
    out = [fields[0][i0:i1, j0:j1, k0:k1], fields[1][i0:i1 + 1, j0:j1, k0:k1],
           fields[2][i0:i1, j0:j1 + 1, k0:k1],
           fields[3][i0:i1, j0:j1, k0:k1 if grid.periodic else k1 + 1], fields[4][i0:i1, j0:j1, k0:k1]]
    return [np.ascontiguousarray(f) for f in out]


def cut_bg(bg, i0, i1):
    return (np.ascontiguousarray(bg[0][i0:i1 + 2]), np.ascontiguousarray(bg[1][i0:i1 + 2]))
