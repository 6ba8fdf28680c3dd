"""Shared helpers of the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs and compare."""
import numpy as np

import paper_2004_13887_gb300 as sph


def rel_err(a, b):
    """max-norm error of a against b, relative to max |b| (per field)."""
    s = float(np.max(np.abs(b)))
    d = float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
    return d / s if s > 0 else d


def to_host(fields):
    return [f.detach().cpu().numpy() for f in fields]


def to_dev(fields):
    import torch
    return [torch.from_numpy(np.array(f, dtype=np.float64, copy=True)).to("cuda") for f in fields]


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
