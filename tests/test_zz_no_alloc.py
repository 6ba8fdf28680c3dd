"""The allocation-free line solver, sph_block_thomas_noalloc, against the
library's regular line solve, sph_sweep.

sph_block_thomas_noalloc serves callers that cannot call cudaMalloc: its
elimination scratch is a file-scope device array inside the library instead of
a buffer the library allocates.  Here it receives the same (I + tau/2 D_d)
block systems that sph_sweep solves internally (assembled line by line by the
oracle from the same state) and must return the same block unknowns (p, T and
the normal velocity) to the line-solve tolerance of the other GPU tests, 1e-12
relative, on consecutive calls that reuse the shared scratch array.  This file
is collected last so that a failure here cannot hide any other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from inputs import cases
from tests.gpu_helpers import perturbed, rel_err, solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


def _lines(g, d):
    """(a, b) of every block line along d"""
    if d == 0:
        return [(j, k) for j in range(g.nt) for k in range(g.np)]
    if d == 1:
        return [(i, k) for i in range(g.nr) for k in range(g.np)]
    return [(i, j) for i in range(g.nr) for j in range(g.nt)]


def _pos(d, a, b, m):
    idx = [a, b]
    idx.insert(d, m)
    return tuple(idx)


def _systems(g, par, bg, Ub, d, tau, rhs):
    """stacked (A, B, C, rhs) of all block lines along d, and the solver's unknown layout"""
    n = (g.nr, g.nt, g.np)[d]
    L = _lines(g, d)
    A = np.zeros((len(L), n, 3, 3))
    B = np.zeros_like(A)
    Cb = np.zeros_like(A)
    r = np.zeros((len(L), n, 3))
    for l, (a, b) in enumerate(L):
        A[l], B[l], Cb[l] = oracle.line_system(g, par, Ub, d, 0, a, b, tau, bg=bg)
        for m in range(n):
            p = _pos(d, a, b, m)
            r[l, m, 0] = rhs[0][p]
            r[l, m, 1] = rhs[4][p]
            if m < n - 1:
                f = list(p)
                f[d] = m + 1
                r[l, m, 2] = rhs[1 + d][tuple(f)]
    return A, B, Cb, r, L


def _gather(g, d, L, x_fields):
    n = (g.nr, g.nt, g.np)[d]
    out = np.zeros((len(L), n, 3))
    for l, (a, b) in enumerate(L):
        for m in range(n):
            p = _pos(d, a, b, m)
            out[l, m, 0] = x_fields[0][p]
            out[l, m, 1] = x_fields[4][p]
            if m < n - 1:
                f = list(p)
                f[d] = m + 1
                out[l, m, 2] = x_fields[1 + d][tuple(f)]
    return out


def test_noalloc_matches_sweep_on_consecutive_calls():
    import torch
    sph.build()
    c = cases.bubble((10, 12, 14), seed=2, dt=1.0)
    g, par, bg = c.grid, c.par, c.bg
    Uk = perturbed(c.init, [5.0, 1e-2, 1e-2, 1e-2, 1e-2], 4, g)
    Ub = [0.5 * (a + b) for a, b in zip(c.init, Uk)]
    s = solver_for(g, par, bg, c.init)
    s.set_iterate(Uk)
    for call, d in enumerate((0, 1, 0)):
        rhs = perturbed(g.zeros(), [1.0] * 5, 50 + call, g)
        ref_fields = to_host(s.sweep(d, c.dt, to_dev(rhs)))
        A, B, Cb, r, L = _systems(g, par, bg, Ub, d, c.dt, rhs)
        dev = [torch.from_numpy(v).cuda().contiguous() for v in (A, B, Cb, r)]
        x = sph.block_thomas_noalloc(*dev).cpu().numpy()
        torch.cuda.synchronize()
        ref = _gather(g, d, L, ref_fields)
        for q in range(3):
            assert rel_err(x[..., q], ref[..., q]) <= 1e-12, (call, d, q, rel_err(x[..., q], ref[..., q]))


def test_noalloc_rejects_sizes_beyond_its_array():
    sph.build()
    lib = sph.load()
    dummy = C.cast(C.c_void_p(16), sph._DP)   # never dereferenced: the size check comes first
    assert lib.sph_block_thomas_noalloc(sph.NOALLOC_MAX_BLOCKS + 1, 1, dummy, dummy, dummy, dummy, dummy,
                                        None) == -1
    assert lib.sph_block_thomas_noalloc(0, 4, dummy, dummy, dummy, dummy, dummy, None) == -1
