"""The bounds-checked debug build (SPH_CHECKED) as the memory checker's stand-in:
every flat field index the kernels form is checked, violations are counted and
redirected, and the run goes on (nothing traps).  Small grids (4^3 .. 8^3 and an
8 x 16 x 16 grid whose 16-cell lines take the partitioned solver) through every
kind of call -- steps in both precisions, the stage calls, wall data, periodic
lines with and without poles, the adjoint -- must leave the count at zero."""
import math

import numpy as np
import pytest

import paper_2004_13887_gb300 as sph
from paper_2004_13887_gb300 import _build
from inputs import Grid, Params, cases
from tests.gpu_helpers import perturbed, solver_for, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    path = _build.build(checked=True)
    prev = sph.use_library(path)
    assert sph.bounds_report()[0] == 0
    yield
    sph.restore_library(prev)


def _cases():
    out = []
    c = cases.sector_mms((4, 5, 6))
    out.append(("sector", c.grid, c.par, c.bg, c.init, c.source(0.5 * c.dt), c.dt))
    c = cases.bubble((6, 7, 8), seed=2, dt=1.0)
    out.append(("bubble", c.grid, c.par, c.bg, c.init, None, c.dt))
    c = cases.sector_mms((3, 5, 7))   # odd field sizes: sub-buffers at odd offsets would misalign pair loads
    out.append(("ragged", c.grid, c.par, c.bg, c.init, c.source(0.5 * c.dt), c.dt))
    c = cases.bubble((8, 16, 16), seed=2, dt=1.0)
    out.append(("bubble16", c.grid, c.par, c.bg, c.init, None, c.dt))
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.05, pinf=2.0, g=0.3, omega=0.4)
    for name, t1, t2 in (("shell", 0.4, 2.7), ("shell_pole", 0.0, math.pi)):
        g = Grid(4, 6, 8, 1.0, 1.3, t1, t2, 0.0, 2 * math.pi, periodic=True)
        U = perturbed(g.zeros(), [0.1, 0.05, 0.05, 0.05, 0.1], 5, g)
        U[2][:, 0] = U[2][:, -1] = 0
        bg = (np.full(g.nr + 2, 20.0), np.full(g.nr + 2, 30.0))
        out.append((name, g, par, bg, U, None, 0.01))
    return out


def test_no_index_leaves_its_field(checked):
    for name, g, par, bg, U, S, dt in _cases():
        for prec in (sph.SPH_PREC_FP64, sph.SPH_PREC_MIXED):
            s = solver_for(g, par, bg, U, precision=prec)
            s.step(dt, 2, S)
            s.set_iterate(perturbed(U, [1e-3] * 5, 6, g))
            s.rhs(dt, S)
            for d in range(3):
                s.sweep(d, dt, to_dev(perturbed(g.zeros(), [1.0] * 5, 7 + d, g)))
            if prec == sph.SPH_PREC_FP64:
                s.set_state(U)
                s.step_adjoint(dt, 2, to_dev(perturbed(g.zeros(), [1.0] * 5, 9, g)),
                               source=to_dev(S) if S is not None else None)
            s.close()
            n, first = sph.bounds_report()
            assert n == 0, (name, prec, n, first)
    w = cases.paper_mms(1e-2, n=(4, 5, 6))
    s = solver_for(w.grid, w.par, w.bg, w.init)
    s.set_bc(w.walls(0.0), w.walls(w.dt))
    s.step(w.dt, 2, w.source(0.5 * w.dt))
    s.close()
    n, first = sph.bounds_report()
    assert n == 0, ("walls", n, first)
