"""Shared pieces of the adjoint tests: seeded generic states on small grids, and
the oracle's finite-difference Jacobian of one step (the oracle-side adjoint:
its transpose applied to a vector)."""
import math

import numpy as np

import oracle
from inputs import Grid, Params, cases


def flat(fields):
    return np.concatenate([np.ravel(f) for f in fields])


def unflat(v, shapes):
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(v[o:o + n].reshape(s).copy())
        o += n
    return out


def generic_state(grid, seed, amp=(2.0, 0.05, 0.05, 0.05, 0.5)):
    """a smooth-ish random state with every component active (walls keep zero
    normal velocity; pole faces zero u_theta)"""
    rng = np.random.default_rng(seed)
    U = [amp[q] * rng.standard_normal(s) for q, s in enumerate(grid.shapes())]
    U[1][0] = U[1][-1] = 0.0
    U[2][:, 0] = U[2][:, -1] = 0.0
    if not grid.periodic:
        U[3][:, :, 0] = U[3][:, :, -1] = 0.0
    return U


def small_cases():
    """name -> (grid, params, background, state, source or None, dt): a walled
    sector with gravity and a radial background, a periodic shell, a shell with
    both poles, and the sector manufactured solution with its source"""
    out = {}
    c = cases.bubble((6, 7, 8), seed=3, dt=1.0)
    out["bubble"] = (c.grid, c.par, c.bg, [a + b for a, b in zip(c.init, generic_state(c.grid, 11, (5.0, 0.02, 0.02, 0.02, 0.05)))],
                     None, 1.0)
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.05, pinf=2.0, g=0.3, omega=0.4)
    bg = lambda g: (np.full(g.nr + 2, 20.0), np.full(g.nr + 2, 30.0))
    g = Grid(5, 6, 8, 1.0, 1.3, 0.4, 2.7, 0.0, 2 * math.pi, periodic=True)
    out["shell"] = (g, par, bg(g), generic_state(g, 12, (0.1, 0.05, 0.05, 0.05, 0.1)), None, 0.01)
    g = Grid(5, 6, 8, 1.0, 1.3, 0.0, math.pi, 0.0, 2 * math.pi, periodic=True)
    out["shell_pole"] = (g, par, bg(g), generic_state(g, 13, (0.1, 0.05, 0.05, 0.05, 0.1)), None, 0.01)
    c = cases.sector_mms((6, 7, 8))
    out["sector_mms"] = (c.grid, c.par, c.bg, c.exact(0.0), c.source(0.5 * c.dt), c.dt)
    return out


def field_scales(U, bg):
    """a magnitude per field for perturbation directions"""
    sc = []
    for q, f in enumerate(U):
        m = float(np.max(np.abs(f)))
        if q == 0:
            m = max(m, 1e-3 * float(np.max(np.abs(bg[0]))))
        if q == 4:
            m = max(m, 1e-3 * float(np.max(np.abs(bg[1]))))
        sc.append(m if m > 0 else 1.0)
    return sc


def oracle_jacobian(grid, par, bg, U, dt, K, S=None, rel=1e-6):
    """d flat(step(U)) / d flat(U) of one oracle step by central differences,
    each column with a step of rel times the field's scale"""
    shapes = grid.shapes()
    x0 = flat(U)
    scales = field_scales(U, bg)
    steps = np.concatenate([np.full(int(np.prod(s)), rel * scales[q]) for q, s in enumerate(shapes)])
    cols = []
    for j in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp[j] += steps[j]
        xm[j] -= steps[j]
        yp, _ = oracle.step(grid, par, unflat(xp, shapes), dt, K, bg=bg, S=S)
        ym, _ = oracle.step(grid, par, unflat(xm, shapes), dt, K, bg=bg, S=S)
        cols.append((flat(yp) - flat(ym)) / (2 * steps[j]))
    return np.stack(cols, axis=1)
