"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This package holds the problem definitions only -- grids, material constants,
initial and background states, wall data and manufactured-solution forcing --
and none of the scheme's arithmetic (no discrete operator, no line solve).

Field order everywhere: U = [p, u_r, u_theta, u_phi, T] (Section 2.1).  Layout:
C order, phi fastest; p, T at cell centres, each velocity component on the
faces normal to it (MAC, Section 2.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Grid:
    """Spherical sector [r1,r2] x [t1,t2] x [p1,p2], nr x nt x np uniform cells."""
    nr: int
    nt: int
    np: int
    r1: float
    r2: float
    t1: float
    t2: float
    p1: float
    p2: float
    periodic: bool = False

    @property
    def npf(self) -> int:
        return self.np if self.periodic else self.np + 1

    @property
    def dr(self):
        return (self.r2 - self.r1) / self.nr

    @property
    def dth(self):
        return (self.t2 - self.t1) / self.nt

    @property
    def dph(self):
        return (self.p2 - self.p1) / self.np

    @property
    def npoints(self) -> int:
        return self.nr * self.nt * self.np

    def shapes(self):
        nr, nt, n, npf = self.nr, self.nt, self.np, self.npf
        return [(nr, nt, n), (nr + 1, nt, n), (nr, nt + 1, n), (nr, nt, npf), (nr, nt, n)]

    def wall_shape(self, c: int, d: int):
        nr, nt, n, npf = self.nr, self.nt, self.np, self.npf
        table = {
            (0, 1): (nr + 1, n), (0, 2): (nr + 1, nt), (0, 0): (nt, n),
            (1, 0): (nt + 1, n), (1, 2): (nr, nt + 1), (1, 1): (nr, n),
            (2, 0): (nt, npf), (2, 1): (nr, npf), (2, 2): (nr, nt),
        }
        return table[(c, d)]

    def zeros(self):
        return [np.zeros(s) for s in self.shapes()]

    # 1-D coordinates
    def rc(self):
        return self.r1 + (np.arange(self.nr) + 0.5) * self.dr

    def rf(self):
        return self.r1 + np.arange(self.nr + 1) * self.dr

    def tc(self):
        return self.t1 + (np.arange(self.nt) + 0.5) * self.dth

    def tf(self):
        return self.t1 + np.arange(self.nt + 1) * self.dth

    def pc(self):
        return self.p1 + (np.arange(self.np) + 0.5) * self.dph

    def pf(self):
        return self.p1 + np.arange(self.npf) * self.dph

    def coords(self, f: int):
        """Broadcastable (R, TH, PH) of field f's locations."""
        R = self.rf() if f == 1 else self.rc()
        TH = self.tf() if f == 2 else self.tc()
        PH = self.pf() if f == 3 else self.pc()
        return R[:, None, None], TH[None, :, None], PH[None, None, :]

    def wall_coords(self, c: int, d: int, s: int):
        """(R, TH, PH) of the wall values of component c on the wall normal to d, side s."""
        lo_hi = [(self.r1, self.r2), (self.t1, self.t2), (self.p1, self.p2)]
        R, TH, PH = self.coords(1 + c)
        axes = [R, TH, PH]
        axes[d] = np.array(lo_hi[d][s]).reshape(1, 1, 1)
        full = np.broadcast_arrays(*axes)
        keep = [a for a in range(3) if a != d]
        sh = tuple(full[0].shape[a] for a in keep)
        return [np.ascontiguousarray(x.squeeze(axis=d)).reshape(sh) for x in full]


@dataclass
class Params:
    """Constants of eqs. (nonconservmass)-(nonconserveos): gamma = cp/cv,
    kappa = mu*cp/Pr; g along e_r on the left-hand side; omega about the polar axis."""
    gamma: float
    cv: float
    Pr: float
    mu: float
    pinf: float = 0.0
    g: float = 0.0
    omega: float = 0.0


def sample(fns, grid: Grid, *args):
    """Evaluate 5 callables f(R, TH, PH, *args) at the staggered locations."""
    out = []
    for f, fn in enumerate(fns):
        R, TH, PH = grid.coords(f)
        v = np.broadcast_to(np.asarray(fn(R, TH, PH, *args), dtype=np.float64),
                            grid.shapes()[f])
        out.append(np.ascontiguousarray(v))
    return out


def sample_walls(vel_fns, grid: Grid, *args):
    """Wall data dict (c, d, s) -> array from exact velocity callables (3 of them)."""
    walls = {}
    for c in range(3):
        for d in range(3):
            if d == 2 and grid.periodic:
                continue
            for s in range(2):
                R, TH, PH = grid.wall_coords(c, d, s)
                v = np.broadcast_to(np.asarray(vel_fns[c](R, TH, PH, *args), dtype=np.float64),
                                    grid.wall_shape(c, d))
                walls[(c, d, s)] = np.ascontiguousarray(v)
    return walls
