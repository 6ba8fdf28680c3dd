"""Plain FP64 CPU oracle of the direction-splitting scheme of Frolov, Minev &
Takhirov (arXiv 2004.13887), Section 2 and Appendix B.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library; the product path never
falls back to it.

State layout (numpy float64, C order, phi fastest), see ``oracle.h``::

    p, T : (nr, nt, np)      cell centres (perturbations about a radial background)
    ur   : (nr+1, nt, np)    r-faces
    ut   : (nr, nt+1, np)    theta-faces
    up   : (nr, nt, npf)     phi-faces, npf = np+1, or np when phi is periodic
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable flags only)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
        ):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            if openmp:
                cmd.insert(1, "-fopenmp")
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class _OgGrid(C.Structure):
    _fields_ = [("nr", C.c_int), ("nt", C.c_int), ("np", C.c_int), ("periodic", C.c_int),
                ("r1", C.c_double), ("r2", C.c_double), ("t1", C.c_double), ("t2", C.c_double),
                ("p1", C.c_double), ("p2", C.c_double)]


class _OgPar(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cv", C.c_double), ("Pr", C.c_double), ("mu", C.c_double),
                ("pinf", C.c_double), ("g", C.c_double), ("omega", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(dp)
        for name in ("og_thomas", "og_cyclic_thomas", "og_block_thomas", "og_block_cyclic"):
            f = getattr(L, name)
            f.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            f.restype = C.c_int
        G, P = C.POINTER(_OgGrid), C.POINTER(_OgPar)
        L.og_apply.argtypes = [G, P, pp, dp, dp, pp, C.c_int, pp, dp, dp, pp, pp]
        L.og_line_system.argtypes = [G, P, pp, dp, dp, pp, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_double, dp, dp, dp]
        L.og_rhs.argtypes = [G, P, dp, dp, pp, pp, pp, pp, C.c_double, pp, pp]
        L.og_sweep.argtypes = [G, P, dp, dp, pp, pp, pp, pp, C.c_double, C.c_int, pp, pp]
        L.og_step.argtypes = [G, P, dp, dp, pp, pp, pp, C.c_double, C.c_int, pp, dp]
        for f in (L.og_apply, L.og_line_system, L.og_rhs, L.og_sweep, L.og_step):
            f.restype = C.c_int
        _lib = L
    return _lib


@dataclass
class Grid:
    """Sector [r1,r2] x [t1,t2] x [p1,p2] with nr x nt x np cells (Section 2.1)."""
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


@dataclass
class Params:
    """Material constants of eqs. (nonconservmass)-(nonconserveos)."""
    gamma: float
    cv: float
    Pr: float
    mu: float
    pinf: float = 0.0
    g: float = 0.0
    omega: float = 0.0


_DP = C.POINTER(C.c_double)


def _cgrid(g):
    """Any object with nr, nt, np, r1..p2, periodic attributes."""
    return _OgGrid(int(g.nr), int(g.nt), int(g.np), int(bool(g.periodic)), float(g.r1), float(g.r2),
                   float(g.t1), float(g.t2), float(g.p1), float(g.p2))


def _cpar(p):
    return _OgPar(float(p.gamma), float(p.cv), float(p.Pr), float(p.mu), float(p.pinf), float(p.g),
                  float(p.omega))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"shape {a.shape} != {tuple(shape)}")
    return a


class _Fields:
    """Keeps contiguous copies alive and exposes a double** view."""

    def __init__(self, grid: Grid, fields, out=False):
        shapes = grid.shapes()
        if out:
            self.arrs = [np.zeros(s) for s in shapes]
        else:
            if len(fields) != 5:
                raise ValueError("need 5 fields p, ur, ut, up, T")
            self.arrs = [_arr(f, s) for f, s in zip(fields, shapes)]
        self.ptrs = (_DP * 5)(*[_ptr(a) for a in self.arrs])


class _Walls:
    """walls: dict (c, d, s) -> array, or None."""

    def __init__(self, grid: Grid, walls):
        self.arrs = [None] * 18
        if walls:
            for (c, d, s), v in walls.items():
                self.arrs[(c * 3 + d) * 2 + s] = _arr(v, grid.wall_shape(c, d))
        self.ptrs = (_DP * 18)(*[_ptr(a) for a in self.arrs])


def _bg(grid: Grid, bg):
    if bg is None:
        return None, None
    bgp, bgT = bg
    bgp = None if bgp is None else _arr(bgp, (grid.nr + 2,))
    bgT = None if bgT is None else _arr(bgT, (grid.nr + 2,))
    return bgp, bgT


def _check(e, what):
    if e < 0:
        raise RuntimeError(f"oracle {what} failed with code {e}")
    return e


# ------------------------------------------------------------ line solvers

def thomas(a, b, c, d):
    n = len(b)
    x = np.zeros(n)
    a, b, c, d = (_arr(v) for v in (a, b, c, d))
    _check(lib().og_thomas(n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x)), "thomas")
    return x


def cyclic_thomas(a, b, c, d):
    n = len(b)
    x = np.zeros(n)
    a, b, c, d = (_arr(v) for v in (a, b, c, d))
    _check(lib().og_cyclic_thomas(n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x)), "cyclic")
    return x


def block_thomas(A, B, Cc, d, cyclic=False):
    """A, B, Cc: (n, 3, 3); d: (n, 3)."""
    n = B.shape[0]
    A, B, Cc, d = (_arr(v) for v in (A, B, Cc, d))
    x = np.zeros((n, 3))
    f = lib().og_block_cyclic if cyclic else lib().og_block_thomas
    _check(f(n, _ptr(A), _ptr(B), _ptr(Cc), _ptr(d), _ptr(x)), "block thomas")
    return x


# ------------------------------------------------------------ scheme

def apply_op(grid: Grid, par: Params, Ubar, which: int, V, bg=None, ubar_walls=None,
             v_bg=None, v_walls=None):
    """D_r (0), D_theta (1), D_phi (2) or D_M (3) with coefficients at Ubar, applied to V."""
    ub = _Fields(grid, Ubar)
    v = _Fields(grid, V)
    out = _Fields(grid, None, out=True)
    bgp, bgT = _bg(grid, bg)
    vbgp, vbgT = _bg(grid, v_bg)
    uw, vw = _Walls(grid, ubar_walls), _Walls(grid, v_walls)
    _check(lib().og_apply(C.byref(_cgrid(grid)), C.byref(_cpar(par)), ub.ptrs, _ptr(bgp), _ptr(bgT),
                          uw.ptrs, which, v.ptrs, _ptr(vbgp), _ptr(vbgT), vw.ptrs, out.ptrs), "apply")
    return out.arrs


def line_system(grid: Grid, par: Params, Ubar, direction: int, kind: int, a: int, b: int,
                tau: float, bg=None, ubar_walls=None):
    """(A, B, C) of (I + tau/2 D_d) on one line: blocks (n,3,3) for kind 0, scalars for 1/2."""
    n = [grid.nr, grid.nt, grid.np][direction]
    w = 9 if kind == 0 else 1
    A, B, Cc = (np.zeros(n * w) for _ in range(3))
    ub = _Fields(grid, Ubar)
    bgp, bgT = _bg(grid, bg)
    uw = _Walls(grid, ubar_walls)
    _check(lib().og_line_system(C.byref(_cgrid(grid)), C.byref(_cpar(par)), ub.ptrs, _ptr(bgp), _ptr(bgT),
                                uw.ptrs, direction, kind, a, b, tau, _ptr(A), _ptr(B), _ptr(Cc)),
           "line_system")
    if kind == 0:
        return A.reshape(n, 3, 3), B.reshape(n, 3, 3), Cc.reshape(n, 3, 3)
    return A, B, Cc


def rhs(grid: Grid, par: Params, Un, Uk, tau, bg=None, walls_n=None, walls_k=None, S=None):
    """Right-hand side of eq. (spl1)."""
    un, uk = _Fields(grid, Un), _Fields(grid, Uk)
    s = _Fields(grid, S) if S is not None else None
    out = _Fields(grid, None, out=True)
    bgp, bgT = _bg(grid, bg)
    wn, wk = _Walls(grid, walls_n), _Walls(grid, walls_k)
    _check(lib().og_rhs(C.byref(_cgrid(grid)), C.byref(_cpar(par)), _ptr(bgp), _ptr(bgT), un.ptrs, wn.ptrs,
                        uk.ptrs, wk.ptrs, tau, s.ptrs if s else None, out.ptrs), "rhs")
    return out.arrs


def sweep(grid: Grid, par: Params, Un, Uk, tau, direction, rhs_fields, bg=None, walls_n=None,
          walls_k=None):
    """Solve (I + tau/2 D_dir(Ubar)) x = rhs on every line (eqs. spl1-spl3)."""
    un, uk, r = _Fields(grid, Un), _Fields(grid, Uk), _Fields(grid, rhs_fields)
    out = _Fields(grid, None, out=True)
    bgp, bgT = _bg(grid, bg)
    wn, wk = _Walls(grid, walls_n), _Walls(grid, walls_k)
    _check(lib().og_sweep(C.byref(_cgrid(grid)), C.byref(_cpar(par)), _ptr(bgp), _ptr(bgT), un.ptrs, wn.ptrs,
                          uk.ptrs, wk.ptrs, tau, direction, r.ptrs, out.ptrs), "sweep")
    return out.arrs


def step(grid: Grid, par: Params, U, tau, K, bg=None, walls_n=None, walls_np1=None, S=None):
    """One time step: K iterations of eq. (splitting2) by eqs. (spl1)-(spl3).

    Returns (U^{n+1} as a new list of arrays, per-field RMS of the last increment)."""
    u = _Fields(grid, U)
    for a in u.arrs:
        a.setflags(write=True)
    u.arrs = [a.copy() for a in u.arrs]
    u.ptrs = (_DP * 5)(*[_ptr(a) for a in u.arrs])
    s = _Fields(grid, S) if S is not None else None
    bgp, bgT = _bg(grid, bg)
    wn = _Walls(grid, walls_n)
    wk = _Walls(grid, walls_np1) if walls_np1 is not None else None
    res = np.zeros(5)
    _check(lib().og_step(C.byref(_cgrid(grid)), C.byref(_cpar(par)), _ptr(bgp), _ptr(bgT), u.ptrs, wn.ptrs,
                         wk.ptrs if wk else None, tau, K, s.ptrs if s else None, _ptr(res)), "step")
    return u.arrs, res
