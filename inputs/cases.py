"""Problem set-ups of Section 3 and of the benchmark workloads.

* ``paper_mms``  -- the manufactured solution of eq. (man_sol) on the paper's
  domain [1,2] x [pi/4,3pi/4] x [pi/4,7pi/4], p0 = 6250, gamma = 1.6, mu = 1,
  Pr = 1, omega = 0, g = 0, c_v = 1 (c_v is not given in Section 3.1; any value
  keeps rho = 1).  Time-dependent Dirichlet velocity on every wall.
* ``sector_mms`` -- a smooth manufactured solution on the regional sector
  r in [6371, 6381] km (non-dimensionalised by 10 km), theta in [pi/4, 3pi/4],
  phi in [0, pi/2]: sin/cos products with seeded random phases, no-slip walls
  and zero normal derivative of p and T (so the boundary data are homogeneous),
  a well-prepared velocity (solenoidal O(u0) part + O(u0 M0) part), Mach 1e-2.
* ``bubble``     -- the rising thermal bubble of Section 3.2 on the sector of
  "Thermal 1" (r in [6371, 6381] km, 20 km x 20 km), dry air, a discretely
  hydrostatic background and a Gaussian potential-temperature perturbation.

Forcing S(t) (eq. dU/dt + N(U) + G = S) needs sympy; ``sector_mms`` with the
default seed reads a module generated from the same sympy definitions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import Grid, Params, sample, sample_walls

SECTOR_SEED = 20041388


@dataclass
class Case:
    name: str
    grid: Grid
    par: Params
    dt: float
    steps: int
    K: int
    bg: Optional[tuple]                      # (bgp, bgT), each nr+2 values
    init: list                               # 5 arrays (perturbation about bg)
    exact: Optional[Callable] = None         # t -> 5 arrays (perturbation form)
    walls: Optional[Callable] = None         # t -> wall dict or None
    source: Optional[Callable] = None        # t -> 5 arrays or None
    info: dict = field(default_factory=dict)


# ------------------------------------------------------------------ helpers

def _const_bg(grid: Grid, p0: float, T0: float):
    return np.full(grid.nr + 2, float(p0)), np.full(grid.nr + 2, float(T0))


def _mms_callables(exprs, p0, T0, par, with_source=True):
    """From sympy full-field expressions build exact(t) / source(t) callables."""
    import sympy as sp
    from .continuous import operator, lambdify, t as ts
    pert = [exprs[0] - p0, exprs[1], exprs[2], exprs[3], exprs[4] - T0]
    ex = lambdify(pert, with_t=True)
    src = None
    if with_source:
        N = operator(*exprs, gamma=par.gamma, cv=par.cv, Pr=par.Pr, mu=par.mu, pinf=par.pinf,
                     g=par.g, omega=par.omega)
        S = [sp.diff(e, ts) + n for e, n in zip(exprs, N)]
        src = lambdify(S, with_t=True)
    return ex, src


# --------------------------------------------------------------- paper MMS

def paper_mms_exprs(u0: float, p0: float = 6250.0, gamma: float = 1.6, cv: float = 1.0):
    import sympy as sp
    from .continuous import r, th, ph, t
    c0 = math.sqrt(gamma * p0)
    p = p0 + u0 ** 2 * (1 + sp.sin(5 * t) + sp.cos(sp.pi * r) ** 2 * sp.cos(4 * ph) ** 2 * sp.cos(4 * th) ** 2)
    ur = u0 * (1 + sp.sin(t)) / (2 * r ** 2) + u0 ** 2 / c0 * (
        1 + sp.sin(4 * t) + sp.sin(r ** 2) * sp.cos(th) ** 3 * sp.sin(ph) ** 2)
    ut = u0 * (1 + sp.cos(3 * t + 2)) / (2 * sp.sin(th)) + u0 ** 2 / c0 * (
        1 + sp.sin(t) + sp.cos(r ** 2) ** 3 * sp.cos(th) ** 2 * sp.sin(ph) ** 3)
    up = u0 * (1 + sp.sin(6 + t)) / 2 + u0 ** 2 / c0 * (
        1 + sp.cos(2 + t) + sp.cos(r) * sp.sin(th) ** 3 * sp.sin(ph) ** 2)
    T = p / (cv * (gamma - 1))
    return [p, ur, ut, up, T]


def paper_mms(M0: float, n=(8, 16, 48), dt: float = 1e-3, steps: int = 10, K: int = 2) -> Case:
    """eq. (man_sol) with u0 = M0 c0, c0 = sqrt(gamma p0) = 100 (Section 3.1)."""
    p0, gamma, cv = 6250.0, 1.6, 1.0
    par = Params(gamma=gamma, cv=cv, Pr=1.0, mu=1.0)
    c0 = math.sqrt(gamma * p0)
    u0 = M0 * c0
    grid = Grid(n[0], n[1], n[2], 1.0, 2.0, math.pi / 4, 3 * math.pi / 4, math.pi / 4, 7 * math.pi / 4)
    exprs = paper_mms_exprs(u0, p0, gamma, cv)
    T0 = p0 / (cv * (gamma - 1))
    ex, src = _mms_callables(exprs, p0, T0, par)
    bg = _const_bg(grid, p0, T0)
    exact = lambda tt: sample(ex, grid, tt)
    walls = lambda tt: sample_walls([lambda R, TH, PH, s, f=ex[c + 1]: f(R, TH, PH, s) for c in range(3)],
                                    grid, tt)
    source = lambda tt: sample(src, grid, tt)
    return Case("paper_mms", grid, par, dt, steps, K, bg, exact(0.0), exact, walls, source,
                info=dict(M0=M0, u0=u0, p0=p0, c0=c0))


# --------------------------------------------------------------- sector MMS

def sector_phases(seed: int = SECTOR_SEED):
    return np.random.default_rng(seed).uniform(0.0, 2 * math.pi, size=12)


def sector_grid(n=(32, 32, 32)) -> Grid:
    L = 1.0e4
    return Grid(n[0], n[1], n[2], 6371e3 / L, 6381e3 / L, math.pi / 4, 3 * math.pi / 4, 0.0, math.pi / 2)


SECTOR_PAR = dict(gamma=1.6, cv=1.0, Pr=1.0, mu=1.0)
SECTOR_P0 = 6250.0


def sector_mms_exprs(seed: int = SECTOR_SEED, M0: float = 1e-2):
    import sympy as sp
    from .continuous import r, th, ph, t
    a = [float(v) for v in sector_phases(seed)]
    g = sector_grid()
    p0, gamma, cv = SECTOR_P0, SECTOR_PAR["gamma"], SECTOR_PAR["cv"]
    c0 = math.sqrt(gamma * p0)
    u0 = M0 * c0
    xi = (r - g.r1) / (g.r2 - g.r1)
    eta = (th - g.t1) / (g.t2 - g.t1)
    zeta = (ph - g.p1) / (g.p2 - g.p1)
    S = lambda x: x ** 2 * (3 - 2 * x)          # S'(0) = S'(1) = 0: zero normal derivative
    pi = sp.pi
    p = p0 + u0 ** 2 * (1 + sp.sin(5 * t + a[0])
                        + sp.cos(pi * S(xi) + a[1]) * sp.cos(2 * pi * S(eta) + a[2]) * sp.cos(2 * pi * S(zeta) + a[3]))
    # solenoidal part: r-theta stream function psi and theta-phi stream function chi
    psi = (u0 / 2000.0) * r ** 2 * (1 + sp.sin(t + a[4]) / 2) * sp.sin(pi * xi) ** 2 * sp.sin(pi * eta) ** 2 \
        * sp.sin(pi * zeta) * (1 + sp.cos(2 * pi * S(eta) + a[5]) / 4)
    chi = (u0 / 3.0) * r * (1 + sp.cos(2 * t + a[6]) / 2) * sp.sin(pi * xi) * sp.sin(pi * eta) ** 2 \
        * sp.sin(pi * zeta) ** 2 * (1 + sp.cos(2 * pi * S(zeta) + a[7]) / 4)
    ur = sp.diff(psi, th) / (r ** 2 * sp.sin(th))
    ut = -sp.diff(psi, r) / (r * sp.sin(th)) + sp.diff(chi, ph) / (r * sp.sin(th))
    up = -sp.diff(chi, th) / r
    # O(u0 M0) compressible part, vanishing on every wall
    W = sp.sin(pi * xi) * sp.sin(pi * eta) * sp.sin(pi * zeta)
    q = u0 * u0 / c0
    ur = ur + q * (1 + sp.sin(4 * t + a[8]) / 2) * W
    ut = ut + q * (1 + sp.sin(t + a[9]) / 2) * W * sp.cos(2 * pi * xi + a[10])
    up = up + q * (1 + sp.cos(3 * t + a[11]) / 2) * W
    T = p / (cv * (gamma - 1))
    return [p, ur, ut, up, T]


def sector_mms(n=(32, 32, 32), seed: int = SECTOR_SEED, dt: float = 1e-3, steps: int = 10, K: int = 2,
               with_source: bool = True, use_sympy: bool = False) -> Case:
    grid = sector_grid(n)
    par = Params(**SECTOR_PAR)
    p0 = SECTOR_P0
    T0 = p0 / (par.cv * (par.gamma - 1))
    bg = _const_bg(grid, p0, T0)
    if seed == SECTOR_SEED and not use_sympy:
        # numpy code generated from the same sympy definitions (inputs/gen_sector_mms.py)
        from . import _sector_mms_generated as gen
        ex, src = gen.EXACT, (gen.SOURCE if with_source else None)
    else:
        exprs = sector_mms_exprs(seed)
        ex, src = _mms_callables(exprs, p0, T0, par, with_source=with_source)
    exact = lambda tt: sample(ex, grid, tt)
    source = (lambda tt: sample(src, grid, tt)) if src is not None else None
    return Case("sector_mms", grid, par, dt, steps, K, bg, exact(0.0), exact, None, source,
                info=dict(seed=seed, M0=1e-2))


# ------------------------------------------------------------------ bubble

AIR = dict(cp=1000.0, cv=713.0, R=287.0, Pr=0.71, mu=1.846e-5, g=9.80665)


def hydrostatic_background(grid: Grid, theta0: float = 300.0, p00: float = 1.0e5, cp: float = 1000.0,
                           cv: float = 713.0, g: float = 9.80665):
    """Radial background (nr+2 values incl. one ghost each side).

    T_ref = theta0 * Pi(h), Pi = 1 - g h / (cp theta0) (d pi0/dx = -g/(cp theta0),
    Section 3.2), and p_ref integrated upward so that the MAC momentum balance
    (p_i - p_{i-1})/dr = -g (rho_{i-1} + rho_i)/2 with rho = p/(R T) holds on
    every r-face: the rest state is then a discrete equilibrium."""
    Rg = cp - cv
    h = (np.arange(-1, grid.nr + 1) + 0.5) * grid.dr
    Pi = 1.0 - g * h / (cp * theta0)
    T = theta0 * Pi
    p = np.empty(grid.nr + 2)
    p[0] = p00 * Pi[0] ** (cp / Rg)
    a = g * grid.dr / (2.0 * Rg)
    for m in range(1, grid.nr + 2):
        p[m] = p[m - 1] * (1.0 - a / T[m - 1]) / (1.0 + a / T[m])
    return p, T, Pi


def bubble_grid(n=(128, 256, 256)) -> Grid:
    half = 10.0 / 6371.0
    return Grid(n[0], n[1], n[2], 6371e3, 6381e3, math.pi / 2 - half, math.pi / 2 + half,
                math.pi - half, math.pi + half)


def bubble_window(n=(128, 256, 256), width=(64, 64)) -> Grid:
    """The central width[0] x width[1] columns of the bubble sector, same cells."""
    g = bubble_grid(n)
    tm, pm = 0.5 * (g.t1 + g.t2), 0.5 * (g.p1 + g.p2)
    return Grid(g.nr, width[0], width[1], g.r1, g.r2, tm - 0.5 * width[0] * g.dth, tm + 0.5 * width[0] * g.dth,
                pm - 0.5 * width[1] * g.dph, pm + 0.5 * width[1] * g.dph)


def bubble(n=(128, 256, 256), seed: int = 1, dt: float = 1.0, steps: int = 200, K: int = 2,
           amplitude: float = 0.5, radius: float = 2000.0, altitude: float = 2000.0, mu: float = None,
           grid: Grid = None, profile: str = "gaussian", jitter: bool = True) -> Case:
    """Rising thermal bubble: dTheta = A f(L), L = |x - x_c| / R, centre at the
    given altitude above the domain centre.  profile "gaussian": f = exp(-L^2)
    (the benchmark workload; centre altitude and radius jittered by +-10 %,
    seeded); "cos2": f = cos^2(pi L / 2) for L <= 1 (Thermal 1, eq. temp_pert);
    "cos": f = (1 + cos(pi L)) / 2 for L <= 1 (Thermal 2).  grid: another grid
    (e.g. a central window of the sector) to sample the same initial state on."""
    grid = bubble_grid(n) if grid is None else grid
    rng = np.random.default_rng(seed)
    if jitter:
        radius = radius * (1.0 + rng.uniform(-0.1, 0.1))
        altitude = altitude * (1.0 + rng.uniform(-0.1, 0.1))
    par = Params(gamma=AIR["cp"] / AIR["cv"], cv=AIR["cv"], Pr=AIR["Pr"],
                 mu=AIR["mu"] if mu is None else mu, g=AIR["g"])
    bgp, bgT, Pi = hydrostatic_background(grid, cp=AIR["cp"], cv=AIR["cv"], g=AIR["g"])
    U = grid.zeros()
    R, TH, PH = grid.coords(0)
    tc, pc = 0.5 * (grid.t1 + grid.t2), 0.5 * (grid.p1 + grid.p2)
    rcen = grid.r1 + altitude
    x = R * np.sin(TH) * np.cos(PH) - rcen * math.sin(tc) * math.cos(pc)
    y = R * np.sin(TH) * np.sin(PH) - rcen * math.sin(tc) * math.sin(pc)
    z = R * np.cos(TH) - rcen * math.cos(tc)
    L2 = (x * x + y * y + z * z) / radius ** 2
    if profile == "gaussian":
        dtheta = amplitude * np.exp(-L2)
    elif profile == "cos2":
        L = np.sqrt(L2)
        dtheta = np.where(L <= 1.0, amplitude * np.cos(0.5 * math.pi * L) ** 2, 0.0)
    elif profile == "cos":
        L = np.sqrt(L2)
        dtheta = np.where(L <= 1.0, amplitude * 0.5 * (1.0 + np.cos(math.pi * L)), 0.0)
    else:
        raise ValueError(profile)
    Pic = Pi[1:-1][:, None, None]
    U[4] = np.ascontiguousarray(np.broadcast_to(Pic * dtheta, grid.shapes()[4]))
    return Case("bubble", grid, par, dt, steps, K, (bgp, bgT), U,
                info=dict(seed=seed, radius=radius, altitude=altitude, amplitude=amplitude))


def thermal1(n=(100, 200, 200), dt: float = 1.0, mu: float = None, K: int = 2) -> Case:
    """Section 3.2, Thermal 1: the 10 km x 20 km x 20 km sector, dTheta =
    2 cos^2(pi L / 2) for L <= 1 (L normalised by R = 2 km, reading R13), centre
    2 km above the bottom on the sector axis; dry air, t_end = 500 s."""
    c = bubble(n, dt=dt, K=K, amplitude=2.0, radius=2000.0, altitude=2000.0, mu=mu, profile="cos2", jitter=False)
    c.info["t_end"] = 500.0
    return c


def thermal2_grid(n=(200, 200, 200)) -> Grid:
    """Section 3.2, Thermal 2 domain: r in [6371, 6372] km (reading R14), theta
    and phi within 0.5 km / 6371 km of the equator and of phi = pi."""
    half = 0.5 / 6371.0
    return Grid(n[0], n[1], n[2], 6371e3, 6372e3, math.pi / 2 - half, math.pi / 2 + half,
                math.pi - half, math.pi + half)


def thermal2(n=(200, 200, 200), dt: float = 1.0, K: int = 2) -> Case:
    """Section 3.2, Thermal 2: the 1 km box, dTheta = (1 + cos(pi L)) / 4 for
    L <= 1, R = 250 m, centre 260 m above the bottom; t_end = 400 s."""
    g = thermal2_grid(n)
    c = bubble(n, dt=dt, K=K, amplitude=0.5, radius=250.0, altitude=260.0, profile="cos", jitter=False, grid=g)
    c.info["t_end"] = 400.0
    return c


ADJOINT_SEED = 4


def adjoint_bubble(n=(96, 192, 192), seed: int = ADJOINT_SEED, dt: float = 1.0, noise: float = 1e-3) -> Case:
    """The gradient workload: a Gaussian bubble (the benchmark's, seeded) on a
    96 x 192 x 192 sector plus white noise of 1e-3 K on the potential-temperature
    perturbation; 20 steps.  info: theta0 (the perturbation, cell centres) and
    Pi (the background Exner function at the centres, T' = Pi theta')."""
    c = bubble(n, seed=seed, dt=dt, steps=20)
    bgT = c.bg[1]
    Pi = (bgT[1:-1] / 300.0)[:, None, None]
    rng = np.random.default_rng(seed + 1000)
    theta0 = c.init[4] / Pi + noise * rng.standard_normal(c.grid.shapes()[4])
    c.init[4] = np.ascontiguousarray(Pi * theta0)
    c.info.update(theta0=theta0, Pi=np.ascontiguousarray(np.broadcast_to(Pi, c.grid.shapes()[4])))
    c.name = "adjoint_bubble"
    return c


ENSEMBLE_SEED = 20041389


def ensemble_specs(count: int = 64, seed: int = ENSEMBLE_SEED):
    """The batched ensemble: `count` independent bubbles on uneven grids of the
    same sector, nr uniform in {16, 32, 48, 64}, n_theta and n_phi uniform in
    {64, 128, 192, 256}, amplitude uniform in [0.2, 1] K, radius uniform in
    [1, 3] km; the per-instance seed drives the bubble's jitter."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = (int(rng.choice([16, 32, 48, 64])), int(rng.choice([64, 128, 192, 256])),
             int(rng.choice([64, 128, 192, 256])))
        out.append(dict(n=n, seed=int(rng.integers(1, 2 ** 31 - 1)), amplitude=float(rng.uniform(0.2, 1.0)),
                        radius=float(rng.uniform(1000.0, 3000.0))))
    return out


# ------------------------------------------------------------------ full sphere

SHELL_SEED = 20041390


def full_sphere_grid(n=(64, 512, 1024), r1: float = 6371e3, r2: float = 6381e3) -> Grid:
    """The whole sphere: theta in [0, pi] (pole faces), phi periodic."""
    return Grid(n[0], n[1], n[2], r1, r2, 0.0, math.pi, 0.0, 2 * math.pi, periodic=True)


def shell_low_mach(n=(64, 512, 1024), M0: float = 1e-4, seed: int = SHELL_SEED, dt: float = 1.0,
                   steps: int = 50, K: int = 2, grid: Grid = None) -> Case:
    """Full spherical shell of air at rest (p0 = 1e5 Pa, T0 = 300 K, no
    gravity) with a smooth random velocity of Mach number M0: amplitude
    M0 c0 times a sum of low spherical modes with seeded coefficients, plus
    1e-3 of that amplitude in smooth seeded noise.  u_r vanishes on the radial
    walls, u_theta and u_phi carry sin(theta), so the field is compatible with
    the walls and the poles; the thermodynamic state starts uniform."""
    grid = full_sphere_grid(n) if grid is None else grid
    rng = np.random.default_rng(seed)
    par = Params(gamma=AIR["cp"] / AIR["cv"], cv=AIR["cv"], Pr=AIR["Pr"], mu=AIR["mu"], g=0.0)
    p0, T0 = 1.0e5, 300.0
    c0 = math.sqrt(par.gamma * p0 / (p0 / (par.cv * (par.gamma - 1.0) * T0)))
    amp = M0 * c0
    coef = rng.standard_normal((3, 4, 4, 2))
    noise = rng.standard_normal((3, 8, 8, 2)) * 1e-3 / 8.0
    def field(c, R, TH, PH):
        xi = (R - grid.r1) / (grid.r2 - grid.r1)
        v = 0.0
        for m in range(4):
            for l in range(4):
                v = v + np.cos(TH) ** l * (coef[c, m, l, 0] * np.cos(m * PH) + coef[c, m, l, 1] * np.sin(m * PH))
        for m in range(8):
            for l in range(8):
                v = v + np.cos(TH) ** l * (noise[c, m, l, 0] * np.cos(m * PH) + noise[c, m, l, 1] * np.sin(m * PH))
        return amp * v * (np.sin(math.pi * xi) if c == 0 else np.sin(TH))
    U = grid.zeros()
    for c in range(3):
        R, TH, PH = grid.coords(1 + c)
        U[1 + c] = np.array(np.broadcast_to(field(c, R, TH, PH), grid.shapes()[1 + c]))
    U[1][0] = U[1][-1] = 0.0          # radial walls
    U[2][:, 0] = U[2][:, -1] = 0.0    # pole faces
    for c in (1, 2, 3):               # peak speed of each component = M0 c0
        U[c] *= amp / max(float(np.max(np.abs(U[c]))), 1e-300)
    bg = _const_bg(grid, p0, T0)
    return Case("shell_low_mach", grid, par, dt, steps, K, bg, U, info=dict(M0=M0, c0=c0, p0=p0, T0=T0))


def rest_state(grid: Grid, hydrostatic: bool = True) -> Case:
    """Air at rest over the discretely balanced background (no perturbation)."""
    par = Params(gamma=AIR["cp"] / AIR["cv"], cv=AIR["cv"], Pr=AIR["Pr"], mu=AIR["mu"],
                 g=AIR["g"] if hydrostatic else 0.0)
    if hydrostatic:
        bgp, bgT, _ = hydrostatic_background(grid, cp=AIR["cp"], cv=AIR["cv"], g=AIR["g"])
    else:
        bgp, bgT = _const_bg(grid, 1.0e5, 300.0)
    return Case("rest", grid, par, 1.0, 1, 2, (bgp, bgT), grid.zeros())
