"""Pins of the oracle's time stepping (Section 2.2, eqs. chapter3mainsd,
splitting1, splitting2, spl1-spl3).

* Fixed point: when the Picard/splitting-error iteration converges, U^{n+1}
  solves the Crank-Nicolson (implicit-midpoint) system
  U^{n+1} - U^n + tau [(D + D_M)(Ubar) Ubar + G - S] = 0, Ubar = (U^{n+1}+U^n)/2.
* K = 1 is the Douglas scheme: the three sweeps invert the factorised operator
  (I + tau/2 D_r)(I + tau/2 D_theta)(I + tau/2 D_phi) of eq. (splitting1).
* Rest states are discrete equilibria; mirror symmetry and periodic shifts are
  preserved.
"""
import math

import numpy as np
import pytest

import oracle
from inputs import Grid, Params, cases


def full_operator(g, par, Ubar, V, bg=None, ubar_walls=None, v_walls=None, v_bg=None):
    tot = [np.zeros(s) for s in g.shapes()]
    for which in range(4):
        out = oracle.apply_op(g, par, Ubar, which, V, bg=bg, ubar_walls=ubar_walls, v_bg=v_bg,
                              v_walls=v_walls)
        for q in range(5):
            tot[q] += out[q]
    return tot


def unknown_mask(g):
    m = [np.ones(s, bool) for s in g.shapes()]
    m[1][0] = m[1][-1] = False
    m[2][:, 0] = m[2][:, -1] = False
    if not g.periodic:
        m[3][:, :, 0] = m[3][:, :, -1] = False
    return m


def test_fixed_point_is_implicit_midpoint():
    c = cases.sector_mms((10, 12, 14))
    g, par = c.grid, c.par
    S = c.source(0.5 * c.dt)
    U1, res = oracle.step(g, par, c.init, c.dt, 30, bg=c.bg, S=S)
    assert np.all(res < 1e-11)
    Ub = [0.5 * (a + b) for a, b in zip(U1, c.init)]
    N = full_operator(g, par, Ub, Ub, bg=c.bg, v_bg=c.bg)
    mask = unknown_mask(g)
    for q in range(5):
        G = par.g if q == 1 else 0.0
        resid = U1[q] - c.init[q] + c.dt * (N[q] + G - S[q])
        scale = np.max(np.abs(U1[q] - c.init[q]))
        assert np.max(np.abs(resid[mask[q]])) <= 1e-9 * scale, q


def test_fixed_point_with_time_dependent_walls():
    """Paper MMS: inhomogeneous, time-dependent Dirichlet velocity on every wall."""
    pytest.importorskip("sympy")
    c = cases.paper_mms(1e-2, n=(6, 7, 9))
    g, par = c.grid, c.par
    tau = c.dt
    wn, wk = c.walls(0.0), c.walls(tau)
    S = c.source(0.5 * tau)
    U1, res = oracle.step(g, par, c.init, tau, 30, bg=c.bg, walls_n=wn, walls_np1=wk, S=S)
    assert np.all(res < 1e-10)
    Ub = [0.5 * (a + b) for a, b in zip(U1, c.init)]
    wb = {key: 0.5 * (wn[key] + wk[key]) for key in wn}
    N = full_operator(g, par, Ub, Ub, bg=c.bg, ubar_walls=wb, v_walls=wb, v_bg=c.bg)
    mask = unknown_mask(g)
    for q in range(5):
        resid = U1[q] - c.init[q] + tau * (N[q] - S[q])
        scale = np.max(np.abs(U1[q] - c.init[q]))
        assert np.max(np.abs(resid[mask[q]])) <= 1e-9 * scale, q
    # the normal wall velocity of U^{n+1} is the t^{n+1} data
    assert np.array_equal(U1[1][0], wk[(0, 0, 0)]) and np.array_equal(U1[1][-1], wk[(0, 0, 1)])


@pytest.mark.parametrize("periodic", [False, True])
def test_single_iteration_is_douglas_factorisation(periodic):
    """K = 1: (I+tau/2 D_r)(I+tau/2 D_th)(I+tau/2 D_ph)(U^1 - U^n) = -tau (D + D_M)(U^n) U^n - tau G + tau S."""
    if periodic:
        g = Grid(6, 7, 9, 1.0, 2.0, 0.5, 2.6, 0.0, 2 * np.pi, periodic=True)
    else:
        g = Grid(6, 7, 9, 1.0, 2.0, np.pi / 4, 3 * np.pi / 4, np.pi / 4, 7 * np.pi / 4)
    par = Params(gamma=1.6, cv=1.0, Pr=1.0, mu=0.3, omega=0.2, g=0.5, pinf=3.0)
    rng = np.random.default_rng(9)
    U = [0.3 * rng.standard_normal(s) for s in g.shapes()]
    U[1][0] = U[1][-1] = 0
    U[2][:, 0] = U[2][:, -1] = 0
    if not periodic:
        U[3][:, :, 0] = U[3][:, :, -1] = 0
    U[0] += 50.0
    U[4] += 80.0
    S = [0.1 * rng.standard_normal(s) for s in g.shapes()]
    tau = 0.02
    U1, _ = oracle.step(g, par, U, tau, 1, S=S)
    delta = [a - b for a, b in zip(U1, U)]
    # apply the three factors right to left with coefficients at U^n
    v = delta
    for d in (2, 1, 0):
        Dv = oracle.apply_op(g, par, U, d, v)
        v = [a + 0.5 * tau * b for a, b in zip(v, Dv)]
    N = full_operator(g, par, U, U)
    mask = unknown_mask(g)
    for q in range(5):
        G = par.g if q == 1 else 0.0
        rhs = -tau * (N[q] + G - S[q])
        assert np.max(np.abs((v[q] - rhs)[mask[q]])) <= 1e-11 * np.max(np.abs(rhs[mask[q]])), q


def test_rest_state_uniform_is_exact():
    g = Grid(5, 6, 7, 1.0, 2.0, 0.7, 2.2, 0.1, 1.9)
    par = Params(gamma=1.4, cv=713.0, Pr=0.71, mu=1e-3)
    U = g.zeros()
    U[0][:] = 1e5
    U[4][:] = 300.0
    U1, res = oracle.step(g, par, U, 0.5, 2)
    # exact in exact arithmetic; the flux stencils of a constant cancel to rounding
    assert np.max(np.abs(U1[0] - U[0])) <= 1e-14 * 1e5
    assert np.max(np.abs(U1[4] - U[4])) <= 1e-14 * 300.0
    for q in (1, 2, 3):
        assert np.max(np.abs(U1[q])) <= 1e-15


@pytest.mark.parametrize("mu", [0.0, 1.846e-5])
def test_hydrostatic_rest_state_stays_at_rest(mu):
    """Discretely balanced background (hydrostatic, Section 3.2): the rest state
    is an equilibrium; with mu > 0 only the conduction of the background
    temperature profile is left, far below the bubble's signal."""
    c = cases.rest_state(cases.bubble_grid((8, 8, 8)))
    c.par.mu = mu
    U = c.init
    for _ in range(3):
        U, res = oracle.step(c.grid, c.par, U, 1.0, 2, bg=c.bg)
    umax = max(np.max(np.abs(U[q])) for q in (1, 2, 3))
    assert umax <= (1e-12 if mu == 0 else 1e-9), umax
    assert np.max(np.abs(U[0])) <= (1e-7 if mu == 0 else 1e-5)


def test_bubble_mirror_symmetry():
    """Bubble centred on the sector axis, no rotation: mirror symmetric in theta and phi."""
    c = cases.bubble((8, 10, 12), seed=3, dt=1.0)
    U = c.init
    for _ in range(3):
        U, _ = oracle.step(c.grid, c.par, U, c.dt, 2, bg=c.bg)
    p, ur, ut, up, T = U
    for name, f, sgn_t, sgn_p in (("p", p, 1, 1), ("ur", ur, 1, 1), ("T", T, 1, 1),
                                  ("ut", ut, -1, 1), ("up", up, 1, -1)):
        s = np.max(np.abs(f)) + 1e-300
        assert np.max(np.abs(f - sgn_t * f[:, ::-1, :])) <= 1e-12 * s, name
        assert np.max(np.abs(f - sgn_p * f[:, :, ::-1])) <= 1e-12 * s, name
    assert np.max(np.abs(ur)) > 1e-6   # the bubble did start to rise


def test_periodic_shift_equivariance():
    g = Grid(6, 8, 12, 1.0, 1.5, 0.4, 2.7, 0.0, 2 * math.pi, periodic=True)
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.02)
    rng = np.random.default_rng(21)
    U = [0.05 * rng.standard_normal(s) for s in g.shapes()]
    U[1][0] = U[1][-1] = 0
    U[2][:, 0] = U[2][:, -1] = 0
    U[0] += 10.0
    U[4] += 20.0
    A, _ = oracle.step(g, par, U, 0.01, 2)
    B, _ = oracle.step(g, par, [np.roll(f, 1, axis=2) for f in U], 0.01, 2)
    for q in range(5):
        s = np.max(np.abs(A[q] - U[q]))
        assert np.max(np.abs(np.roll(A[q], 1, axis=2) - B[q])) <= 1e-12 * max(s, 1e-300) + 1e-14 * np.max(np.abs(A[q]))
    # phi-independent data stay phi-independent
    V = [np.repeat(f[:, :, :1], g.np, axis=2) for f in U]
    C, _ = oracle.step(g, par, V, 0.01, 2)
    for q in range(5):
        assert np.max(np.abs(C[q] - C[q][:, :, :1])) <= 1e-12 * (np.max(np.abs(C[q])) + 1e-300)


def _closed_box_flow(n):
    """A sourceless flow in a closed sector: no-slip walls with zero normal
    velocity, smooth velocity and pressure perturbations (paper's constants of
    Section 3.1, mu = 0.05)."""
    from inputs import Grid, Params
    par = Params(gamma=1.6, cv=1.0, Pr=1.0, mu=0.05)
    p0 = 6250.0
    T0 = p0 / (par.cv * (par.gamma - 1))
    g = Grid(n, n, n, 1.0, 2.0, np.pi / 4, 3 * np.pi / 4, np.pi / 4, 7 * np.pi / 4)
    U = g.zeros()
    for f in (1, 2, 3):
        R, TH, PH = g.coords(f)
        xi, et, ze = (R - g.r1) / (g.r2 - g.r1), (TH - g.t1) / (g.t2 - g.t1), (PH - g.p1) / (g.p2 - g.p1)
        U[f][:] = 5.0 * np.sin(np.pi * xi) * np.sin(np.pi * et) * np.sin(np.pi * ze) * (
            1 + 0.5 * np.cos(2 * np.pi * (xi + 0.3 * f)) * np.sin(np.pi * (et + ze)))
    U[1][0] = U[1][-1] = 0
    U[2][:, 0] = U[2][:, -1] = 0
    U[3][:, :, 0] = U[3][:, :, -1] = 0
    R, TH, PH = g.coords(0)
    xi, et, ze = (R - g.r1) / (g.r2 - g.r1), (TH - g.t1) / (g.t2 - g.t1), (PH - g.p1) / (g.p2 - g.p1)
    U[0][:] = 20 * np.cos(np.pi * xi) * np.cos(np.pi * et) * np.cos(np.pi * ze)
    bg = (np.full(n + 2, p0), np.full(n + 2, T0))
    return g, par, bg, U, p0, T0


def _mass(g, par, U, p0, T0):
    """sum of rho (eq. nonconserveos) times the exact cell volumes"""
    rf, tf = g.rf(), g.tf()
    V = ((rf[1:] ** 3 - rf[:-1] ** 3) / 3)[:, None, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :, None] * g.dph
    rho = (p0 + U[0]) / (par.cv * (par.gamma - 1) * (T0 + U[4]))
    return float(np.sum(rho * V))


def test_mass_drift_falls_at_second_order():
    """The scheme evolves p and T, not rho (the T-equation replaces the mass
    equation, Section 2.1 and Appendix A), so the total mass of a closed,
    sourceless flow -- exactly conserved by the continuous problem -- is not a
    discrete invariant: it drifts, and the drift is a discretisation error that
    falls at second order under refinement (tau small enough that the O(tau^2)
    part does not mask it)."""
    tau, steps = 1.25e-4, 80
    drift = []
    for n in (8, 16, 32):
        g, par, bg, U, p0, T0 = _closed_box_flow(n)
        m0 = _mass(g, par, U, p0, T0)
        for _ in range(steps):
            U, _ = oracle.step(g, par, U, tau, 2, bg=bg)
        drift.append(abs(_mass(g, par, U, p0, T0) - m0) / m0)
    drift = np.array(drift)
    rates = np.log2(drift[:-1] / drift[1:])
    assert drift[0] > 1e-8, drift           # not conserved to round-off: a non-conservative scheme
    assert np.all(rates >= 1.8), (drift, rates)
