"""Mixed precision (SPH_PREC_MIXED: FP32 stencils and line solves, FP64 state,
update, divergence and cyclic corrections) against the FP64 oracle and the
FP64 library path.

The sweeps of the mixed mode take the partitioned line solver (one warp per
line, chunk elimination + parallel cyclic reduction across the lanes) for
lines of 64, 128 or 256 cells and the thread-per-line block Thomas solver
otherwise; both are checked here.

Bounds:
* each FP32 line solve: 1e-5 relative (max norm per field) against the oracle;
* the right-hand side: 1e-5 relative per field against the oracle, plus the
  oracle's own evaluation-order noise;
* whole steps: the relative L2 error of the physical fields -- pressure p,
  density rho, potential temperature theta, temperature T and velocity u -- is
  at most 1e-6 against the FP64 path (the error statement of the mixed mode).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from inputs import cases
from tests.gpu_helpers import perturbed, rel_err, solver_for, to_dev, to_host
from tests.test_gpu_parity import CASES, _bubble, _sector, _shell, rhs_midpoint

pytestmark = pytest.mark.gpu
MIXED = sph.SPH_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()
    oracle.build()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("d", [0, 1, 2])
def test_mixed_sweep_vs_oracle(name, d):
    g, par, bg, Un, Uk, S, dt = CASES[name]()
    s = solver_for(g, par, bg, Un, precision=MIXED)
    s.set_iterate(Uk)
    rhs = perturbed(g.zeros(), [1.0] * 5, 20 + d, g)
    x = to_host(s.sweep(d, dt, to_dev(rhs)))
    ref = oracle.sweep(g, par, Un, Uk, dt, d, rhs, bg=bg)
    for q in range(5):
        assert rel_err(x[q], ref[q]) <= 1e-5, (name, d, q, rel_err(x[q], ref[q]))


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_rhs_vs_oracle(name):
    g, par, bg, Un, Uk, S, dt = CASES[name]()
    s = solver_for(g, par, bg, Un, precision=MIXED)
    s.set_iterate(Uk)
    R = to_host(s.rhs(dt, S))
    ref = oracle.rhs(g, par, Un, Uk, dt, bg=bg, S=S)
    mid = rhs_midpoint(g, par, bg, Un, Uk, dt, S)
    for q in range(5):
        noise = float(np.max(np.abs(mid[q] - ref[q])))
        err = float(np.max(np.abs(R[q] - ref[q])))
        assert err <= 1e-5 * float(np.max(np.abs(ref[q]))) + 2 * noise, (name, q, err)


def physical_fields(U, bg, par):
    """p, rho, theta, T and |u| components from a state (perturbations + background)."""
    p = U[0] + bg[0][1:-1][:, None, None]
    T = U[4] + bg[1][1:-1][:, None, None]
    Rg = par.cv * (par.gamma - 1.0)
    rho = (p + par.pinf) / (Rg * T)
    cp = par.gamma * par.cv
    p00 = float(bg[0][1]) if float(bg[0][1]) > 0 else 1.0
    theta = T * (p00 / p) ** (Rg / cp)
    return {"p": p, "rho": rho, "theta": theta, "T": T, "ur": U[1], "ut": U[2], "up": U[3]}


def l2_rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def velocity_l2(A, B):
    num = sum(np.linalg.norm(A[k] - B[k]) ** 2 for k in ("ur", "ut", "up"))
    den = sum(np.linalg.norm(B[k]) ** 2 for k in ("ur", "ut", "up"))
    return math.sqrt(num / max(den, 1e-300))


def run_both(case, nsteps, K=2, source=None):
    s64 = solver_for(case.grid, case.par, case.bg, case.init)
    s32 = solver_for(case.grid, case.par, case.bg, case.init, precision=MIXED)
    for n in range(nsteps):
        S = source((n + 0.5) * case.dt) if source else None
        s64.step(case.dt, K, S)
        s32.step(case.dt, K, S)
    return to_host(s64.get_state()), to_host(s32.get_state())


def test_mixed_steps_bubble_small():
    c = cases.bubble((24, 32, 32), seed=1, dt=1.0)
    U64, U32 = run_both(c, 10)
    A, B = physical_fields(U32, c.bg, c.par), physical_fields(U64, c.bg, c.par)
    for k in ("p", "rho", "theta", "T"):
        assert l2_rel(A[k], B[k]) <= 1e-6, (k, l2_rel(A[k], B[k]))
    assert velocity_l2(A, B) <= 1e-6, velocity_l2(A, B)


def test_mixed_steps_sector_mms():
    c = cases.sector_mms((32, 32, 32))
    U64, U32 = run_both(c, 10, source=c.source)
    A, B = physical_fields(U32, c.bg, c.par), physical_fields(U64, c.bg, c.par)
    for k in ("p", "rho", "T"):
        assert l2_rel(A[k], B[k]) <= 1e-6, (k, l2_rel(A[k], B[k]))
    assert velocity_l2(A, B) <= 1e-6, velocity_l2(A, B)


def test_mixed_steps_full_size_bubble():
    """The benchmark workload, 20 steps: mixed vs FP64 per physical field."""
    c = cases.bubble((128, 256, 256), seed=1, dt=1.0)
    U64, U32 = run_both(c, 20)
    A, B = physical_fields(U32, c.bg, c.par), physical_fields(U64, c.bg, c.par)
    errs = {k: l2_rel(A[k], B[k]) for k in ("p", "rho", "theta", "T")}
    errs["u"] = velocity_l2(A, B)
    print("mixed vs fp64, 20 steps:", errs)
    for k, v in errs.items():
        assert v <= 1e-6, (k, v)


def test_mixed_steps_full_size_200():
    """The benchmark workload for the 200 steps it is defined with: mixed vs
    FP64 per physical field (relative L2) stays within 1e-6."""
    c = cases.bubble((128, 256, 256), seed=1, dt=1.0)
    U64, U32 = run_both(c, 200)
    A, B = physical_fields(U32, c.bg, c.par), physical_fields(U64, c.bg, c.par)
    errs = {k: l2_rel(A[k], B[k]) for k in ("p", "rho", "theta", "T")}
    errs["u"] = velocity_l2(A, B)
    print("mixed vs fp64, 200 steps:", errs)
    for k, v in errs.items():
        assert v <= 1e-6, (k, v)


# Line lengths 64 to 1024 in every direction (16 lanes per line with chunks
# of 4 and 8 cells, 32 lanes with chunks of 8), periodic and walled phi, a
# pole, directions of other lengths (block Thomas) next to partitioned ones,
# and line counts that leave the last group of a launch partly empty (r lines
# of 64, 128 and 256 cells in groups of 16, 8 and 8; theta lines of 256 in
# groups of 8; cyclic phi lines of 128 in groups of 8).  Phi lines of 512 and
# 1024 cells span 2 and 4 warps (walled and cyclic, with partial groups of 4
# lines); r and theta lines of 512 and 1024 take block Thomas.  Lines of 16,
# 32, 48 and 192 cells (chunks of 1, 2, 3 on 16 lanes and of 6 on 32; walled
# and cyclic, partial groups of 32 and 8 lines) are the short and mid lengths
# of uneven ensembles.
PART_CASES = {
    "bubble_64x64x128": lambda: _bubble((64, 64, 128)),
    "shell_64x128x256": lambda: _shell((64, 128, 256), pole=False),
    "shell_pole_128x64x64": lambda: _shell((128, 64, 64), pole=True),
    "sector_40x256x64": lambda: _sector((40, 256, 64)),
    "sector_64x36x100": lambda: _sector((64, 36, 100)),
    "bubble_128x24x20": lambda: _bubble((128, 24, 20)),
    "shell_40x36x128": lambda: _shell((40, 36, 128), pole=False),
    "sector_40x256x20": lambda: _sector((40, 256, 20)),
    "bubble_256x20x12": lambda: _bubble((256, 20, 12)),
    "shell_16x512x1024": lambda: _shell((16, 512, 1024), pole=False),
    "sector_16x1024x41": lambda: _sector((16, 1024, 41)),
    "bubble_16x38x512": lambda: _bubble((16, 38, 512)),
    "shell_16x66x512": lambda: _shell((16, 66, 512), pole=False),
    "sector_16x48x192": lambda: _sector((16, 48, 192)),
    "shell_32x20x192": lambda: _shell((32, 20, 192), pole=False),
    "bubble_48x36x16": lambda: _bubble((48, 36, 16)),
    "shell_16x40x16": lambda: _shell((16, 40, 16), pole=False),
    "sector_512x8x13": lambda: _sector((512, 8, 13)),
}


@pytest.mark.parametrize("name", list(PART_CASES))
@pytest.mark.parametrize("d", [0, 1, 2])
def test_partitioned_sweep_vs_oracle(name, d):
    g, par, bg, Un, Uk, S, dt = PART_CASES[name]()
    s = solver_for(g, par, bg, Un, precision=MIXED)
    s.set_iterate(Uk)
    rhs = perturbed(g.zeros(), [1.0] * 5, 30 + d, g)
    x = to_host(s.sweep(d, dt, to_dev(rhs)))
    ref = oracle.sweep(g, par, Un, Uk, dt, d, rhs, bg=bg)
    for q in range(5):
        assert rel_err(x[q], ref[q]) <= 1e-5, (name, d, q, rel_err(x[q], ref[q]))


# The narrow layout (4 lanes with chunks of 4 for lines of 16 cells, 8 lanes
# with chunks of 4, 6 and 8 for 32, 48 and 64): walled and cyclic lines of
# each length, along every direction, and line counts that leave the last
# group of a launch partly empty (32 lines a group for 16 and 32 cells, 16
# for 48 and 64).
NARROW_CASES = ["shell_16x40x16", "bubble_48x36x16", "sector_16x48x192", "shell_32x20x192", "bubble_64x64x128",
                "sector_40x256x64", "sector_16x1024x41", "shell_64x36x48", "sector_32x32x33"]
PART_CASES["shell_64x36x48"] = lambda: _shell((64, 36, 48), pole=False)
PART_CASES["sector_32x32x33"] = lambda: _sector((32, 32, 33))


@pytest.mark.parametrize("name", NARROW_CASES)
@pytest.mark.parametrize("d", [0, 1, 2])
def test_narrow_sweep_vs_oracle(name, d):
    g, par, bg, Un, Uk, S, dt = PART_CASES[name]()
    s = solver_for(g, par, bg, Un, precision=MIXED)
    s.set_line_solver(sph.SPH_LINES_PARTITIONED_NARROW)
    s.set_iterate(Uk)
    rhs = perturbed(g.zeros(), [1.0] * 5, 60 + d, g)
    x = to_host(s.sweep(d, dt, to_dev(rhs)))
    ref = oracle.sweep(g, par, Un, Uk, dt, d, rhs, bg=bg)
    for q in range(5):
        assert rel_err(x[q], ref[q]) <= 1e-5, (name, d, q, rel_err(x[q], ref[q]))


def test_line_solver_option():
    g, par, bg, Un, Uk, S, dt = PART_CASES["shell_64x128x256"]()
    s = solver_for(g, par, bg, Un, precision=MIXED)
    with pytest.raises(sph.SphError):
        s.set_line_solver(7)
    s.set_iterate(Uk)
    rhs = to_dev(perturbed(g.zeros(), [1.0] * 5, 40, g))
    for d in range(3):
        xp = to_host(s.sweep(d, dt, rhs))
        s.set_line_solver(sph.SPH_LINES_PARTITIONED_WARP)
        xw = to_host(s.sweep(d, dt, rhs))
        s.set_line_solver(sph.SPH_LINES_PARTITIONED_NARROW)
        xn = to_host(s.sweep(d, dt, rhs))
        s.set_line_solver(sph.SPH_LINES_THOMAS)
        xt = to_host(s.sweep(d, dt, rhs))
        s.set_line_solver(sph.SPH_LINES_PARTITIONED)
        for q in range(5):
            assert rel_err(xp[q], xt[q]) <= 1e-5, (d, q, rel_err(xp[q], xt[q]))
            assert rel_err(xw[q], xt[q]) <= 1e-5, (d, q, rel_err(xw[q], xt[q]))
            assert rel_err(xn[q], xt[q]) <= 1e-5, (d, q, rel_err(xn[q], xt[q]))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_partitioned_sweep_full_size(d):
    """The benchmark grid (128 x 256 x 256: chunks of 4, 8, 8): the mixed sweep
    against the FP64 library sweep on the same inputs, every point."""
    c = cases.bubble((128, 256, 256), seed=1, dt=1.0)
    it = perturbed(c.init, [5.0, 1e-2, 1e-2, 1e-2, 1e-2], 9, c.grid)
    rhs = to_dev(perturbed(c.grid.zeros(), [1.0] * 5, 50 + d, c.grid))
    xs = []
    for prec in (sph.SPH_PREC_FP64, MIXED):
        s = solver_for(c.grid, c.par, c.bg, c.init, precision=prec)
        s.set_iterate(it)
        xs.append(to_host(s.sweep(d, c.dt, rhs)))
        s.close()
    for q in range(5):
        assert rel_err(xs[1][q], xs[0][q]) <= 1e-5, (d, q, rel_err(xs[1][q], xs[0][q]))


def test_partitioned_steps_cyclic():
    """Whole steps on a periodic shell: partitioned vs Thomas vs FP64."""
    g, par, bg, Un, Uk, S, dt = PART_CASES["shell_64x128x256"]()
    outs = []
    for prec, which in ((sph.SPH_PREC_FP64, None), (MIXED, sph.SPH_LINES_THOMAS), (MIXED, sph.SPH_LINES_PARTITIONED),
                        (MIXED, sph.SPH_LINES_PARTITIONED_WARP), (MIXED, sph.SPH_LINES_PARTITIONED_NARROW)):
        s = solver_for(g, par, bg, Un, precision=prec)
        if which is not None:
            s.set_line_solver(which)
        for _ in range(5):
            s.step(dt, 2, S)
        outs.append(to_host(s.get_state()))
        s.close()
    for q in range(5):
        scale = float(np.max(np.abs(outs[0][q] - Un[q]))) or 1.0
        for o in outs[1:]:
            err = float(np.max(np.abs(o[q] - outs[0][q])))
            assert err <= 1e-5 * scale, (q, err, scale)


def test_mixed_low_mach_pressure_fluctuation():
    """Low Mach number (M0 ~ 1e-4, p - p0 ~ 1e-4 on p0 = 6250, far below the
    FP32 resolution of p itself): the mixed path must follow the FP64 pressure
    fluctuation, which needs the FP64 state, p stored as a perturbation and
    div(Ubar) formed without FP32 cancellation.  Initial data: the wall-
    compatible sector field, velocities scaled by 1e-2 and the thermodynamic
    perturbations by 1e-4 (Mach number 1e-2 -> 1e-4); no source."""
    c = cases.sector_mms((32, 32, 64))
    U0 = [f.copy() for f in c.init]
    U0[0] *= 1e-4
    U0[4] *= 1e-4
    for q in (1, 2, 3):
        U0[q] *= 1e-2
    outs = []
    for prec in (sph.SPH_PREC_FP64, MIXED):
        s_ = solver_for(c.grid, c.par, c.bg, U0, precision=prec)
        for _ in range(10):
            s_.step(c.dt, 2)
        outs.append(to_host(s_.get_state()))
        s_.close()
    U64, U32 = outs
    p0 = float(c.bg[0][1])
    A, B = physical_fields(U32, c.bg, c.par), physical_fields(U64, c.bg, c.par)
    fluct = float(np.max(np.abs(B["p"] - p0)))
    err = float(np.max(np.abs(A["p"] - B["p"])))
    print("low-Mach p - p0:", fluct, "mixed error:", err)
    assert 0 < fluct < 1e-3
    assert err <= 1e-2 * fluct, (err, fluct)
