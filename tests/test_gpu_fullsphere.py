"""The full sphere at full size (64 x 512 x 1024 cells, theta in [0, pi] with
pole faces, periodic phi: cyclic lines in every phi-sweep), air at rest with a
smooth random velocity at low Mach number: one FP64 step against the oracle
on the whole grid, the mixed mode against FP64 at M0 = 1e-4, 1e-5, 1e-6, and 50
mixed steps at the configuration's time step."""
import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from inputs import cases
from tests.gpu_helpers import solver_for, to_host

pytestmark = pytest.mark.gpu
N = (64, 512, 1024)


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()
    oracle.build()


def _run(c, prec, steps):
    s = solver_for(c.grid, c.par, c.bg, c.init, precision=prec)
    for _ in range(steps):
        s.step(c.dt, 2)
    out = to_host(s.get_state())
    s.close()
    return out


def test_full_sphere_step_vs_oracle():
    """One K = 2 step, every output compared.  Bound: 1e-12 of each field's
    natural scale -- the background value for p and T, the sound speed for the
    velocities (the scale of the acoustic terms whose rounding differs)."""
    c = cases.shell_low_mach(N, M0=1e-4)
    U = _run(c, sph.SPH_PREC_FP64, 1)
    Uo, _ = oracle.step(c.grid, c.par, c.init, c.dt, 2, bg=c.bg)
    c0 = c.info["c0"]
    scale = [c.info["p0"], c0, c0, c0, c.info["T0"]]
    for q in range(5):
        err = float(np.max(np.abs(U[q] - Uo[q])))
        assert err <= 1e-12 * scale[q], (q, err, scale[q])
    # the step did something on the cyclic lines and near the poles
    assert float(np.max(np.abs(U[0]))) > 0.0


@pytest.mark.parametrize("M0", [1e-4, 1e-5, 1e-6])
def test_full_sphere_mixed_low_mach(M0):
    """Mixed vs FP64 after 4 steps: the pressure fluctuation p - p0 (of order
    rho c0 M0 c0, 1e-8..1e-4 of p0) to 1e-2 of itself, and the velocity to
    1e-6 (relative L2)."""
    c = cases.shell_low_mach(N, M0=M0)
    U64 = _run(c, sph.SPH_PREC_FP64, 4)
    U32 = _run(c, sph.SPH_PREC_MIXED, 4)
    fl = float(np.max(np.abs(U64[0])))          # p' = p - p0 (constant background)
    err = float(np.max(np.abs(U32[0] - U64[0])))
    print(f"M0={M0}: max|p-p0|={fl:.3e} mixed error={err:.3e}")
    assert fl > 0 and err <= 1e-2 * fl, (fl, err)
    num = sum(float(np.linalg.norm(U32[q] - U64[q])) ** 2 for q in (1, 2, 3)) ** 0.5
    den = sum(float(np.linalg.norm(U64[q])) ** 2 for q in (1, 2, 3)) ** 0.5
    assert num <= 1e-6 * den, (num, den)


def test_full_sphere_fifty_steps():
    """50 mixed steps at dt = 1 s (acoustic Courant number ~3 in r and near the
    poles in phi): the state stays finite and the speed stays at the initial
    Mach number scale."""
    c = cases.shell_low_mach(N, M0=1e-4)
    s = solver_for(c.grid, c.par, c.bg, c.init, precision=sph.SPH_PREC_MIXED)
    for _ in range(50):
        s.step(c.dt, 2)
    U = to_host(s.get_state())
    s.close()
    assert all(np.all(np.isfinite(f)) for f in U)
    umax = max(float(np.max(np.abs(U[q]))) for q in (1, 2, 3))
    assert umax <= 3 * 1e-4 * c.info["c0"], umax
