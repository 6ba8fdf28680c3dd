"""Section 3.2's rising thermal bubbles, Thermal 1 (100 x 200 x 200 cells,
500 s) and Thermal 2 (200^3 cells, 400 s), in the mixed mode.  The paper shows
these as contour plots only, so there is nothing to compare numbers with; the
tests check the qualitative statements it makes about them:

Thermal 1: viscosity up to 1.846e-2 kg/(m s) hardly changes the solution, 1.846e1
smooths it; tau = 0.2 s and 1 s agree; tau = 50 s with K = 2 changes it
dramatically and slows the bubble, K = 50 compensates in part.
Thermal 2: tau = 1 s with K = 2 is smoother than tau = 0.25 s; K = 10 removes
much of that difference (the splitting error).

Measures: theta' = T (p00/p)^(R/cp) - 300 K; relative L2 differences of theta'
fields; the altitude of theta'-weighted centroid of the warm anomaly; the L2
norm of the grid gradient of theta' (smoothness)."""
import numpy as np
import pytest

import paper_2004_13887_gb300 as sph
from inputs import cases
from tests.gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()


def theta_prime(U, c):
    bgp, bgT = c.bg
    p = U[0] + bgp[1:-1][:, None, None]
    T = U[4] + bgT[1:-1][:, None, None]
    Rg = c.par.cv * (c.par.gamma - 1.0)
    return T * (1e5 / p) ** (Rg / (c.par.gamma * c.par.cv)) - 300.0


def run(c, dt, K):
    s = sph.Solver(c.grid, c.par, precision=sph.SPH_PREC_MIXED)
    s.set_background(*c.bg)
    s.set_state(to_dev(c.init))
    for _ in range(int(round(c.info["t_end"] / dt))):
        s.step(dt, K)
    U = to_host(s.get_state())
    s.close()
    assert all(np.all(np.isfinite(f)) for f in U)
    th = theta_prime(U, c)
    w = np.clip(th, 0.0, None)
    z = c.grid.rc()[:, None, None] - c.grid.r1
    cen = float((w * z).sum() / w.sum())
    grad = float(sum(np.linalg.norm(g) for g in np.gradient(th)))
    return th, cen, grad


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_thermal1_qualitative_claims():
    n = (100, 200, 200)
    c0 = cases.thermal1(n)
    th0 = theta_prime(c0.init, c0)
    cen0 = float((np.clip(th0, 0, None) * (c0.grid.rc()[:, None, None] - c0.grid.r1)).sum() / np.clip(th0, 0, None).sum())
    base, cen_b, _ = run(cases.thermal1(n, dt=1.0), 1.0, 2)
    assert cen_b > cen0 + 1500.0                                  # the bubble rises
    small_tau, _, _ = run(cases.thermal1(n, dt=0.2), 0.2, 2)
    assert rel(small_tau, base) < 0.1                             # tau 0.2 s ~ tau 1 s
    mu2, _, _ = run(cases.thermal1(n, mu=1.846e-2), 1.0, 2)
    assert rel(mu2, base) < 0.01                                  # 1e3 x air viscosity: no effect
    mu1, _, _ = run(cases.thermal1(n, mu=1.846e1), 1.0, 2)
    assert rel(mu1, base) > 10 * rel(mu2, base) and mu1.max() < base.max()   # 1e6 x: smoothing
    big2, cen2, _ = run(cases.thermal1(n, dt=50.0), 50.0, 2)
    assert rel(big2, base) > 0.5 and cen2 < cen_b - 1000.0         # tau 50 s, K = 2: dramatic, slower
    big50, cen50, _ = run(cases.thermal1(n, dt=50.0, K=50), 50.0, 50)
    assert rel(big50, base) < rel(big2, base) and cen2 < cen50 < cen_b   # K = 50 compensates in part
    assert rel(big50, base) > 0.2                                 # ... but stays different


def test_thermal2_qualitative_claims():
    n = (200, 200, 200)
    fine, _, g_fine = run(cases.thermal2(n, dt=0.25), 0.25, 2)
    k2, _, g_k2 = run(cases.thermal2(n, dt=1.0), 1.0, 2)
    k10, _, g_k10 = run(cases.thermal2(n, dt=1.0, K=10), 1.0, 10)
    assert g_k2 < 0.8 * g_fine and k2.max() < fine.max()          # larger step: smoother
    assert rel(k10, fine) < 0.6 * rel(k2, fine)                   # more iterations: much of it back
    assert g_k10 > g_k2
