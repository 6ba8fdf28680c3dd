"""The step adjoint (sph_step_adjoint) and the gradient through time stepping.

* Central finite differences of the library's own FP64 steps along 8 seeded
  directions (step eps = 1e-4 of each field's scale) against <dJ/dU0, v> from
  the adjoint, J a seeded linear functional of U^N after two steps, on a
  walled sector with gravity and a radial background, a periodic shell, a
  shell with both poles and the sector manufactured solution with its source:
  relative difference <= 1e-4 (the bound the gradient is stated to).
* J^T lambda of one step against the transpose of the oracle's
  finite-difference Jacobian (4 x 5 x 6 cells), the oracle-side adjoint.
* The autograd Function with sqrt(N) checkpointing: the gradient of the final
  kinetic energy with respect to the initial potential-temperature perturbation
  of a small bubble (Gaussian plus 1e-3 white noise), against central
  differences along 8 seeded directions.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from inputs import Grid, Params, cases
from tests.adjoint_helpers import field_scales, flat, generic_state, oracle_jacobian, small_cases, unflat
from tests.gpu_helpers import solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()
    oracle.build()


def _run(s, U0, dt, K, n, S):
    s.set_state(to_dev(U0))
    for _ in range(n):
        s.step(dt, K, S)
    return to_host(s.get_state())


def _adjoint(s, U0, dt, K, n, S, lam):
    """dJ/dU0 from dJ/dU^n = lam through n steps (states kept, walked backwards)"""
    states = [to_dev(U0)]
    s.set_state(states[0])
    for _ in range(n - 1):
        s.step(dt, K, S)
        states.append([f.clone() for f in s.get_state()])
    lam_d = to_dev(lam)
    for st in reversed(states):
        s.set_state(st)
        lam_d = s.step_adjoint(dt, K, lam_d, source=S)
    return to_host(lam_d)


@pytest.mark.parametrize("name", ["bubble", "shell", "shell_pole", "sector_mms"])
def test_adjoint_vs_central_differences(name):
    g, par, bg, U0, S, dt = small_cases()[name]
    K, nsteps = 2, 2
    s = solver_for(g, par, bg)
    Sd = to_dev(S) if S is not None else None
    rng = np.random.default_rng(40)
    w = [rng.standard_normal(sh) for sh in g.shapes()]           # J(U) = <w, U>
    J = lambda U: float(sum(np.sum(a * b) for a, b in zip(w, U)))
    grad = _adjoint(s, U0, dt, K, nsteps, Sd, w)
    sc = field_scales(U0, bg)
    eps = 1e-4
    worst = 0.0
    for q in range(8):
        v = [sc[f] * rng.standard_normal(sh) for f, sh in enumerate(g.shapes())]
        Up = [a + eps * b for a, b in zip(U0, v)]
        Um = [a - eps * b for a, b in zip(U0, v)]
        fd = (J(_run(s, Up, dt, K, nsteps, Sd)) - J(_run(s, Um, dt, K, nsteps, Sd))) / (2 * eps)
        ad = float(sum(np.sum(a * b) for a, b in zip(grad, v)))
        rel = abs(fd - ad) / max(abs(fd), 1e-300)
        worst = max(worst, rel)
        assert rel <= 1e-4, (name, q, fd, ad, rel)
    longest, cap = s.tape_use()
    print(f"{name}: worst relative difference adjoint vs central differences {worst:.2e}; tape {longest}/{cap}")
    s.close()


def test_adjoint_vs_oracle_jacobian():
    """J^T lambda of one K = 2 step against the transpose of the oracle's
    central-difference Jacobian (every input and output entry, 4 x 5 x 6 cells,
    walled, gravity, rotation, a radial background)."""
    g = Grid(4, 5, 6, 1.0, 1.4, 0.6, 2.4, 0.2, 1.6)
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.05, pinf=2.0, g=0.3, omega=0.2)
    bg = (np.full(g.nr + 2, 20.0), np.full(g.nr + 2, 30.0))
    U = generic_state(g, 21, (0.1, 0.05, 0.05, 0.05, 0.1))
    dt = 0.01
    Jo = oracle_jacobian(g, par, bg, U, dt, 2, rel=1e-6)
    s = solver_for(g, par, bg)
    rng = np.random.default_rng(41)
    for q in range(4):
        lam = rng.standard_normal(Jo.shape[0])
        ref = Jo.T @ lam
        s.set_state(to_dev(U))
        got = flat(to_host(s.step_adjoint(dt, 2, to_dev(unflat(lam, g.shapes())))))
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print(f"J^T lambda vs the oracle's FD Jacobian, draw {q}: {err:.2e}")
        assert err <= 1e-6, (q, err)
    s.close()


def test_gradient_of_kinetic_energy_wrt_initial_theta():
    """The gradient a user takes: final kinetic energy after 6 steps of a small
    bubble, with respect to the initial potential-temperature perturbation
    (Gaussian plus 1e-3 white noise), through the autograd Function with
    checkpoints every ceil(sqrt(6)) = 3 steps, against central differences."""
    import torch
    from paper_2004_13887_gb300 import adjoint
    c = cases.bubble((8, 10, 12), seed=4, dt=1.0)
    g, par, bg = c.grid, c.par, c.bg
    rng = np.random.default_rng(42)
    Pi = torch.as_tensor(bg[1][1:-1] / 300.0, dtype=torch.float64, device="cuda")[:, None, None]
    th0 = torch.as_tensor(c.init[4] / (bg[1][1:-1] / 300.0)[:, None, None] + 1e-3 * rng.standard_normal(g.shapes()[4]),
                          dtype=torch.float64, device="cuda")
    s = sph.Solver(g, par)
    s.set_background(*bg)
    base = to_dev(c.init)

    def J_of(theta, grad=False):
        U0 = [base[0], base[1], base[2], base[3], Pi * theta]
        UN = adjoint.steps(s, c.dt, 2, 6, U0)
        return adjoint.kinetic_energy(UN, g, bg, par)

    th = th0.clone().requires_grad_(True)
    J = J_of(th)
    J.backward()
    grad = th.grad.detach().cpu().numpy()
    eps = 1e-4
    worst = 0.0
    with torch.no_grad():
        for q in range(8):
            v = torch.as_tensor(rng.standard_normal(g.shapes()[4]), dtype=torch.float64, device="cuda")
            fd = (float(J_of(th0 + eps * v)) - float(J_of(th0 - eps * v))) / (2 * eps)
            ad = float(np.sum(grad * v.cpu().numpy()))
            rel = abs(fd - ad) / max(abs(fd), 1e-300)
            worst = max(worst, rel)
            assert rel <= 1e-4, (q, fd, ad, rel)
    print(f"dKE/dtheta0: worst relative difference vs central differences {worst:.2e}, KE {float(J):.4e}")
    s.close()


def test_adjoint_with_wall_data():
    """The step adjoint on a solver whose walls move (the paper's manufactured
    solution, wall data and source held fixed over the steps), after a forward
    step with them: against central differences of the same steps."""
    c = cases.paper_mms(1e-2, n=(6, 7, 9))
    g, par, bg, dt = c.grid, c.par, c.bg, c.dt
    s = solver_for(g, par, bg)
    s.set_bc(c.walls(0.0), c.walls(dt))
    S = to_dev(c.source(0.5 * dt))
    U0 = c.init
    rng = np.random.default_rng(43)
    w = [rng.standard_normal(sh) for sh in g.shapes()]
    J = lambda U: float(sum(np.sum(a * b) for a, b in zip(w, U)))
    grad = _adjoint(s, U0, dt, 2, 2, S, w)
    sc = field_scales(U0, bg)
    eps = 1e-4
    for q in range(4):
        v = [sc[f] * rng.standard_normal(sh) for f, sh in enumerate(g.shapes())]
        fd = (J(_run(s, [a + eps * b for a, b in zip(U0, v)], dt, 2, 2, S))
              - J(_run(s, [a - eps * b for a, b in zip(U0, v)], dt, 2, 2, S))) / (2 * eps)
        ad = float(sum(np.sum(a * b) for a, b in zip(grad, v)))
        assert abs(fd - ad) <= 1e-4 * abs(fd), (q, fd, ad)
    s.close()
