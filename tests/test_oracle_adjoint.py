"""The oracle-side adjoint: the transpose of the finite-difference Jacobian of
one oracle step (4 x 5 x 6 cells), the reference the library's step adjoint is
compared with.  Pinned here by its own convergence: the Jacobians at two
difference steps agree to the O(step^2) truncation error, and on a state at
rest with no gravity (no advection, only the linear acoustic and viscous
operators acting) the step is linear, so the Jacobian applied to any state
reproduces the step itself."""
import numpy as np

import oracle
from inputs import Grid, Params
from tests.adjoint_helpers import flat, generic_state, oracle_jacobian, unflat


def _case():
    g = Grid(4, 5, 6, 1.0, 1.4, 0.6, 2.4, 0.2, 1.6)
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.05, pinf=2.0, g=0.3, omega=0.2)
    bg = (np.full(g.nr + 2, 20.0), np.full(g.nr + 2, 30.0))
    return g, par, bg, generic_state(g, 21, (0.1, 0.05, 0.05, 0.05, 0.1)), 0.01


def test_fd_jacobian_converged():
    oracle.build()
    g, par, bg, U, dt = _case()
    J1 = oracle_jacobian(g, par, bg, U, dt, 2, rel=1e-5)
    J2 = oracle_jacobian(g, par, bg, U, dt, 2, rel=2e-6)
    assert np.max(np.abs(J1 - J2)) <= 1e-7 * np.max(np.abs(J1)), np.max(np.abs(J1 - J2))


def test_fd_jacobian_of_a_linear_step():
    """Around a uniform state at rest with g = 0 and no rotation the step's
    operators freeze at constant coefficients only through Ubar; with a
    perturbation 1e-8 of the background, step(U) is linear in U to 1e-8, so
    J U equals step(U) (both perturbations of the rest state)."""
    oracle.build()
    g = Grid(4, 5, 6, 1.0, 1.4, 0.6, 2.4, 0.2, 1.6)
    par = Params(gamma=1.4, cv=2.5, Pr=0.7, mu=0.05)
    bg = (np.full(g.nr + 2, 20.0), np.full(g.nr + 2, 30.0))
    U = generic_state(g, 22, (1e-7, 1e-8, 1e-8, 1e-8, 1e-7))
    J = oracle_jacobian(g, par, bg, g.zeros(), 0.01, 2, rel=1e-4)
    y, _ = oracle.step(g, par, U, 0.01, 2, bg=bg)
    lin = J @ flat(U)
    assert np.max(np.abs(lin - flat(y))) <= 1e-6 * np.max(np.abs(flat(y))), np.max(np.abs(lin - flat(y)))
