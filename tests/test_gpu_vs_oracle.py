"""Whole steps of the configurations against the FP64 oracle directly (not only
against the library's own FP64 mode): the mixed mode on the benchmark workload,
the full sphere in FP64 and its mixed-mode error over the configuration's 50
steps, ensemble instances stepped by the batched CUDA graph, and the Thermal 1
and Thermal 2 bubbles of Section 3.2 with their cos^2 perturbations at K = 10
and 50.

Bounds: relative L2 per physical field (p, rho, theta, T; the velocity as one
vector) of 1e-6 for the mixed mode -- the error statement of the mixed
precision path -- and, for FP64, 1e-12 of each field's natural scale."""
import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from inputs import cases
from tests.gpu_helpers import field_errors, solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu
MIXED = sph.SPH_PREC_MIXED


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()
    oracle.build()


def _oracle_steps(c, steps, K=2):
    U = c.init
    for _ in range(steps):
        U, _ = oracle.step(c.grid, c.par, U, c.dt, K, bg=c.bg)
    return U


def _lib_steps(c, steps, K=2, prec=MIXED):
    s = solver_for(c.grid, c.par, c.bg, c.init, precision=prec)
    for _ in range(steps):
        s.step(c.dt, K)
    U = to_host(s.get_state())
    s.close()
    return U


def test_mixed_full_size_vs_oracle():
    """The benchmark workload (bubble, 128 x 256 x 256), two mixed steps against
    two oracle steps on the whole grid."""
    c = cases.bubble((128, 256, 256), seed=1, dt=1.0)
    errs = field_errors(_lib_steps(c, 2), _oracle_steps(c, 2), c.bg, c.par)
    print("mixed vs oracle, bubble 128x256x256, 2 steps:", errs)
    for k, v in errs.items():
        assert v <= 1e-6, (k, v)


def test_full_sphere_fp64_two_steps_vs_oracle():
    c = cases.shell_low_mach((64, 512, 1024), M0=1e-4)
    U = _lib_steps(c, 2, prec=sph.SPH_PREC_FP64)
    Uo = _oracle_steps(c, 2)
    c0 = c.info["c0"]
    scale = [c.info["p0"], c0, c0, c0, c.info["T0"]]
    for q in range(5):
        err = float(np.max(np.abs(U[q] - Uo[q])))
        assert err <= 1e-12 * scale[q], (q, err, scale[q])


@pytest.mark.parametrize("M0", [1e-4, 1e-5, 1e-6])
def test_full_sphere_mixed_error_over_fifty_steps(M0):
    """The full-sphere configuration's error statement at its own length: mixed
    vs FP64 after 50 steps, per physical field."""
    c = cases.shell_low_mach((64, 512, 1024), M0=M0)
    U64 = _lib_steps(c, 50, prec=sph.SPH_PREC_FP64)
    U32 = _lib_steps(c, 50)
    errs = field_errors(U32, U64, c.bg, c.par)
    fl = float(np.max(np.abs(U64[0])))
    errs["p_fluct"] = float(np.max(np.abs(U32[0] - U64[0]))) / fl
    print(f"full sphere, M0={M0}, 50 steps, mixed vs fp64:", errs)
    for k in ("p", "rho", "theta", "T", "u"):
        assert errs[k] <= 1e-6, (k, errs)


@pytest.mark.parametrize("fused", [False, True])
def test_ensemble_instances_vs_oracle(fused):
    """Three instances of different shapes stepped together by the batched CUDA
    graph (one branch each, or batched launches over all three), against the
    oracle stepping each alone."""
    import torch
    specs = [((16, 64, 64), 11), ((32, 64, 128), 12), ((48, 128, 64), 13)]
    cs = [cases.bubble(n, seed=sd, dt=1.0, amplitude=0.5, radius=1800.0) for n, sd in specs]
    solvers = []
    for c in cs:
        s = sph.Solver(c.grid, c.par, precision=MIXED, stream=torch.cuda.Stream())
        s.set_background(*c.bg)
        s.set_state(to_dev(c.init))
        solvers.append(s)
    if fused:
        solvers[0].set_line_solver(sph.SPH_LINES_PARTITIONED_NARROW)
    b = sph.Batch(solvers)
    b.capture(1.0, 2, steps=2, fused=fused)
    b.launch(2)
    b.status()
    for s, c in zip(solvers, cs):
        errs = field_errors(to_host(s.get_state()), _oracle_steps(c, 4), c.bg, c.par)
        print("ensemble instance", "fused" if fused else "graph", c.grid.nr, c.grid.nt, c.grid.np, errs)
        for k, v in errs.items():
            assert v <= 1e-6, (c.grid, k, v)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("which,K", [("thermal1", 10), ("thermal2", 50)])
def test_thermal_bubbles_vs_oracle(which, K):
    """Section 3.2's bubbles with the paper's cos^2 perturbations on small grids
    of their domains, three steps at the paper's larger time steps and K = 10
    (Thermal 1 at tau = 50 s's companion setting) and 50."""
    if which == "thermal1":
        c = cases.thermal1((20, 40, 40), dt=5.0, K=K)
    else:
        c = cases.thermal2((24, 24, 24), dt=1.0, K=K)
    errs = field_errors(_lib_steps(c, 3, K=K), _oracle_steps(c, 3, K=K), c.bg, c.par)
    print(which, "K", K, errs)
    for k, v in errs.items():
        assert v <= 1e-6, (k, v)
