"""Batched ensembles (independent problems of different sizes stepped by one
CUDA graph whose branches run concurrently), the enqueue-only step and its
status, and the per-shape line-solver autotuner."""
import numpy as np
import pytest

import paper_2004_13887_gb300 as sph
from paper_2004_13887_gb300 import ensemble
from inputs import cases
from tests.gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu
MIXED = sph.SPH_PREC_MIXED

# uneven grids: partitioned lengths (64, 128) next to block Thomas ones (16, 48, 192)
SHAPES = [(16, 64, 64), (32, 64, 128), (16, 128, 64), (48, 64, 64), (32, 192, 64), (64, 64, 128)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()


def _cases():
    return [cases.bubble(n, seed=10 + q, dt=1.0, amplitude=0.2 + 0.1 * q, radius=1500.0 + 200.0 * q)
            for q, n in enumerate(SHAPES)]


def _solver(c, prec=MIXED):
    import torch
    s = sph.Solver(c.grid, c.par, precision=prec, stream=torch.cuda.Stream())
    s.set_background(*c.bg)
    s.set_state(to_dev(c.init))
    return s


def test_batch_graph_equals_individual_steps():
    """Replaying the captured graph gives bit-for-bit the states of stepping
    each solver on its own (same kernels, same inputs)."""
    cs = _cases()
    ref = []
    for c in cs:
        s = _solver(c)
        for _ in range(4):
            s.step(c.dt, 2)
        ref.append(to_host(s.get_state()))
        s.close()
    solvers = [_solver(c) for c in cs]
    b = sph.Batch(solvers)
    b.capture(1.0, 2, steps=2)
    b.launch(2)
    b.status()
    for q, s in enumerate(solvers):
        got = to_host(s.get_state())
        for f in range(5):
            assert np.array_equal(got[f], ref[q][f]), (SHAPES[q], f)
    b.close()


# every line layout the batched launches take: 16 (narrow 4x4 and 16x1), 32
# (narrow), 48 (16x3), 64 (narrow, 16x4, one warp), 128 (16x8, one warp), 192,
# 256, cyclic phi lines (a periodic shell) next to walled ones, and stencil
# tiles of several shapes in one launch
FUSED = [((16, 64, 64), sph.SPH_LINES_PARTITIONED_NARROW, (1, 1)),
         ((32, 64, 128), sph.SPH_LINES_PARTITIONED, (2, 1)),
         ((16, 128, 64), sph.SPH_LINES_PARTITIONED, (2, 2)),
         ((48, 64, 64), sph.SPH_LINES_PARTITIONED_WARP, (4, 1)),
         ((32, 192, 64), sph.SPH_LINES_PARTITIONED_NARROW, (1, 2)),
         ((64, 64, 128), sph.SPH_LINES_PARTITIONED_WARP, (2, 1)),
         ((48, 256, 48), sph.SPH_LINES_PARTITIONED_NARROW, (4, 2)),
         ((64, 128, 256), sph.SPH_LINES_PARTITIONED_NARROW, (1, 1))]


def _fused_cases():
    out = []
    for q, (n, which, tile) in enumerate(FUSED):
        out.append((cases.bubble(n, seed=30 + q, dt=1.0, amplitude=0.3 + 0.1 * q, radius=1200.0 + 250.0 * q),
                    which, tile))
    # a whole shell (cyclic phi lines of 64, pole faces) among the sectors
    out.append((cases.shell_low_mach((32, 48, 64), M0=1e-3, dt=1.0), sph.SPH_LINES_PARTITIONED, (1, 1)))
    return out


def _tuned(c, which, tile):
    s = _solver(c)
    s.set_line_solver(which)
    s.set_tile(*tile)
    return s


def test_fused_batch_equals_individual_steps():
    """The batched launches (one kernel per stage and line layout over every
    instance, descriptor tables in device memory) give the states of stepping
    each solver on its own, in far fewer launches.  They run the same device
    code, compiled into other kernels, where the compiler may contract other
    FP32 multiply-adds: the increments agree to FP32 rounding (1e-5 of each
    field's change over the steps), not bit for bit."""
    cs = _fused_cases()
    ref, single = [], 0
    for c, which, tile in cs:
        s = _tuned(c, which, tile)
        l0 = s.launches
        for _ in range(4):
            s.step(c.dt, 2)
        single += s.launches - l0
        ref.append(to_host(s.get_state()))
        s.close()
    solvers = [_tuned(c, which, tile) for c, which, tile in cs]
    b = sph.Batch(solvers)
    b.capture(1.0, 2, steps=2, fused=True)
    l0 = sum(s.launches for s in solvers)
    b.launch(2)
    b.status()
    fused = sum(s.launches for s in solvers) - l0
    worst = 0.0
    for q, s in enumerate(solvers):
        got = to_host(s.get_state())
        c = cs[q][0]
        for f in range(5):
            scale = float(np.max(np.abs(ref[q][f] - c.init[f]))) or 1.0
            err = float(np.max(np.abs(got[f] - ref[q][f]))) / scale
            worst = max(worst, err)
            assert err <= 1e-5, ((c.grid.nr, c.grid.nt, c.grid.np), f, err)
    print(f"batched vs per-instance steps: worst difference {worst:.2e} of a field's change; "
          f"{fused} launches vs {single}")
    # per iteration: 6 stencil launches and two per line layout of each
    # direction (this set has many layouts; the 64-instance ensemble, ~35
    # launches per iteration against 64 x 12)
    assert 0 < fused < single / 2, (fused, single)
    # a replay after the states moved on keeps stepping them (the graph's
    # tables hold both buffers of every instance)
    b.launch(1)
    b.status()
    b.close()
    for s in solvers:
        s.close()


def test_fused_batch_refuses_what_it_cannot_batch():
    cs = _cases()[:2]
    for prec, which in ((sph.SPH_PREC_FP64, sph.SPH_LINES_PARTITIONED), (MIXED, sph.SPH_LINES_THOMAS)):
        solvers = [_solver(c, prec) for c in cs]
        solvers[1].set_line_solver(which)
        b = sph.Batch(solvers)
        with pytest.raises(sph.SphError):
            b.capture(1.0, 2, steps=2, fused=True)
        with pytest.raises(sph.SphError):
            b.capture(1.0, 2, steps=3, fused=True)
        b.close()
        for s in solvers:
            s.close()


def test_step_async_equals_step():
    c = _cases()[1]
    a, b = _solver(c), _solver(c)
    for _ in range(3):
        a.step(c.dt, 2)
        b.step_async(c.dt, 2)
    res = b.status(residual=True)
    assert res is not None and np.all(np.isfinite(res))
    for f in range(5):
        assert np.array_equal(to_host(a.get_state())[f], to_host(b.get_state())[f])


def test_batch_status_reports_the_failed_instance():
    cs = _cases()[:3]
    bad = [f.copy() for f in cs[2].init]
    bad[4][1, 2, 3] = np.nan
    solvers = [_solver(c) for c in cs]
    solvers[2].set_state(to_dev(bad))
    b = sph.Batch(solvers)
    b.capture(1.0, 2, steps=2)
    b.launch(1)
    with pytest.raises(sph.SphError):
        b.status()
    assert b.bad == 2
    b.close()


def test_batch_refuses_a_state_in_the_other_buffer():
    cs = _cases()[:2]
    solvers = [_solver(c) for c in cs]
    b = sph.Batch(solvers)
    b.capture(1.0, 2, steps=2)
    solvers[0].step(1.0, 2)       # one step outside the graph: U^n moved buffers
    with pytest.raises(sph.SphError):
        b.launch(1)
    solvers[0].step(1.0, 2)       # back in the captured buffer
    b.launch(1)
    b.status()
    with pytest.raises(sph.SphError):
        b.capture(1.0, 2, steps=3)   # odd step counts cannot be replayed
    b.close()


def test_autotune_choices_agree():
    cs = _cases()
    choice = ensemble.autotune(cs, 1.0, 2)
    assert set(choice) == {(c.grid.nr, c.grid.nt, c.grid.np) for c in cs}
    assert all(v[0] in (sph.SPH_LINES_THOMAS, sph.SPH_LINES_PARTITIONED, sph.SPH_LINES_PARTITIONED_WARP,
                        sph.SPH_LINES_PARTITIONED_NARROW)
               and v[1] in ensemble.TILES for v in choice.values())
    c = cs[5]   # 64 x 64 x 128: every solver applies
    xs = []
    for which in (sph.SPH_LINES_THOMAS, sph.SPH_LINES_PARTITIONED, sph.SPH_LINES_PARTITIONED_WARP,
                  sph.SPH_LINES_PARTITIONED_NARROW):
        s = _solver(c)
        s.set_line_solver(which)
        for _ in range(2):
            s.step(c.dt, 2)
        xs.append(to_host(s.get_state()))
        s.close()
    for f in range(5):
        scale = float(np.max(np.abs(xs[0][f] - c.init[f]))) or 1.0
        for x in xs[1:]:
            assert float(np.max(np.abs(xs[0][f] - x[f]))) <= 1e-5 * scale


def test_tile_shape_leaves_results_unchanged():
    """The stencil tile shape the autotuner picks changes how the kernels are
    launched, not what they compute: every shape gives bit-for-bit the same
    step."""
    c = _cases()[3]   # 48 x 64 x 64: boundary and interior tiles in r and theta
    ref = None
    for tj, ti in ensemble.TILES:
        s = _solver(c)
        s.set_tile(tj, ti)
        s.step(c.dt, 2)
        got = to_host(s.get_state())
        s.close()
        if ref is None:
            ref = got
        for f in range(5):
            assert np.array_equal(got[f], ref[f]), ((tj, ti), f)
    s = _solver(c)
    with pytest.raises(sph.SphError):
        s.set_tile(3, 1)
    with pytest.raises(sph.SphError):
        s.set_tile(4, 4)
    s.close()


def test_ensemble_of_config_five():
    """The 64-instance ensemble (uneven grids, random bubbles): 10 steps through
    the graph, every instance finite, and two instances against the FP64 mode
    (relative L2 of T and u <= 1e-6)."""
    specs = cases.ensemble_specs()
    cs = [cases.bubble(sp["n"], seed=sp["seed"], dt=1.0, amplitude=sp["amplitude"], radius=sp["radius"])
          for sp in specs]
    ens = ensemble.Ensemble(cs, dt=1.0, n_iter=2)
    ens.run(10)
    ens.status()
    for q in (0, 37):
        c = cs[q]
        got = to_host(ens.solvers[q].get_state())
        assert all(np.all(np.isfinite(f)) for f in got)
        s = _solver(c, prec=sph.SPH_PREC_FP64)
        for _ in range(10):
            s.step(c.dt, 2)
        ref = to_host(s.get_state())
        s.close()
        T = lambda U: U[4] + c.bg[1][1:-1][:, None, None]
        assert np.linalg.norm(T(got) - T(ref)) <= 1e-6 * np.linalg.norm(T(ref))
        du = sum(np.linalg.norm(got[k] - ref[k]) ** 2 for k in (1, 2, 3)) ** 0.5
        nu = sum(np.linalg.norm(ref[k]) ** 2 for k in (1, 2, 3)) ** 0.5
        assert du <= 1e-6 * nu, (q, du, nu)
    ens.close()
