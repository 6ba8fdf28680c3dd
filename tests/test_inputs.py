"""The seeded input generators: the generated sector manufactured-solution
module matches the sympy definition it was produced from, and the thermal
bubble background is in discrete hydrostatic balance."""
import numpy as np
import pytest

from inputs import cases, sample


def test_generated_sector_mms_matches_sympy():
    pytest.importorskip("sympy")
    gen = cases.sector_mms((6, 7, 8))
    ref = cases.sector_mms((6, 7, 8), use_sympy=True)
    for t in (0.0, 3.7e-3):
        for a, b in zip(gen.exact(t), ref.exact(t)):
            assert np.max(np.abs(a - b)) <= 1e-12 * (np.max(np.abs(b)) + 1e-300)
        for a, b in zip(gen.source(t), ref.source(t)):
            assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_sector_mms_boundary_data_are_homogeneous():
    c = cases.sector_mms((6, 7, 8))
    p, ur, ut, up, T = c.exact(1e-3)
    assert np.max(np.abs(ur[0])) < 1e-14 and np.max(np.abs(ur[-1])) < 1e-14
    assert np.max(np.abs(ut[:, 0])) < 1e-14 and np.max(np.abs(ut[:, -1])) < 1e-14
    assert np.max(np.abs(up[:, :, 0])) < 1e-14 and np.max(np.abs(up[:, :, -1])) < 1e-14


def test_hydrostatic_background_balance():
    g = cases.bubble_grid((16, 4, 4))
    p, T, _ = cases.hydrostatic_background(g)
    Rg = cases.AIR["cp"] - cases.AIR["cv"]
    rho = p / (Rg * T)
    lhs = (p[1:] - p[:-1]) / g.dr
    rhs = -cases.AIR["g"] * 0.5 * (rho[1:] + rho[:-1])
    assert np.max(np.abs(lhs - rhs)) <= 1e-10 * np.max(np.abs(rhs))
    # close to the continuous profile p00 * Pi^(cp/R) (Section 3.2)
    h = (np.arange(-1, g.nr + 1) + 0.5) * g.dr
    pc = 1e5 * (1 - cases.AIR["g"] * h / (cases.AIR["cp"] * 300.0)) ** (cases.AIR["cp"] / Rg)
    assert np.max(np.abs(p - pc) / pc) < 1e-3


def test_bubble_is_seeded():
    a, b = cases.bubble((4, 6, 6), seed=1), cases.bubble((4, 6, 6), seed=1)
    assert np.array_equal(a.init[4], b.init[4])
    c = cases.bubble((4, 6, 6), seed=2)
    assert not np.array_equal(a.init[4], c.init[4])
