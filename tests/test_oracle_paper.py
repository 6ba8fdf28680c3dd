"""The oracle against the numbers Section 3.1 prints for the manufactured
solution of eq. (man_sol), and against second-order convergence.

Fixtures (tests/golden/):
  tab_inc.txt -- Table tab:inc, max |p - p0|/p0 after n steps, tau = 1e-3
  tab_tcr.txt -- Tables tab:timept / tab:timeu, time convergence rates

Readings (the paper does not give them): c_v = 1, the source is evaluated at
t^{n+1/2}, and tab:inc's "grid diameter 0.12" is replaced by a 16 x 11 x 33 grid
whose cell centres reach the maxima of the exact pressure (max cell diagonal
0.41); at M0 >= 1e-4 the table is set by the exact solution and is insensitive
to the grid.
"""
import math
import os

import numpy as np
import pytest

import oracle
from inputs import cases

pytest.importorskip("sympy")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_tab_inc_matches_closed_form_of_the_manufactured_solution():
    """max over the domain of (p - p0)/p0 for eq. (man_sol) is u0^2 (2 + sin 5t)/p0
    with u0 = M0 c0, c0 = sqrt(gamma p0) = 100: the printed table follows it for
    M0 >= 1e-3 (to the two printed digits)."""
    p0, c0 = 6250.0, 100.0
    for row in _load("tab_inc.txt"):
        n = int(row[0])
        t = n * 1e-3
        for M0, printed in zip((1e-2, 1e-3), map(float, row[1:3])):
            closed = (M0 * c0) ** 2 * (2 + math.sin(5 * t)) / p0
            assert abs(closed - printed) <= 0.05 * 10 ** math.floor(math.log10(printed)), (n, M0)


def _run_paper_mms(M0, n, steps, K=2, tau=1e-3, record=()):
    c = cases.paper_mms(M0, n=n)
    U, out = c.init, {}
    for s in range(steps):
        t = s * tau
        U, _ = oracle.step(c.grid, c.par, U, tau, K, bg=c.bg, walls_n=c.walls(t), walls_np1=c.walls(t + tau),
                           S=c.source(t + 0.5 * tau))
        if s + 1 in record:
            out[s + 1] = np.max(np.abs(U[0])) / c.info["p0"]
    return U, out, c


def test_tab_inc_low_mach_pressure_fluctuations():
    rows = {int(r[0]): list(map(float, r[1:])) for r in _load("tab_inc.txt")}
    for col, M0 in enumerate((1e-2, 1e-3, 1e-4, 1e-5, 1e-6)):
        _, got, _ = _run_paper_mms(M0, (16, 11, 33), 100, record=(1, 50, 100))
        for n in (1, 50, 100):
            printed = rows[n][col]
            if M0 >= 1e-4:
                assert abs(got[n] - printed) <= 0.03 * printed, (M0, n, got[n], printed)
            else:
                # Delta p stays O(M0^2): within a small factor of the printed value and far
                # below the O(M0) level of spurious acoustic waves
                assert got[n] <= 4.0 * printed and got[n] < 1e-3 * M0, (M0, n, got[n], printed)


def _tcr_table():
    """Tables tab:timept / tab:timeu (tests/golden/tab_tcr.txt): (field, tau, M0) -> printed TCR"""
    out = {}
    for row in _load("tab_tcr.txt"):
        for M0, v in zip((1e-2, 1e-4, 1e-6), row[2:5]):
            out[(row[0], float(row[1]), M0)] = float(v)
    return out


def test_time_convergence_rates():
    """TCR(tau) = log2(|u^tau - u^{tau/2}| / |u^{tau/2} - u^{tau/4}|) at the printed
    tau in {2e-3, 1e-3, 5e-4}, against Tables tab:timept and tab:timeu
    (tests/golden/tab_tcr.txt; the paper's grid is not stated, so the rates are
    compared, not matched digit by digit):
    * every rate at least the smallest printed for that M0 less 0.3 (the printed
      rates scatter from 1.4 to 3.2 around second order);
    * at the smallest printed tau, 5e-4, the mean over the five fields within
      0.3 of the printed mean, and no field above the largest printed rate of
      that M0 plus 0.5.
    (At tau = 2e-3 and 1e-3 the velocity rates at low Mach number can exceed the
    printed maximum: the error there is pre-asymptotic and falls faster than
    second order.)"""
    tend = 0.01
    table = _tcr_table()
    fields = ["p", "ur", "ut", "up", "T"]
    for M0 in (1e-2, 1e-6):
        sols = {}
        for tau in (2e-3, 1e-3, 5e-4, 2.5e-4, 1.25e-4):
            U, _, _ = _run_paper_mms(M0, (8, 8, 24), int(round(tend / tau)), tau=tau)
            sols[tau] = U
        printed_all = [v for (f, t, m), v in table.items() if m == M0]
        for tau in (2e-3, 1e-3, 5e-4):
            t2, t4 = tau / 2, tau / 4
            tcr = {f: math.log2(np.linalg.norm(sols[tau][q] - sols[t2][q]) / np.linalg.norm(sols[t2][q] - sols[t4][q]))
                   for q, f in enumerate(fields)}
            for f, v in tcr.items():
                assert v >= min(printed_all) - 0.3, (M0, tau, f, v)
            if tau == 5e-4:
                printed = [table[(f, tau, M0)] for f in fields]
                assert abs(np.mean(list(tcr.values())) - np.mean(printed)) <= 0.3, (M0, tcr, printed)
                assert max(tcr.values()) <= max(printed_all) + 0.5, (M0, tcr)


def test_space_convergence_sector_mms():
    """Second-order l2 error of p and u_phi under refinement (cf. fig:conv), on the
    sector manufactured solution with no-slip walls."""
    tau, steps = 2e-4, 5
    errs = []
    for n in (8, 16, 32):
        c = cases.sector_mms((n, n, n))
        U = c.init
        for s in range(steps):
            U, _ = oracle.step(c.grid, c.par, U, tau, 2, bg=c.bg, S=c.source((s + 0.5) * tau))
        ex = c.exact(steps * tau)
        errs.append([np.sqrt(np.mean((U[q] - ex[q]) ** 2)) for q in (0, 3)])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > 1.8), (errs, rates)


def test_space_convergence_paper_mms():
    """Same with the paper's solution and its time-dependent wall data, M0 = 1e-2."""
    tau, steps = 1e-4, 4
    errs = []
    for n in ((4, 4, 12), (8, 8, 24), (16, 16, 48)):
        U, _, c = _run_paper_mms(1e-2, n, steps, tau=tau)
        ex = c.exact(steps * tau)
        errs.append([np.sqrt(np.mean((U[q] - ex[q]) ** 2)) for q in (0, 3)])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > 1.7), (errs, rates)


@pytest.mark.parametrize("M0", [1e-4, 1e-6])
def test_space_convergence_paper_mms_low_mach(M0):
    """Second-order l2 error in space at M0 = 1e-4 and 1e-6 as well (fig:conv,
    tau = 2e-5 instead of the paper's 1e-5 to halve the run, t = 1e-3): the pressure rate approaches 2
    from below (1.4 between the two coarser grids, 1.8 between the finer ones);
    at M0 = 1e-6 the u_phi error is at the round-off level (the paper notes the
    same), so it is bounded instead of rated."""
    tau, steps = 2e-5, 50
    errs = []
    for n in ((16, 16, 48), (32, 32, 96)):
        U, _, c = _run_paper_mms(M0, n, steps, tau=tau)
        ex = c.exact(steps * tau)
        errs.append([np.sqrt(np.mean((U[q] - ex[q]) ** 2)) for q in (0, 3)])
    errs = np.array(errs)
    rates = np.log2(errs[0] / errs[1])
    assert rates[0] > 1.7, (errs, rates)
    if M0 >= 1e-4:
        assert rates[1] > 1.9, (errs, rates)
    else:
        assert errs[1, 1] < 1e-12, errs


def test_tab_inc_at_the_paper_grid_diameter():
    """Table tab:inc's grid diameter, 0.12 (max cell diagonal in physical space,
    reading R13): 14 x 45 x 135 cells, diameter 0.122, one step of tau = 1e-3.
    * M0 = 1e-2 reproduces the printed 3.2e-4 within 3 %.
    * At M0 = 1e-6 the fluctuation with K = 2 carries an O(M0) part (7.6e-10,
      against the printed 3.9e-12): the unconverged splitting iteration at an
      acoustic Courant number c0 tau / h of about 3 on this grid (0.7 on the
      16 x 11 x 33 grid of the test above).  K = 6 removes more than 90 % of it,
      which pins the cause: the iteration, not the operators."""
    n = (14, 45, 135)
    got = {}
    for M0, K in ((1e-2, 2), (1e-6, 2), (1e-6, 6)):
        c = cases.paper_mms(M0, n=n)
        U, _ = oracle.step(c.grid, c.par, c.init, 1e-3, K, bg=c.bg, walls_n=c.walls(0.0), walls_np1=c.walls(1e-3),
                           S=c.source(0.5e-3))
        got[(M0, K)] = np.max(np.abs(U[0])) / c.info["p0"]
    rows = {int(r[0]): list(map(float, r[1:])) for r in _load("tab_inc.txt")}
    assert abs(got[(1e-2, 2)] - rows[1][0]) <= 0.03 * rows[1][0], got
    assert got[(1e-6, 2)] > 10 * rows[1][4], got                 # the O(M0) splitting part is there
    assert got[(1e-6, 6)] < 0.1 * got[(1e-6, 2)], got            # and it is the iteration's
