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


def test_time_convergence_rates():
    """TCR at least the printed minimum 1.4 at tau = 1e-3 and 5e-4; at the smallest
    tau every field inside the printed range [1.4, 3.3] and the mean close to 2.
    (At tau = 1e-3 the velocity rate can exceed the printed maximum: the error is
    still pre-asymptotic and falls faster than second order.)"""
    tend = 0.01
    fields = ["p", "ur", "ut", "up", "T"]
    for M0 in (1e-2, 1e-6):
        sols = {}
        for tau in (1e-3, 5e-4, 2.5e-4, 1.25e-4):
            U, _, _ = _run_paper_mms(M0, (8, 8, 24), int(round(tend / tau)), tau=tau)
            sols[tau] = U
        for tau in (1e-3, 5e-4):
            t2, t4 = tau / 2, tau / 4
            tcr = [math.log2(np.linalg.norm(sols[tau][q] - sols[t2][q]) / np.linalg.norm(sols[t2][q] - sols[t4][q]))
                   for q in range(5)]
            for f, v in zip(fields, tcr):
                assert v >= 1.4, (M0, tau, f, v)
                if tau == 5e-4:
                    assert v <= 3.3, (M0, tau, f, v)
            if tau == 5e-4:
                assert 1.8 <= np.mean(tcr) <= 2.3, (M0, tcr)


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
