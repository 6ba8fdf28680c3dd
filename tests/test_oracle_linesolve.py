"""Pins of the oracle's line solvers (Section 2.2: block-tridiagonal Thomas; the
cyclic variants serve periodic phi).  Each solver is checked against a dense
LU solve (numpy.linalg.solve) of the same matrix written out in full, on
random diagonally dominant systems and on systems assembled from the scheme."""
import numpy as np
import pytest

import oracle
from inputs import Grid, Params, cases


def dense_scalar(a, b, c, cyclic=False):
    n = len(b)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    if cyclic:
        M[0, n - 1] += a[0]
        M[n - 1, 0] += c[n - 1]
    return M


def dense_block(A, B, C, cyclic=False):
    n = B.shape[0]
    M = np.zeros((3 * n, 3 * n))
    for m in range(n):
        M[3 * m:3 * m + 3, 3 * m:3 * m + 3] = B[m]
        if m > 0:
            M[3 * m:3 * m + 3, 3 * (m - 1):3 * m] = A[m]
        if m < n - 1:
            M[3 * m:3 * m + 3, 3 * (m + 1):3 * (m + 2)] = C[m]
    if cyclic:
        M[0:3, 3 * (n - 1):] += A[0]
        M[3 * (n - 1):, 0:3] += C[n - 1]
    return M


@pytest.mark.parametrize("n", [1, 2, 5, 33, 64])
def test_thomas_vs_dense(n):
    rng = np.random.default_rng(n)
    a, c, d = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    b = 4.0 + rng.random(n)
    if n > 1:
        a[0] = 0.0
        c[-1] = 0.0
    x = oracle.thomas(a, b, c, d)
    ref = np.linalg.solve(dense_scalar(a, b, c), d)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [3, 4, 17, 64])
def test_cyclic_thomas_vs_dense(n):
    rng = np.random.default_rng(100 + n)
    a, c, d = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    b = 4.0 + rng.random(n)
    x = oracle.cyclic_thomas(a, b, c, d)
    ref = np.linalg.solve(dense_scalar(a, b, c, cyclic=True), d)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def _random_blocks(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, 3, 3)) * 0.5
    C = rng.standard_normal((n, 3, 3)) * 0.5
    # non-symmetric diagonal blocks that need pivoting inside the block
    B = rng.standard_normal((n, 3, 3)) + 5.0 * np.eye(3)
    B[:, 0, 0] = 1e-3 * rng.standard_normal(n)   # small leading entry: exercises partial pivoting
    B[:, 0, 1] += 6.0
    B[:, 1, 0] += 6.0
    d = rng.standard_normal((n, 3))
    return A, B, C, d


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_block_thomas_vs_dense(n):
    A, B, C, d = _random_blocks(n, n)
    A[0] = 0
    C[-1] = 0
    x = oracle.block_thomas(A, B, C, d)
    ref = np.linalg.solve(dense_block(A, B, C), d.ravel()).reshape(n, 3)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [3, 5, 64])
def test_block_cyclic_vs_dense(n):
    A, B, C, d = _random_blocks(n, 1000 + n)
    x = oracle.block_thomas(A, B, C, d, cyclic=True)
    ref = np.linalg.solve(dense_block(A, B, C, cyclic=True), d.ravel()).reshape(n, 3)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def _assembled_case(periodic):
    """A sector state with non-trivial velocity, so that every coefficient is active."""
    if periodic:
        g = Grid(6, 7, 9, 1.0, 2.0, 0.5, 2.6, 0.0, 2 * np.pi, periodic=True)
    else:
        g = Grid(6, 7, 9, 1.0, 2.0, np.pi / 4, 3 * np.pi / 4, np.pi / 4, 7 * np.pi / 4)
    par = Params(gamma=1.6, cv=1.0, Pr=1.0, mu=0.3, omega=0.2, g=0.5)
    rng = np.random.default_rng(7)
    U = [rng.standard_normal(s) for s in g.shapes()]
    U[0] = 50.0 + U[0]
    U[4] = 80.0 + U[4]
    return g, par, U


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_assembled_lines_vs_dense(periodic, direction, kind):
    g, par, U = _assembled_case(periodic)
    tau = 0.05
    cyc = periodic and direction == 2
    a, b = (1, 1) if kind else (2, 3)
    A, B, C = oracle.line_system(g, par, U, direction, kind, a, b, tau)
    rng = np.random.default_rng(11)
    if kind == 0:
        d = rng.standard_normal(B.shape[:2])
        x = oracle.block_thomas(A, B, C, d, cyclic=cyc)
        ref = np.linalg.solve(dense_block(A, B, C, cyclic=cyc), d.ravel()).reshape(d.shape)
    else:
        d = rng.standard_normal(B.shape)
        x = (oracle.cyclic_thomas if cyc else oracle.thomas)(A, B, C, d)
        ref = np.linalg.solve(dense_scalar(A, B, C, cyclic=cyc), d)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))
