"""Seeded block lines and a plain reference of the three arithmetic steps of the
partitioned block Thomas algorithm (dense solves with torch on the CPU), so
that the communication order of paper_2004_13887_gb300.schur can run on CPU
ranks."""
import numpy as np


def block_lines(nlines, n, seed, cyclic):
    """diagonally dominant random 3x3-block lines (A_0 / C_{n-1} zero when walled)"""
    rng = np.random.default_rng(seed)
    A = 0.3 * rng.standard_normal((nlines, n, 3, 3))
    C = 0.3 * rng.standard_normal((nlines, n, 3, 3))
    B = 0.3 * rng.standard_normal((nlines, n, 3, 3)) + 3.0 * np.eye(3)
    d = rng.standard_normal((nlines, n, 3))
    if not cyclic:
        A[:, 0] = 0.0
        C[:, -1] = 0.0
    return A, B, C, d


def segment(arrs, rank, world):
    """rank's consecutive share of the blocks of every line"""
    n = arrs[0].shape[1]
    cuts = np.linspace(0, n, world + 1).round().astype(int)
    return [a[:, cuts[rank]:cuts[rank + 1]].copy() for a in arrs]


class ReferenceOps:
    """the three steps by dense solves (torch CPU float64), for the rank tests"""

    def local(self, A, B, Cb, d):
        import torch
        nl, m = B.shape[0], B.shape[1]
        T = torch.zeros((nl, 3 * m, 3 * m), dtype=torch.float64)
        for i in range(m):
            T[:, 3 * i:3 * i + 3, 3 * i:3 * i + 3] = B[:, i]
            if i > 0:
                T[:, 3 * i:3 * i + 3, 3 * i - 3:3 * i] = A[:, i]
            if i < m - 1:
                T[:, 3 * i:3 * i + 3, 3 * i + 3:3 * i + 6] = Cb[:, i]
        rhs = torch.zeros((nl, 3 * m, 7), dtype=torch.float64)
        rhs[:, :, 0] = d.reshape(nl, 3 * m)
        rhs[:, 0:3, 1:4] = A[:, 0]
        rhs[:, 3 * m - 3:, 4:7] = Cb[:, m - 1]
        X = torch.linalg.solve(T, rhs).reshape(nl, m, 3, 7)
        return X[..., 0].contiguous(), X[..., 1:4].contiguous(), X[..., 4:7].contiguous()

    def reduced(self, iface, cyclic):
        import torch
        P, nl = iface.shape[0], iface.shape[1]
        n = 6 * P
        M = torch.eye(n, dtype=torch.float64).repeat(nl, 1, 1)
        rhs = torch.zeros((nl, n), dtype=torch.float64)
        for p in range(P):
            f = iface[p]
            V0, Vm, W0, Wm = (f[:, 9 * q:9 * q + 9].reshape(nl, 3, 3) for q in range(4))
            rhs[:, 6 * p:6 * p + 3] = f[:, 36:39]
            rhs[:, 6 * p + 3:6 * p + 6] = f[:, 39:42]
            left, right = p - 1, p + 1
            if cyclic or left >= 0:
                left %= P
                M[:, 6 * p:6 * p + 3, 6 * left + 3:6 * left + 6] += V0
                M[:, 6 * p + 3:6 * p + 6, 6 * left + 3:6 * left + 6] += Vm
            if cyclic or right < P:
                right %= P
                M[:, 6 * p:6 * p + 3, 6 * right:6 * right + 3] += W0
                M[:, 6 * p + 3:6 * p + 6, 6 * right:6 * right + 3] += Wm
        z = torch.linalg.solve(M, rhs)
        return z.reshape(nl, 2 * P, 3)

    def back(self, Y, V, W, xl, xr):
        import torch
        return Y - torch.einsum("lmij,lj->lmi", V, xl) - torch.einsum("lmij,lj->lmi", W, xr)
