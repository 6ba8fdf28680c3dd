"""The partitioned block Thomas kernels (sph_schur_local, sph_schur_reduced,
sph_schur_back) on the GPU: P ranks' segments emulated in one process (each
rank's steps called in turn, the all-gather by stacking -- no kernel waits on
another), against the oracle's whole-line block Thomas and cyclic block Thomas
(1e-12), and each step against the plain reference of the CPU rank test."""
import numpy as np
import pytest

import oracle
import paper_2004_13887_gb300 as sph
from paper_2004_13887_gb300 import schur
from tests.schur_helpers import ReferenceOps, block_lines, segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    sph.build()
    oracle.build()


@pytest.mark.parametrize("P", [1, 2, 4, 8])
@pytest.mark.parametrize("cyclic", [False, True])
def test_schur_kernels_vs_oracle(P, cyclic):
    import torch
    nl, n = 300, 48
    arrs = block_lines(nl, n, 91 + P, cyclic)
    ops = schur.CudaOps()
    parts = []
    for r in range(P):
        seg = [torch.from_numpy(a).cuda() for a in segment(arrs, r, P)]
        parts.append((seg, ops.local(*seg)))
    iface = torch.stack([schur.interface_rows(*lp) for _, lp in parts])
    z = ops.reduced(iface, cyclic)
    xs = []
    for r, (seg, (Y, V, W)) in enumerate(parts):
        xl, xr = schur.neighbour_blocks(z, r, P, cyclic)
        xs.append(ops.back(Y, V, W, xl, xr).cpu().numpy())
    x = np.concatenate(xs, axis=1)
    A, B, C, d = arrs
    worst = 0.0
    for l in range(0, nl, 7):
        ref = oracle.block_thomas(A[l], B[l], C[l], d[l], cyclic=cyclic)
        worst = max(worst, np.max(np.abs(x[l] - ref)) / np.max(np.abs(ref)))
    assert worst <= 1e-12, worst
    # each step against the reference arithmetic
    ref_ops = ReferenceOps()
    seg = [torch.from_numpy(a) for a in segment(arrs, 0, P)]
    for got, want in zip(parts[0][1], ref_ops.local(*seg)):
        assert torch.max(torch.abs(got.cpu() - want)) <= 1e-12 * torch.max(torch.abs(want))
    zr = ref_ops.reduced(iface.cpu(), cyclic)
    assert torch.max(torch.abs(z.cpu() - zr)) <= 1e-12 * torch.max(torch.abs(zr))


def test_schur_rejects_bad_sizes():
    lib = sph.load()
    import ctypes as C
    dummy = C.cast(C.c_void_p(16), sph._DP)
    flag = C.cast(C.c_void_p(16), C.POINTER(C.c_int))
    assert lib.sph_schur_local(4, 1, dummy, dummy, dummy, dummy, dummy, dummy, dummy, dummy, flag, None) == -1
    assert lib.sph_schur_reduced(4, 9, 0, dummy, dummy, flag, None) == -1
