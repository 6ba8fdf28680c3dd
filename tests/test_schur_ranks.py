"""The partitioned (Schur-complement) block Thomas algorithm of Section 2.2 --
lines split across ranks, local elimination, an all-gather of the interface
rows, one reduced solve on every rank, back-substitution -- run as 2 and 4
gloo ranks on the CPU with a plain reference of the arithmetic steps, against
the oracle's single-domain block Thomas and cyclic block Thomas solves of the
whole lines (1e-12)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from tests.schur_helpers import ReferenceOps, block_lines, segment  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, cyclic, out):
    from paper_2004_13887_gb300 import schur
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, B, C, d = segment(block_lines(5, 24, 77, cyclic), rank, world)
        t = [torch.from_numpy(a) for a in (A, B, C, d)]
        x = schur.solve(*t, cyclic=cyclic, ops=ReferenceOps())
        out[rank] = x.numpy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("cyclic", [False, True])
def test_partitioned_block_thomas_on_cpu_ranks(world, cyclic):
    oracle.build()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), cyclic, out), nprocs=world, join=True,
                       start_method="spawn")
    x = np.concatenate([out[r] for r in range(world)], axis=1)
    A, B, C, d = block_lines(5, 24, 77, cyclic)
    for l in range(A.shape[0]):
        ref = oracle.block_thomas(A[l], B[l], C[l], d[l], cyclic=cyclic)
        err = np.max(np.abs(x[l] - ref)) / np.max(np.abs(ref))
        assert err <= 1e-12, (world, cyclic, l, err)
