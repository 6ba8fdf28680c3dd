"""The multi-GPU path of bench.py is replicas only (independent copies of the
workload, no data exchange): its host logic -- the job time is the slowest
rank's, the throughput counts every rank's points -- run as two gloo ranks on
the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 7.5 * rank            # the ranks' own timings
        t = bench.max_over_ranks(ms, dist, device="cpu")
        out[rank] = (t, bench.job_throughput(1000, 4, world, t))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        t, v = out[r]
        assert t == 17.5
        assert v == pytest.approx(1000 * 4 * world / 17.5e-3)


def test_single_rank_is_its_own_time():
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_throughput(10, 3, 1, 1000.0) == pytest.approx(30.0)


def _partition_rank(rank, world, port, out):
    """each rank takes its share of the 64-instance ensemble and tells the others
    which instances it took (the only exchange, and only in this test)"""
    import numpy as np
    from inputs import cases
    from paper_2004_13887_gb300 import ensemble
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts = [int(np.prod(sp["n"])) for sp in cases.ensemble_specs()]
        mine = ensemble.partition(pts, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        out[rank] = (got, [sum(pts[q] for q in part) for part in got], pts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_ensemble_partition_across_ranks(world):
    """The ensemble partitioned across gloo ranks: each rank computes its share
    on its own; the shares are disjoint, cover every instance, agree between
    ranks, and their point counts are balanced to within the largest instance."""
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_partition_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    parts, loads, pts = out[0]
    for r in range(1, world):
        assert out[r][0] == parts
    flat = sorted(q for p in parts for q in p)
    assert flat == list(range(len(pts)))
    assert max(loads) - min(loads) <= max(pts), loads
