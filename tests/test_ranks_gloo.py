"""The multi-GPU path is replicas only: every rank runs the same workload on its own GPU and
the bench reports the units of all ranks over the slowest rank's time.  That host logic runs
here on two gloo ranks on CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.0 + 0.5 * rank  # rank 1 is the slower one
        t = bench.max_over_ranks(mine, dist)
        out[rank] = (t, bench.whole_job_rate(1000.0, world, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_units():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 1.5
        assert abs(rate - 2 * 1000.0 / 1.5) < 1e-9


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.0) == 2.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
