"""The bench's multi-GPU path on CPU: replicas over a world_size-2 gloo process group.

With N > 1 every rank advances its own suspension (no collective on the data path); the
only collective is the max over ranks of the timed region, and the job's throughput is
N x steps / (slowest rank's time).  The reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank,) + bench.replica_throughput(times[rank], 5, world, dist, "cpu"))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [2.0, 3.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max in res:
        assert t_max == 3.0
        assert value == pytest.approx(2 * 5 / 3.0)


def test_single_rank_throughput():
    import bench
    assert bench.replica_throughput(2.5, 5, 1) == (2.0, 2.5)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, ref_bodies=4)
    assert bench.run_reference(args, world=2, rank=1) == 0
    assert capsys.readouterr().out == ""
