"""The multi-GPU path of bench.py is replicas only (the method has no data-path exchange on one
problem per GPU): every rank solves its own copy and the slowest rank sets the job time.  This
checks that aggregation with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_time = [0.25, 0.4][rank]                     # the second replica is slower
        t = bench.max_over_ranks(local_time, dist, "cpu")
        dist.barrier()
        out[rank] = (t, bench.job_throughput(world, 1_000_000, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, value = res[0]
    assert t == 0.4
    assert value == pytest.approx(2 * 1_000_000 / 0.4 / 1e9)


def test_without_a_process_group_the_local_value_stands():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3) == 0.3
    assert bench.job_throughput(1, 2e9, 2.0) == 1.0
