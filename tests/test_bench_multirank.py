"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks reduce
their step times with max-over-ranks and report whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slowest replica
    tmax = bench.max_over_ranks(torch, dist, local_ms, "cpu")
    value = bench.replica_throughput(1000, world, tmax)
    out[rank] = (tmax, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tmax, value = res[rank]
        assert tmax == 15.0
        assert abs(value - 2 * 1000 / 0.015) < 1e-6


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(torch, None, 3.5, "cpu") == 3.5
    assert bench.replica_throughput(10, 1, 1000.0) == 10.0
