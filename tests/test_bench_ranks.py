"""Multi-process path of bench.py on CPU: two gloo ranks, replicas of the workload; the job's
time is the slowest rank's and its units are the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.reduce_over_ranks(10.0 * (rank + 1), 100 + rank)
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0, 201), (1, 20.0, 201)]


def test_reduce_without_distributed_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7) == (3.5, 7)
