"""The replica (N > 1) timing path of bench.py on CPU: world_size-2 gloo process group, max over
ranks, whole-job throughput = all ranks' units / slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = 1.0 + rank  # rank 1 is the slow one
    value, t = bench.aggregate(100.0, secs, world, dist, "cpu")
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, t in out:
        assert t == 2.0
        assert value == pytest.approx(world * 100.0 / 2.0)


def test_single_rank_aggregate():
    import bench
    value, t = bench.aggregate(50.0, 0.5, 1)
    assert value == 100.0 and t == 0.5
