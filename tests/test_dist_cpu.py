"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
replicas report the slowest rank's time and the whole-job aggregate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")        # rank 1 is the slowest
    rate = bench.aggregate_rate(1e9, world, t)
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 2e9 / 2.5) < 1e-3 for r in res)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.aggregate_rate(10.0, 1, 2.0) == 5.0
