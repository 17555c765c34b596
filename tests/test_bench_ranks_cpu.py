"""bench.py's multi-rank arithmetic on CPU ranks (gloo, world size 2): every
rank learns the slowest rank's time, and the whole-job rate counts every
rank's keys over that time (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank                       # rank 1 is the slowest
        slowest = bench.max_over_ranks(mine, torch.device("cpu"), world)
        q.put((rank, slowest, bench.whole_job_rate(1 << 20, world, slowest * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_whole_job_rate():
    import bench
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * (1 << 20) / 15e-3 / 1e9)
    assert bench.max_over_ranks(3.0, None, 1) == 3.0
