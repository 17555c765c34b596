"""The paper's multi-processor protocol on CPU ranks (gloo, world size 2 and 3):
the ranks' buckets, concatenated, are the stable sort, and the bucket vector
equals the single-process one."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, name, n, s, q):
    import torch.distributed as dist

    from oracle.sharded import sharded_sort
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dtype, keys, _ = inputs.workload(name, n=n)
        vals = inputs.index_payload(n)
        b = O.run_bounds(n, world)
        k, v, e = sharded_sort(keys[b[rank]:b[rank + 1]], vals[b[rank]:b[rank + 1]], n, dtype, s)
        q.put((rank, k, v, e))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name,n,s", [(2, "zipf_dup_f32", 20_011, 64), (2, "normal_lognormal_u64", 9_000, 16),
                                            (3, "exponential_u32", 12_345, 32)])
def test_sharded_protocol_on_cpu_ranks(world, name, n, s):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, n, s, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    got_k = np.concatenate([r[1] for r in res])
    got_v = np.concatenate([r[2] for r in res])
    assert np.array_equal(got_k, want_k) and np.array_equal(got_v, want_v)
    ref = O.buckets(keys, world, dtype, samples_per_run=s)
    for r in res:
        assert np.array_equal(r[3], ref["e"])
    assert [len(r[1]) for r in res] == list(np.diff(ref["e"]))
