"""The sharded sort's choreography (paper_1611_00463_gb300.sharded: size,
sample and count all-gathers, the investigator's cut matrix on every rank, the
all-to-all of segments, the merge on the receiver) on CPU ranks over gloo,
world sizes 2 and 3, with the rank steps computed by the oracle: the ranks'
buckets concatenated are the stable sort, and the bucket vector and cut matrix
are the single-process oracle's for P = world size."""
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
    import torch
    import torch.distributed as dist

    from paper_1611_00463_gb300.sharded import sharded_sort
    from tests.sharded_steps import OracleSteps, to_np, to_t
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dtype, keys, _ = inputs.workload(name, n=n)
        vals = inputs.index_payload(n)
        b = O.run_bounds(n, world)
        k = to_t(keys[b[rank]:b[rank + 1]], dtype)
        v = torch.from_numpy(vals[b[rank]:b[rank + 1]].view(np.int32).copy())
        bk, bv, e, cut = sharded_sort(k, v, dtype=dtype, steps=OracleSteps(dtype, s))
        q.put((rank, to_np(bk, dtype), bv.numpy().view(np.uint32), e.numpy(), cut.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name,n,s", [(2, "zipf_dup_f32", 20_011, 64), (3, "normal_lognormal_u64", 9_001, 16),
                                            (3, "exponential_u32", 12_000, 5), (2, "uniform_u32", 7, 3)])
def test_sharded_driver_on_cpu_ranks(world, name, n, s):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, n, s, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    ref = O.buckets(keys, world, dtype, samples_per_run=s)
    for rank, k, v, e, cut in got:
        assert np.array_equal(e, ref["e"]) and np.array_equal(cut, ref["cut"])
        assert np.array_equal(k, want_k[e[rank]:e[rank + 1]])
        assert np.array_equal(v, want_v[e[rank]:e[rank + 1]])
