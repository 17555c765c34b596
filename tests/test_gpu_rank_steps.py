"""The sharded sort's rank steps through the C ABI, checked against the oracle.

- pgs_merge_lists (step 6 on a receiving rank, Section IV-C): the stable merge
  of k sorted lists equals the oracle's Fig. 2 merge, for every key type, k
  from 1 to 300, empty lists, heavy ties, both merge widths.
- Steps 1-6 for G ranks run one after another in this process (the exchange
  done on the host): the splitters, the cut matrix and the bucket bounds equal
  the oracle's for P = G with every investigator rule, and every rank's merged
  bucket is its slice of the stable sort.
- The driver (paper_1611_00463_gb300.sharded) with 2 and 3 processes on this
  GPU, collectives through host memory over gloo (no kernel waits on another
  process's kernel)."""
import os
import socket

import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    from paper_1611_00463_gb300 import pgs
    return pgs.as_device_keys(a, dtype)


def _vals(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32"])
@pytest.mark.parametrize("merge_ways", [2, 4])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 13, 64, 300])
def test_merge_lists_is_the_stable_merge(dtype, merge_ways, k):
    import torch
    from paper_1611_00463_gb300 import pgs
    g = np.random.default_rng(1000 * k + merge_ways)
    lens = g.integers(0, 9000, size=k)
    lens[g.random(k) < 0.2] = 0                               # empty lists
    n = int(lens.sum())
    gen = {"u32": inputs.exponential_u32, "u64": inputs.normal_lognormal_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(max(n, 1), seed=k)[:n]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    lists = []
    for j in range(k):
        kk, vv = O.stable_sort(keys[off[j]:off[j + 1]], vals[off[j]:off[j + 1]], dtype)
        keys[off[j]:off[j + 1]], vals[off[j]:off[j + 1]] = kk, vv
        lists.append((kk, vv))
    want_k, want_v = O.balanced_merge(lists, dtype) if k else (keys, vals)
    kin, vin = _dev(keys, dtype), _vals(vals)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    cfg0 = pgs.make_config(dtype=dtype, merge_ways=merge_ways)
    ws = torch.empty(pgs.pgs_merge_workspace_bytes(n, k, cfg0), dtype=torch.uint8, device="cuda")
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device="cuda")
    cfg = pgs.make_config(dtype=dtype, merge_ways=merge_ways, workspace=ws, stats=st)
    pgs.pgs_merge_lists(kin, vin, off, kout, vout, cfg)
    torch.cuda.synchronize()
    assert np.array_equal(pgs.to_numpy_keys(kout, dtype), want_k)
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), want_v)
    assert np.array_equal(pgs.to_numpy_keys(kin, dtype), keys)         # inputs only read
    if n:
        assert pgs.pgs_get_stats(st)["error"] == 0


def test_merge_lists_rejects_bad_offsets():
    import ctypes
    import torch
    from paper_1611_00463_gb300 import pgs
    lib = pgs.load()
    k = torch.zeros(16, dtype=torch.int32, device="cuda")
    o = torch.zeros(16, dtype=torch.int32, device="cuda")
    cfg = pgs.make_config()
    for bad in ([1, 4, 16], [0, 9, 4, 16]):
        off = np.asarray(bad, dtype=np.uint64)
        assert lib.pgs_merge_lists(k.data_ptr(), None, off.ctypes.data, len(off) - 1, o.data_ptr(), None, None,
                                   ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID
    off = np.asarray([0, 8, 16], dtype=np.uint64)
    assert lib.pgs_merge_lists(k.data_ptr(), None, off.ctypes.data, 2, o.data_ptr(), None, None,
                               ctypes.byref(cfg)) == pgs.PGS_ERR_WORKSPACE


def run_rank_steps_in_one_process(keys, vals, G, dtype, investigator="rank", s=None, **opts):
    """Steps 1-6 for every rank in turn on this GPU; the all-gathers are
    concatenations and the all-to-all is done on the host."""
    import torch
    from paper_1611_00463_gb300 import pgs
    from paper_1611_00463_gb300.sharded import CudaSteps
    N = len(keys)
    b = O.run_bounds(N, G)
    sizes = [int(b[r + 1] - b[r]) for r in range(G)]
    steps = CudaSteps(dtype, "cuda", investigator=investigator, samples_per_run=s or 0, **opts)
    sk, sv = [], []
    for r in range(G):
        k, v = steps.local_sort(_dev(keys[b[r]:b[r + 1]], dtype), _vals(vals[b[r]:b[r + 1]]))
        sk.append(k)
        sv.append(v)
    s_used = steps.samples_per_run(G)
    smp = torch.cat([steps.samples(sk[r], s_used) for r in range(G)])
    spl = steps.splitters(smp, G)
    cnt_all = torch.cat([steps.counts(sk[r], spl, G) for r in range(G)])
    cut, e = steps.cuts(cnt_all, sizes, spl, G)
    cut_h = cut.cpu().numpy()
    out = []
    for dst in range(G):
        rk = torch.cat([sk[r][int(cut_h[r, dst]):int(cut_h[r, dst + 1])] for r in range(G)])
        rv = torch.cat([sv[r][int(cut_h[r, dst]):int(cut_h[r, dst + 1])] for r in range(G)])
        off = np.concatenate([[0], np.cumsum(cut_h[:, dst + 1] - cut_h[:, dst])]).astype(np.uint64)
        mk, mv = steps.merge(rk, rv, off)
        out.append((pgs.to_numpy_keys(mk, dtype), mv.cpu().numpy().view(np.uint32)))
    return s_used, pgs.to_numpy_keys(spl, dtype), cut_h, e.cpu().numpy(), out


@pytest.mark.parametrize("name,n,G", [("zipf_dup_f32", 300_007, 8), ("normal_lognormal_u64", 200_000, 5),
                                      ("exponential_u32", 250_000, 16), ("uniform_u32", 1000, 3)])
@pytest.mark.parametrize("investigator", ["rank", "equal", "off"])
def test_rank_steps_match_the_oracle(name, n, G, investigator):
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    variant = {"rank": O.INVESTIGATOR_RANK, "equal": O.INVESTIGATOR_EQUAL, "off": O.INVESTIGATOR_OFF}[investigator]
    s, spl, cut, e, out = run_rank_steps_in_one_process(keys, vals, G, dtype, investigator)
    ref = O.buckets(keys, G, dtype, samples_per_run=s, variant=variant)
    assert np.array_equal(O.ord_bits(spl, dtype), ref["splitters"])
    assert np.array_equal(cut, ref["cut"]) and np.array_equal(e, ref["e"])
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    for r, (k, v) in enumerate(out):
        assert np.array_equal(k, want_k[e[r]:e[r + 1]])
        assert np.array_equal(v, want_v[e[r]:e[r + 1]])


def test_rank_steps_guaranteed_mode_bound():
    n, G = 1 << 20, 16
    dtype, keys, _ = inputs.workload("zipf_dup_f32", n=n)
    vals = inputs.index_payload(n)
    s, _, _, e, _ = run_rank_steps_in_one_process(keys, vals, G, dtype, guaranteed=True)
    assert s == max(O.paper_samples_per_run(G, 4), O.guaranteed_samples_per_run(G, 0.05))
    m = n // G
    assert np.diff(e).max() < 1.05 * m + G


def _free_port():
    so = socket.socket()
    so.bind(("127.0.0.1", 0))
    port = so.getsockname()[1]
    so.close()
    return port


def _rank_main(rank, world, port, name, n, q):
    import torch
    import torch.distributed as dist
    from paper_1611_00463_gb300 import pgs
    from paper_1611_00463_gb300.sharded import sharded_sort
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        dtype, keys, _ = inputs.workload(name, n=n)
        vals = inputs.index_payload(n)
        b = O.run_bounds(n, world)
        bk, bv, e, cut = sharded_sort(_dev(keys[b[rank]:b[rank + 1]], dtype), _vals(vals[b[rank]:b[rank + 1]]),
                                      dtype=dtype, stage_on_host=True)
        torch.cuda.synchronize()
        q.put((rank, pgs.to_numpy_keys(bk, dtype), bv.cpu().numpy().view(np.uint32), e.cpu().numpy(),
               cut.cpu().numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name,n", [(2, "zipf_dup_f32", 400_003), (3, "normal_lognormal_u64", 300_000)])
def test_sharded_driver_processes_on_one_gpu(world, name, n):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    ref = O.buckets(keys, world, dtype)
    for rank, k, v, e, cut in got:
        assert np.array_equal(e, ref["e"]) and np.array_equal(cut, ref["cut"])
        assert np.array_equal(k, want_k[e[rank]:e[rank + 1]]) and np.array_equal(v, want_v[e[rank]:e[rank + 1]])
