"""The batched sort (many instances, one launch sequence) against the oracle,
instance by instance, and replayed from a CUDA graph."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def make_batch(num, seed, hi, dtype="u64", mu=7.0, extra=()):
    sizes = np.concatenate([inputs.batched_sizes(num - len(extra), seed=seed, lo=1, hi=hi, mu=mu, sigma=1.5),
                            np.array(extra, dtype=np.int64)])
    offsets = np.zeros(num + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    if dtype == "u64":
        keys = np.concatenate([inputs.batched_instance_keys(i, int(sizes[i])) for i in range(num)])
    elif dtype == "f32":
        keys = np.concatenate([inputs.zipf_dup_f32(int(sizes[i]), seed=i) for i in range(num)])
    else:
        keys = np.concatenate([inputs.exponential_u32(int(sizes[i]), seed=i, scale=1e3) for i in range(num)])
    vals = np.arange(n, dtype=np.uint32)
    return offsets, keys, vals


def run_batch(offsets, keys, vals, P, dtype, graph=False, **opts):
    import torch
    from paper_1611_00463_gb300 import pgs
    bt = pgs.Batch(offsets, P, dtype=dtype, with_vals=vals is not None, **opts)
    k = pgs.as_device_keys(keys, dtype)
    v = torch.from_numpy(vals.view(np.int32)).cuda() if vals is not None else None
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device="cuda")
    cfg = bt.config(stats=st)
    if graph:
        k0, v0 = k.clone(), (v.clone() if v is not None else None)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.sort(k, v, stream=s, cfg=cfg)
        torch.cuda.synchronize()
        for _ in range(2):                       # replay twice from the same unsorted input
            k.copy_(k0)
            if v is not None:
                v.copy_(v0)
            g.replay()
        torch.cuda.synchronize()
    else:
        bt.sort(k, v, cfg=cfg)
        torch.cuda.synchronize()
    stats = pgs.pgs_get_stats(st)
    return (pgs.to_numpy_keys(k, dtype), v.cpu().numpy().view(np.uint32) if v is not None else None, stats)


def check(offsets, keys, vals, got_k, got_v, P, dtype, stats=None, **ref_opts):
    mx, mn = 0, None
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        wk, wv = O.stable_sort(keys[a:b], None if vals is None else vals[a:b], dtype)
        assert np.array_equal(got_k[a:b], wk), f"instance {i} keys"
        if vals is not None:
            assert np.array_equal(got_v[a:b], wv), f"instance {i} vals"
        if b > a:
            Pi = P[i] if P is not None else None
            res = O.buckets(keys[a:b], Pi, dtype, **ref_opts)
            mx = max(mx, res["stats"]["max"])
            mn = res["stats"]["min"] if mn is None else min(mn, res["stats"]["min"])
    if stats is not None:
        assert stats["max_bucket"] == mx and stats["min_bucket"] == mn


@pytest.mark.parametrize("dtype", ["u64", "u32", "f32"])
def test_batch_explicit_partitions(dtype):
    offsets, keys, vals = make_batch(40, seed=3, hi=60_000, dtype=dtype)
    rng = np.random.default_rng(5)
    P = rng.integers(1, 40, size=40).astype(np.uint32)
    got_k, got_v, st = run_batch(offsets, keys, vals, P, dtype)
    Peff = [max(1, min(int(P[i]), int(offsets[i + 1] - offsets[i]))) for i in range(40)]
    check(offsets, keys, vals, got_k, got_v, Peff, dtype, stats=st)


def test_batch_auto_partitions_and_keys_only():
    from paper_1611_00463_gb300 import pgs
    offsets, keys, vals = make_batch(25, seed=9, hi=400_000, extra=(300_000, 140_000))
    sizes = np.diff(offsets)
    P = [pgs.pgs_batch_auto_partitions(int(x)) for x in sizes]
    assert max(P) >= 2
    got_k, _, _ = run_batch(offsets, keys, None, None, "u64")
    check(offsets, keys, None, got_k, None, [max(1, min(p, int(s))) for p, s in zip(P, sizes)], "u64")


def test_batch_empty_and_tiny_instances():
    sizes = [0, 1, 2, 0, 5, 4352, 4353, 0, 17]
    offsets = np.zeros(len(sizes) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    keys = inputs.structured_u32("few", n, seed=2)
    vals = np.arange(n, dtype=np.uint32)
    P = np.array([3, 1, 4, 2, 8, 16, 3, 1, 17], dtype=np.uint32)
    got_k, got_v, _ = run_batch(offsets, keys, vals, P, "u32")
    Peff = [max(1, min(int(p), int(s))) for p, s in zip(P, sizes)]
    check(offsets, keys, vals, got_k, got_v, Peff, "u32")


def test_batch_graph_replay():
    offsets, keys, vals = make_batch(30, seed=11, hi=100_000)
    rng = np.random.default_rng(7)
    P = rng.integers(1, 20, size=30).astype(np.uint32)
    got_k, got_v, st = run_batch(offsets, keys, vals, P, "u64", graph=True)
    Peff = [max(1, min(int(P[i]), int(offsets[i + 1] - offsets[i]))) for i in range(30)]
    check(offsets, keys, vals, got_k, got_v, Peff, "u64", stats=st)


def test_single_sort_is_batch_of_one():
    from tests.gpu_helpers import gpu_sort
    n, P = 70_001, 24
    keys = inputs.normal_lognormal_u64(n, 4)
    vals = inputs.index_payload(n)
    offsets = np.array([0, n], dtype=np.uint64)
    got_k, got_v, st = run_batch(offsets, keys, vals, [P], "u64")
    single = gpu_sort(keys, vals, P, "u64")
    assert np.array_equal(got_k, single["keys"]) and np.array_equal(got_v, single["vals"])
    assert st["max_bucket"] == single["stats"]["max_bucket"]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_merge_tile_shape_gives_the_stable_sort(variant):
    from tests.gpu_helpers import gpu_sort
    n = 90_017
    keys = inputs.zipf_dup_f32(n, 12)
    vals = inputs.index_payload(n)
    got = gpu_sort(keys, vals, 20, "f32", tile_variant=variant)
    want_k, want_v = O.stable_sort(keys, vals, "f32")
    assert np.array_equal(got["keys"], want_k) and np.array_equal(got["vals"], want_v)
    assert np.array_equal(got["e"], O.buckets(keys, 20, "f32")["e"])


def test_tuner_and_out_of_place_batch():
    import torch
    from paper_1611_00463_gb300 import pgs
    offsets, keys, vals = make_batch(30, seed=2, hi=200_000)
    P = np.random.default_rng(1).integers(1, 16, size=30).astype(np.uint32)
    bt = pgs.Batch(offsets, P, dtype="u64", with_vals=True)
    sk = torch.empty(bt.n, dtype=torch.int64, device="cuda")
    sv = torch.empty(bt.n, dtype=torch.int32, device="cuda")
    chosen, ms = bt.tune(sk, sv)
    assert 0 <= chosen < pgs.TILE_VARIANTS and all(m > 0 for m in ms) and ms[chosen] == min(ms)
    kin = pgs.as_device_keys(keys, "u64")
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    bt.sort_copy(kin, vin, kout, vout)
    torch.cuda.synchronize()
    assert np.array_equal(pgs.to_numpy_keys(kin, "u64"), keys)          # input untouched
    Peff = [max(1, min(int(P[i]), int(offsets[i + 1] - offsets[i]))) for i in range(30)]
    check(offsets, keys, vals, pgs.to_numpy_keys(kout, "u64"), vout.cpu().numpy().view(np.uint32), Peff, "u64")
