"""Launch-sequence replay (pgs_graph_cache): the second call with the same
arguments captures its launches into a CUDA graph and later identical calls
replay it.  Every call must still sort the data the buffers hold at that
moment, exactly as the oracle does."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu

GEN = {"u64": inputs.normal_lognormal_u64, "u32": inputs.exponential_u32, "f32": inputs.zipf_dup_f32}


def setup(n, P, dtype, **opts):
    import torch
    from paper_1611_00463_gb300 import pgs
    kin = pgs.as_device_keys(GEN[dtype](n, 1), dtype)
    vin = torch.zeros(n, dtype=torch.int32, device="cuda")
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    ws = pgs.workspace(n, P, pgs.make_config(dtype=dtype, **opts))
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device="cuda")
    bounds = torch.empty(min(P, n) + 1, dtype=torch.int64, device="cuda")
    cfg = pgs.make_config(dtype=dtype, workspace=ws, stats=st, bucket_bounds=bounds, **opts)
    return kin, vin, kout, vout, cfg, st, bounds


def fill(kin, vin, keys, dtype):
    import torch
    from paper_1611_00463_gb300 import pgs
    kin.copy_(pgs.as_device_keys(keys, dtype))
    vin.copy_(torch.arange(len(keys), dtype=torch.int32, device="cuda"))


def check(kout, vout, bounds, keys, P, dtype, vals=None):
    """The output equals the oracle's stable sort of (keys, vals) (vals: the
    input payload, default the input positions) and the bucket bounds equal the
    oracle's for this input order.  Returns the expected output."""
    import torch
    from paper_1611_00463_gb300 import pgs
    torch.cuda.synchronize()
    vals = np.arange(len(keys), dtype=np.uint32) if vals is None else vals
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(pgs.to_numpy_keys(kout, dtype), want_k)
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), want_v)
    assert np.array_equal(bounds.cpu().numpy().astype(np.uint64), O.buckets(keys, P, dtype)["e"].astype(np.uint64))
    return want_k, want_v


@pytest.mark.parametrize("dtype,n,P", [("u64", 300_011, 64), ("f32", 200_003, 16), ("u32", 70_001, 1),
                                       ("u32", 1_000_003, 256)])
def test_repeated_calls_sort_each_new_input(dtype, n, P):
    """Call 1 launches directly, call 2 captures and launches the graph, calls
    3-5 replay it, on fresh data every time; the statistics stay those of the
    launch sequence."""
    import torch
    from paper_1611_00463_gb300 import pgs
    kin, vin, kout, vout, cfg, st, bounds = setup(n, P, dtype)
    launches = None
    for i in range(5):
        keys = GEN[dtype](n, 100 + i)
        fill(kin, vin, keys, dtype)
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)
        check(kout, vout, bounds, keys, P, dtype)
        s = pgs.pgs_get_stats(st, torch.cuda.current_stream())
        assert s["error"] == 0
        launches = launches or s["launches"]
        assert s["launches"] == launches


def test_replay_on_other_streams_and_in_place():
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P, dtype = 250_007, 32, "u64"
    kin, vin, kout, vout, cfg, st, bounds = setup(n, P, dtype)
    streams = [torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.current_stream()]
    for i, s in enumerate(streams * 2):
        keys = GEN[dtype](n, 200 + i)
        fill(kin, vin, keys, dtype)
        torch.cuda.synchronize()
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream=s)
        check(kout, vout, bounds, keys, P, dtype)
    # In place: every other call re-sorts what the previous one left (sorted
    # keys, permuted payloads), the others sort fresh keys.
    prev = None
    for i in range(6):
        if i % 2 == 0:
            keys, vals = GEN[dtype](n, 300 + i), None
            fill(kin, vin, keys, dtype)
        else:
            keys, vals = prev
        pgs.pgs_sort(kin, vin, P, cfg)
        prev = check(kin, vin, bounds, keys, P, dtype, vals)


def test_cache_off_and_timer_launch_directly():
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P, dtype = 150_001, 16, "f32"
    kin, vin, kout, vout, cfg, st, bounds = setup(n, P, dtype, graph_cache="off")
    for i in range(3):
        keys = GEN[dtype](n, 400 + i)
        fill(kin, vin, keys, dtype)
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)
        check(kout, vout, bounds, keys, P, dtype)
    # With a timer every call records every launch (direct launches).
    tm = pgs.Timer(capacity=4096)
    ws = pgs.workspace(n, P, pgs.make_config(dtype=dtype))
    cfg_t = pgs.make_config(dtype=dtype, workspace=ws, stats=st, bucket_bounds=bounds, timer=tm)
    counts = []
    for i in range(3):
        keys = GEN[dtype](n, 500 + i)
        fill(kin, vin, keys, dtype)
        tm.reset()
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg_t)
        check(kout, vout, bounds, keys, P, dtype)
        recs, dropped = tm.read()
        counts.append(len(recs))
    assert counts[0] == counts[1] == counts[2] == pgs.pgs_get_stats(st, torch.cuda.current_stream())["launches"]


def test_more_keys_than_the_cache_holds():
    """20 different calls, each made three times in a row (direct, capture,
    replay), then the round again: graphs are evicted (some while still in
    flight) and rebuilt, and no result changes."""
    from paper_1611_00463_gb300 import pgs
    n, dtype = 60_013, "u32"
    setups = {P: setup(n, P, dtype) for P in range(2, 22)}
    for rep in range(2):
        for P, (kin, vin, kout, vout, cfg, st, bounds) in setups.items():
            for k in range(3):
                keys = GEN[dtype](n, 600 + 10 * P + 3 * rep + k)
                fill(kin, vin, keys, dtype)
                pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)
                check(kout, vout, bounds, keys, P, dtype)


def test_caller_capture_of_a_cached_call():
    """A caller may capture the call into its own graph after the library has
    cached it: inside a capture the library launches directly."""
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P, dtype = 180_001, 24, "u64"
    kin, vin, kout, vout, cfg, st, bounds = setup(n, P, dtype)
    for i in range(3):
        keys = GEN[dtype](n, 700 + i)
        fill(kin, vin, keys, dtype)
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)
        check(kout, vout, bounds, keys, P, dtype)
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=gs):
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream=gs)
    for i in range(2):
        keys = GEN[dtype](n, 800 + i)
        fill(kin, vin, keys, dtype)
        torch.cuda.synchronize()
        g.replay()
        check(kout, vout, bounds, keys, P, dtype)


def test_repeated_batched_calls_sort_each_new_input():
    """The batched sort goes through the same cache: one plan and one set of
    buffers, fresh keys on every call (direct, capture, replays), each
    instance exact; a new plan at the same buffers is not mistaken for it."""
    import torch
    from paper_1611_00463_gb300 import pgs
    sizes = [0, 1, 5000, 70_001, 123, 40_000]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(offsets[-1])
    for Pv in ([1, 1, 4, 32, 2, 16], None):
        bt = pgs.Batch(offsets, None if Pv is None else np.array(Pv, np.uint32), dtype="u64", with_vals=True)
        k = torch.empty(n, dtype=torch.int64, device="cuda")
        v = torch.empty(n, dtype=torch.int32, device="cuda")
        ko, vo = torch.empty_like(k), torch.empty_like(v)
        for i in range(4):
            keys = inputs.normal_lognormal_u64(n, 900 + i)
            k.copy_(pgs.as_device_keys(keys, "u64"))
            v.copy_(torch.arange(n, dtype=torch.int32, device="cuda"))
            bt.sort_copy(k, v, ko, vo)
            torch.cuda.synchronize()
            got_k, got_v = pgs.to_numpy_keys(ko, "u64"), vo.cpu().numpy().view(np.uint32)
            for a, b in zip(offsets[:-1].astype(int), offsets[1:].astype(int)):
                wk, wv = O.stable_sort(keys[a:b], np.arange(a, b, dtype=np.uint32), "u64")
                assert np.array_equal(got_k[a:b], wk) and np.array_equal(got_v[a:b], wv)
