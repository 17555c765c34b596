"""pgs_sort_host (host buffers in and out, copies inside the call) against the oracle.

The sorted keys and payloads must equal the oracle's stable sort bit for bit
and the bucket vector must equal the oracle's step 1-4 computation, for run
groups of every shape (fewer runs than copy groups, ragged groups, one run),
the default copies (one piece each way below 2^25 keys, groups above) and the
explicit GROUPS and AT_END forms, pinned and pageable host memory, keys only
and with payloads.
"""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu

TILE = 17 * 256


def host_tensor(a, dtype, pinned):
    import torch
    view = np.ascontiguousarray(a).view(np.int64 if dtype == "u64" else np.int32)
    t = torch.from_numpy(view.copy())
    return t.pin_memory() if pinned else t


def run_host(keys, vals, P, dtype, pinned=True, **opts):
    import torch
    from paper_1611_00463_gb300 import pgs
    hk = host_tensor(keys, dtype, pinned)
    hv = host_tensor(vals, "u32", pinned) if vals is not None else None
    ko, vo, info = pgs.sort(hk, hv, P, dtype=dtype, **opts)
    torch.cuda.synchronize()
    got_k = ko.numpy().view(np.uint64 if dtype == "u64" else np.uint32)
    got_v = vo.numpy().view(np.uint32) if vo is not None else None
    e = info["bucket_bounds"].cpu().numpy()
    return got_k, got_v, e, hk, hv


def check(keys, vals, P, dtype, **kw):
    got_k, got_v, e, hk, hv = run_host(keys, vals, P, dtype, **kw)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(got_k, want_k), "keys differ"
    if vals is not None:
        assert np.array_equal(got_v, want_v), "payload differs"
    assert np.array_equal(e, O.buckets(keys, P, dtype)["e"]), "bucket bounds differ"
    # inputs are left unchanged
    assert np.array_equal(hk.numpy().view(got_k.dtype), np.ascontiguousarray(keys).view(got_k.dtype))


@pytest.mark.parametrize("dtype,n,P", [("u64", 300_007, 128), ("u32", 3 * TILE + 77, 3), ("f32", 200_003, 16),
                                       ("u32", 50_000, 1), ("u64", 7, 64), ("u32", 1, 5), ("f32", 123_457, 11),
                                       # from 2^25 keys the default copies go in groups of runs and of buckets
                                       ("u32", (1 << 25) + 12_345, 24)])
def test_host_sort_matches_oracle(dtype, n, P):
    gen = {"u32": inputs.exponential_u32, "u64": inputs.normal_lognormal_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(n, n % 89 + 1)
    check(keys, inputs.index_payload(n), P, dtype)


def test_host_sort_pageable_memory_and_keys_only():
    n, P = 150_001, 24
    keys = inputs.normal_lognormal_u64(n, 5)
    check(keys, inputs.index_payload(n), P, "u64", pinned=False)
    got_k, got_v, e, _, _ = run_host(keys, None, P, "u64")
    assert got_v is None
    assert np.array_equal(got_k, O.stable_sort(keys, None, "u64")[0])


def test_host_sort_equals_device_sort():
    from tests.gpu_helpers import gpu_sort
    n, P = 400_000, 40
    keys = inputs.zipf_dup_f32(n, 8)
    vals = inputs.index_payload(n)
    dev = gpu_sort(keys, vals, P, "f32")
    got_k, got_v, e, _, _ = run_host(keys, vals, P, "f32")
    assert np.array_equal(got_k, dev["keys"]) and np.array_equal(got_v, dev["vals"])
    assert np.array_equal(e, dev["e"])


def test_host_sort_rejects_device_buffers_and_small_workspace():
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P = 10_000, 4
    hk = torch.zeros(n, dtype=torch.int32).pin_memory()
    ko = torch.zeros(n, dtype=torch.int32).pin_memory()
    dk = torch.zeros(n, dtype=torch.int32, device="cuda")
    cfg0 = pgs.make_config()
    ws = torch.empty(pgs.pgs_host_workspace_bytes(n, P, cfg0), dtype=torch.uint8, device="cuda")
    cfg = pgs.make_config(workspace=ws)
    rc = pgs.load().pgs_sort_host(dk.data_ptr(), None, ko.data_ptr(), None, n, P, pgs._stream(None),
                                  pgs.ctypes.byref(cfg))
    assert rc == pgs.PGS_ERR_INVALID
    with pytest.raises(ValueError):
        pgs.pgs_sort_host(dk, None, ko, None, P, cfg)
    small = pgs.make_config(workspace=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    with pytest.raises(pgs.PgsError) as ei:
        pgs.pgs_sort_host(hk, None, ko, None, P, small)
    assert ei.value.status == pgs.PGS_ERR_WORKSPACE
    assert pgs.pgs_host_workspace_bytes(n, P, cfg0) > pgs.pgs_workspace_bytes(n, P, cfg0)


@pytest.mark.parametrize("copy_back", ["groups", "end", "auto"])
def test_host_sorts_in_flight_on_two_streams(copy_back):
    """Consecutive calls on two streams with their own workspaces overlap on the
    GPU (one call's copy in during the other's merges); each result is exact.
    With copy_back = "end" no call waits, so all six are queued at once and a
    lane's next call must wait for its previous one on the device, and so
    with "auto" at this size (one copy each way)."""
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P = 600_011, 32
    sets = [inputs.normal_lognormal_u64(n, 30 + i) for i in range(6)]
    vals = inputs.index_payload(n)
    hv = host_tensor(vals, "u32", True)
    cfg0 = pgs.make_config(dtype="u64", copy_back=copy_back)
    lanes = []
    for _ in range(2):
        ws = torch.empty(pgs.pgs_host_workspace_bytes(n, P, cfg0), dtype=torch.uint8, device="cuda")
        lanes.append((torch.cuda.Stream(), pgs.make_config(dtype="u64", workspace=ws, copy_back=copy_back), ws))
    outs = []
    for i, keys in enumerate(sets):
        s, cfg, _ = lanes[i % 2]
        hk = host_tensor(keys, "u64", True)
        ko = torch.empty_like(hk).pin_memory()
        vo = torch.empty_like(hv).pin_memory()
        pgs.pgs_sort_host(hk, hv, ko, vo, P, cfg, stream=s)
        outs.append((hk, ko, vo))
    torch.cuda.synchronize()
    for keys, (_, ko, vo) in zip(sets, outs):
        want_k, want_v = O.stable_sort(keys, vals, "u64")
        assert np.array_equal(ko.numpy().view(np.uint64), want_k)
        assert np.array_equal(vo.numpy().view(np.uint32), want_v)


@pytest.mark.parametrize("opts,P", [({"merge_ways": 4}, 64), ({"merge_ways": 4}, 32), ({"exchange": "scatter"}, 16),
                                    ({"exchange": "scatter", "merge_ways": 4}, 128), ({"splitters": "learned"}, 24),
                                    ({"investigator": "local"}, 12), ({"guaranteed": True}, 40), ({}, 2), ({}, 3),
                                    ({"copy_back": "end"}, 64), ({"copy_back": "end", "merge_ways": 4}, 5),
                                    ({"copy_back": "end"}, 1)])
def test_host_sort_bucket_groups_with_every_option(opts, P):
    """Step 6 in bucket groups under four-way rounds, the scatter exchange,
    learned splitters and every P shape (bucket rounds after the first: none,
    odd, even), with the copies in groups (copy_back GROUPS unless the case
    says AT_END)."""
    n = 4 * TILE * 9 + 123
    keys = inputs.zipf_dup_f32(n, P)
    vals = inputs.index_payload(n)
    got_k, got_v, e, _, _ = run_host(keys, vals, P, "f32", **{"copy_back": "groups", **opts})
    if opts.get("investigator") == "local":
        ref = O.sample_sort(keys, vals, P, "f32", variant=O.INVESTIGATOR_LOCAL)
        assert np.array_equal(got_k, ref["keys"]) and np.array_equal(got_v, ref["vals"])
        assert np.array_equal(e, ref["e"])
        return
    want_k, want_v = O.stable_sort(keys, vals, "f32")
    assert np.array_equal(got_k, want_k) and np.array_equal(got_v, want_v)
    if "splitters" not in opts:
        s = (max(O.paper_samples_per_run(P, 4), O.guaranteed_samples_per_run(P, 0.05))
             if opts.get("guaranteed") else None)
        assert np.array_equal(e, O.buckets(keys, P, "f32", samples_per_run=s)["e"])
