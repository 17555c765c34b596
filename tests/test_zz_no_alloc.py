"""pgs_sort_static, the sort for callers that cannot allocate device memory
(allocator callbacks, plug-ins whose host owns every allocation): it must give
exactly what pgs_sort_copy with a caller workspace gives, call after call,
although every call reuses the same library-owned scratch array, and calls
after the first must leave the device's free memory unchanged.

Collected last on purpose, so a run that stops at the first failure has run
every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_sort(keys, vals, P, dtype, **opts):
    import torch
    from paper_1611_00463_gb300 import pgs
    k = pgs.as_device_keys(keys, dtype)
    v = torch.from_numpy(vals.view(np.int32)).cuda() if vals is not None else None
    bounds = torch.full((min(P, len(keys)) + 1,), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device="cuda")
    cfg = pgs.make_config(dtype=dtype, bucket_bounds=bounds, stats=st, **opts)
    rc = pgs.load().pgs_sort_static(k.data_ptr(), v.data_ptr() if v is not None else None, len(keys), P,
                                    torch.cuda.current_stream().cuda_stream, ctypes.byref(cfg))
    assert rc == 0, pgs.pgs_strerror(rc)
    torch.cuda.synchronize()
    return (pgs.to_numpy_keys(k, dtype), v.cpu().numpy().view(np.uint32) if v is not None else None,
            bounds.cpu().numpy(), pgs.pgs_get_stats(st))


def test_static_scratch_matches_workspace_sort_twice():
    from tests.gpu_helpers import gpu_sort
    cases = [("f32", inputs.zipf_dup_f32(50_000, seed=31), 16),
             ("u64", inputs.normal_lognormal_u64(1 << 16, seed=32), 64)]
    for dtype, keys, P in cases:          # two calls in a row on the shared scratch
        vals = inputs.index_payload(len(keys))
        want = gpu_sort(keys, vals, P, dtype)
        got_k, got_v, got_e, _ = _static_sort(keys, vals, P, dtype)
        assert np.array_equal(got_k, want["keys"])
        assert np.array_equal(got_v, want["vals"])
        assert np.array_equal(got_e, want["e"])


@pytest.mark.parametrize("splitters", ["sampled", "learned"])
@pytest.mark.parametrize("merge_ways", [2, 4])
@pytest.mark.parametrize("dtype", ["u32", "u64"])
@pytest.mark.parametrize("P", [63, 64])
def test_static_scratch_every_option_at_the_limits(dtype, merge_ways, splitters, P):
    # n = 2^16 keys is the largest request.  P = 64 has the most partitions;
    # P = 63 the most scratch with pairwise rounds (its bucket rounds are still
    # small enough for the offsets kernel to plan them all, each in its own
    # tables); learned splitters and four-way rounds need the most otherwise.
    import torch
    from tests.gpu_helpers import gpu_sort
    n = 1 << 16
    keys = inputs.exponential_u32(n, 33) if dtype == "u32" else inputs.normal_lognormal_u64(n, 34)
    vals = inputs.index_payload(n)
    opts = dict(merge_ways=merge_ways, splitters=splitters)
    want = gpu_sort(keys, vals, P, dtype, **opts)
    _static_sort(keys, vals, P, dtype, **opts)                 # warm-up: set-up and first launches
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        got_k, got_v, got_e, stats = _static_sort(keys, vals, P, dtype, **opts)
        assert np.array_equal(got_k, want["keys"])
        assert np.array_equal(got_v, want["vals"])
        assert np.array_equal(got_e, want["e"])
        assert stats["fallback"] == want["stats"]["fallback"]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "a call after the first changed the device's free memory"


def test_static_scratch_clamps_P_before_its_limit():
    from tests.gpu_helpers import gpu_sort
    keys = inputs.uniform_u32(40, 35)
    vals = inputs.index_payload(40)
    want = gpu_sort(keys, vals, 1000, "u32")                  # P clamps to n = 40 <= 64
    got_k, got_v, got_e, _ = _static_sort(keys, vals, 1000, "u32")
    assert np.array_equal(got_k, want["keys"]) and np.array_equal(got_v, want["vals"])
    assert np.array_equal(got_e, want["e"])


def test_static_scratch_rejects_sizes_beyond_its_limit():
    from paper_1611_00463_gb300 import pgs
    import torch
    lib = pgs.load()
    cfg = pgs.make_config()
    k = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.pgs_sort_static(k.data_ptr(), None, pgs.STATIC_MAX_KEYS + 1, 4, None,
                               ctypes.byref(cfg)) == pgs.PGS_ERR_UNSUPPORTED
    k2 = torch.zeros(200, dtype=torch.int32, device="cuda")
    assert lib.pgs_sort_static(k2.data_ptr(), None, 200, pgs.STATIC_MAX_P + 1, None,
                               ctypes.byref(cfg)) == pgs.PGS_ERR_UNSUPPORTED
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    cfg_ws = pgs.make_config(workspace=ws)
    assert lib.pgs_sort_static(k.data_ptr(), None, 8, 4, None, ctypes.byref(cfg_ws)) == pgs.PGS_ERR_INVALID
