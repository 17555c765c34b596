"""pgs_sort_static, the sort for callers that cannot allocate device memory
(allocator callbacks, plug-ins whose host owns every allocation): it must give
exactly what pgs_sort_copy with a caller workspace gives, call after call,
although every call reuses the same library-owned scratch array.

Collected last on purpose, so a run that stops at the first failure has run
every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_sort(keys, vals, P, dtype):
    import torch
    from paper_1611_00463_gb300 import pgs
    k = pgs.as_device_keys(keys, dtype)
    v = torch.from_numpy(vals.view(np.int32)).cuda() if vals is not None else None
    bounds = torch.full((min(P, len(keys)) + 1,), -1, dtype=torch.int64, device="cuda")
    cfg = pgs.make_config(dtype=dtype, bucket_bounds=bounds)
    rc = pgs.load().pgs_sort_static(k.data_ptr(), v.data_ptr() if v is not None else None, len(keys), P,
                                    torch.cuda.current_stream().cuda_stream, ctypes.byref(cfg))
    assert rc == 0, pgs.pgs_strerror(rc)
    torch.cuda.synchronize()
    return (pgs.to_numpy_keys(k, dtype), v.cpu().numpy().view(np.uint32) if v is not None else None,
            bounds.cpu().numpy())


def test_static_scratch_matches_workspace_sort_twice():
    from tests.gpu_helpers import gpu_sort
    cases = [("f32", inputs.zipf_dup_f32(50_000, seed=31), 16),
             ("u64", inputs.normal_lognormal_u64(1 << 16, seed=32), 64)]
    for dtype, keys, P in cases:          # two calls in a row on the shared scratch
        vals = inputs.index_payload(len(keys))
        want = gpu_sort(keys, vals, P, dtype)
        got_k, got_v, got_e = _static_sort(keys, vals, P, dtype)
        assert np.array_equal(got_k, want["keys"])
        assert np.array_equal(got_v, want["vals"])
        assert np.array_equal(got_e, want["e"])


def test_static_scratch_rejects_sizes_beyond_its_limit():
    from paper_1611_00463_gb300 import pgs
    import torch
    lib = pgs.load()
    cfg = pgs.make_config()
    k = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.pgs_sort_static(k.data_ptr(), None, pgs.STATIC_MAX_KEYS + 1, 4, None,
                               ctypes.byref(cfg)) == pgs.PGS_ERR_UNSUPPORTED
    assert lib.pgs_sort_static(k.data_ptr(), None, 8, pgs.STATIC_MAX_P + 1, None,
                               ctypes.byref(cfg)) == pgs.PGS_ERR_UNSUPPORTED
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    cfg_ws = pgs.make_config(workspace=ws)
    assert lib.pgs_sort_static(k.data_ptr(), None, 8, 4, None, ctypes.byref(cfg_ws)) == pgs.PGS_ERR_INVALID
