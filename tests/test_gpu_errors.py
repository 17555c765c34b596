"""Failure paths of the C ABI on the GPU, made without any GPU fault.

A bounded device-side wait is made to run out by fault injection (a merge tile
announces its copies to its barrier and issues none, so nothing is in flight
and nothing ever completes the barrier): the kernel gives up after
cfg.spin_limit, the call's statistics report PGS_ERR_TIMEOUT, and the context
stays usable.  Every entry point also leaves the caller's current device as it
found it."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sorted_ok(kout, vout, keys, vals, dtype="u32"):
    from paper_1611_00463_gb300 import pgs
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(pgs.to_numpy_keys(kout, dtype), want_k)
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), want_v)


@pytest.mark.parametrize("merge_ways", [2, 4])
def test_wait_timeout_is_reported_and_the_next_sort_is_correct(merge_ways):
    import torch
    from paper_1611_00463_gb300 import pgs
    n, P = 200_003, 16                        # runs of 12,500 keys: the first merge round is step 1's
    keys = inputs.uniform_u32(n, 11)
    vals = inputs.index_payload(n)
    kin = pgs.as_device_keys(keys, "u32")
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device="cuda")
    ws = pgs.workspace(n, P, pgs.make_config(merge_ways=merge_ways))
    stream = torch.cuda.current_stream()
    limit_ns = 1_000_000                      # 1 ms instead of the default 2 s
    cfg = pgs.make_config(workspace=ws, stats=st, merge_ways=merge_ways, spin_limit=limit_ns,
                          fault_inject="wait_timeout", graph_cache="off")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream)
    e1.record(stream)
    with pytest.raises(pgs.PgsError) as err:
        pgs.pgs_get_stats(st, stream)
    assert err.value.status == pgs.PGS_ERR_TIMEOUT
    ms = e0.elapsed_time(e1)
    assert 1.0 <= ms < 500.0, f"the injected wait took {ms} ms: spin_limit not honoured"
    # The context is usable: the same workspace sorts correctly on the same stream.
    cfg_ok = pgs.make_config(workspace=ws, stats=st, merge_ways=merge_ways)
    pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg_ok, stream)
    stats = pgs.pgs_get_stats(st, stream)
    assert stats["error"] == 0
    _sorted_ok(kout, vout, keys, vals)


def test_fault_inject_rejects_unknown_values():
    import ctypes
    import torch
    from paper_1611_00463_gb300 import pgs
    k = torch.zeros(16, dtype=torch.int32, device="cuda")
    ws = pgs.workspace(16, 2, pgs.make_config())
    cfg = pgs.make_config(workspace=ws)
    cfg.fault_inject = 7
    assert pgs.load().pgs_sort(k.data_ptr(), None, 16, 2, None, ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID


def test_current_device_is_left_as_found():
    import torch
    from paper_1611_00463_gb300 import pgs
    from tests.gpu_helpers import gpu_sort
    torch.cuda.set_device(0)
    n, P = 50_000, 8
    keys = inputs.normal_lognormal_u64(n, 3)
    vals = inputs.index_payload(n)
    gpu_sort(keys, vals, P, "u64")
    assert torch.cuda.current_device() == 0
    kd = pgs.as_device_keys(np.sort(keys), "u64")
    pos = torch.empty(100, dtype=torch.int64, device="cuda")
    pgs.pgs_search(kd, kd[:100].clone(), pos, dtype="u64")
    assert torch.cuda.current_device() == 0
    hk = torch.from_numpy(keys.view(np.int64)).pin_memory()
    hv = torch.from_numpy(vals.view(np.int32)).pin_memory()
    pgs.sort(hk, hv, P, dtype="u64")
    assert torch.cuda.current_device() == 0
    b = pgs.Batch([0, 1000, n], dtype="u64")
    kb = pgs.as_device_keys(keys, "u64")
    vb = torch.from_numpy(vals.view(np.int32)).cuda()
    b.sort(kb, vb)
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == 0
