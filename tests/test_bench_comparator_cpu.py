"""The bench's library comparator maps keys to signed integers whose order is
the key order (float32 by IEEE totalOrder): torch.sort(stable=True) on the
mapped keys then equals the oracle's stable sort, and the map is its own
inverse."""
import numpy as np
import pytest
import torch

import bench
from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs


@pytest.mark.parametrize("dtype,gen", [("u64", inputs.normal_lognormal_u64), ("u32", inputs.exponential_u32),
                                       ("f32", inputs.zipf_dup_f32), ("u32", lambda n, s: inputs.structured_u32("extremes", n, s))])
def test_mapped_torch_sort_is_the_stable_sort(dtype, gen):
    keys = gen(20000, 3)
    raw = torch.from_numpy(keys.view(np.int64 if dtype == "u64" else np.int32).copy())
    mapped = bench.order_as_signed(raw, dtype)
    assert torch.equal(bench.order_as_signed(mapped, dtype), raw)
    sk, idx = torch.sort(mapped, stable=True)
    want_k, want_v = O.stable_sort(keys, np.arange(len(keys), dtype=np.uint32), dtype)
    assert np.array_equal(bench.order_as_signed(sk, dtype).numpy().view(want_k.dtype), want_k)
    assert np.array_equal(idx.numpy().astype(np.uint32), want_v)


def test_clock_summary_keeps_the_timed_window():
    """Samples before the timed region are dropped; the one right after it is
    kept (it covers the region's last interval); throttle reasons are read."""
    c = bench.ClockSampler(0)
    row = "{sm}, 2070, 900.0, 0x0, Not Active, Not Active, {thermal}, Not Active"
    c.lines = [(0.0, row.format(sm=1200, thermal="Not Active")),          # before: warm-up
               (1.0, row.format(sm=2070, thermal="Not Active")),
               (1.1, row.format(sm=2055, thermal="Active")),
               (1.3, row.format(sm=2070, thermal="Not Active")),          # first after the end
               (2.0, row.format(sm=900, thermal="Not Active"))]           # later: dropped
    c.t0, c.t1 = 0.5, 1.2
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_thermal_slowdown"]
