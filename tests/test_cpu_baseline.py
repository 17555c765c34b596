"""The multi-core CPU baseline (oracle/cpu_sort.c) gives exactly the oracle's
stable sort, on every key type, thread count and size edge (it is timed
beside the GPU, so it must compute the same result)."""
import numpy as np
import pytest

from oracle import cpu_sort
from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs


@pytest.mark.parametrize("name,n", [("zipf_dup_f32", 300_007), ("normal_lognormal_u64", 1 << 20),
                                    ("exponential_u32", 777), ("uniform_u32", 2), ("uniform_u32", 0),
                                    ("uniform_u32", 33)])
@pytest.mark.parametrize("threads", [1, 3, 8, 64])
def test_parallel_cpu_sort_is_the_stable_sort(name, n, threads):
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    k, v = cpu_sort.stable_sort(keys, vals, dtype, threads)
    wk, wv = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(k, wk) and np.array_equal(v, wv)


def test_keys_only_and_float_specials():
    specials = np.array([0x7FC00000, 0xFFC00000, 0x80000000, 0, 0x7F800000, 0xFF800000, 1, 0x80000001] * 50,
                        dtype=np.uint32)
    k, v = cpu_sort.stable_sort(specials, None, "f32", 4)
    assert v is None
    assert np.array_equal(k, O.stable_sort(specials, None, "f32")[0])
