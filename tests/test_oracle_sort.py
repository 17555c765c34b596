"""Pins of the oracle's Part 1 (the sorted output) and of its key order."""
import itertools

import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs
from tests.pins import (check_stable_sorted, golden_lines, insertion_sort_order,
                        multiset_digest, total_order_key)


def test_f32_total_order_matches_ieee_golden():
    # The golden file lists binary32 patterns in IEEE 754 totalOrder.
    pats = np.array([int(ln.split()[0], 16) for ln in golden_lines("f32_total_order.txt")],
                    dtype=np.uint32)
    o = O.ord_bits(pats, "f32").astype(np.uint64)
    assert np.all(o[:-1] < o[1:])
    # The independent restatement in the pins agrees on the same sequence.
    t = total_order_key(pats, "f32").astype(np.uint64)
    assert np.all(t[:-1] < t[1:])


def test_f32_order_agrees_with_float_compare_on_numbers():
    g = np.random.default_rng(11)
    x = np.concatenate([g.standard_normal(5000).astype(np.float32) * 1e3,
                        np.array([np.inf, -np.inf, 0.0, -0.0, 1e-45, -1e-45, 3.4e38, -3.4e38], np.float32)])
    o = O.ord_bits(x.view(np.uint32), "f32")
    a, b = g.integers(0, len(x), 20000), g.integers(0, len(x), 20000)
    fa, fb = x[a].astype(np.float64), x[b].astype(np.float64)
    assert np.all(o[a][fa < fb] < o[b][fa < fb])
    assert np.all(o[a][fa > fb] > o[b][fa > fb])
    # Equal floats differ in bits only as -0 / +0, and -0 orders first.
    eq = (fa == fb) & (x[a].view(np.uint32) != x[b].view(np.uint32))
    neg_first = np.signbit(x[a][eq])
    assert np.all((o[a][eq] < o[b][eq]) == neg_first)


def test_ord_is_a_bijection():
    x = np.arange(0, 1 << 32, 65537, dtype=np.uint64).astype(np.uint32)
    o = O.ord_bits(x, "f32")
    assert len(np.unique(o)) == len(x)
    assert np.array_equal(O.ord_bits(x, "u32"), x)


@pytest.mark.parametrize("n", range(0, 7))
def test_brute_force_three_values(n):
    # Every input of length n over {0, 1, 2}, payload = index, against a
    # textbook stable insertion sort.
    for tup in itertools.product(range(3), repeat=n):
        keys = np.array(tup, dtype=np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        k, v = O.stable_sort(keys, vals, "u32")
        order = insertion_sort_order(list(tup))
        assert list(v) == order
        assert list(k) == [tup[i] for i in order]


def test_brute_force_float_specials():
    specials = np.array([0x80000000, 0x00000000, 0x7FC00000, 0xFFC00000, 0xBF800000],
                        dtype=np.uint32)
    rank = {int(b): i for i, b in enumerate([0xFFC00000, 0xBF800000, 0x80000000,
                                             0x00000000, 0x7FC00000])}
    for n in range(0, 5):
        for tup in itertools.product(range(len(specials)), repeat=n):
            keys = specials[list(tup)] if n else specials[:0]
            vals = np.arange(n, dtype=np.uint32)
            k, v = O.stable_sort(keys, vals, "f32")
            order = insertion_sort_order([rank[int(b)] for b in keys])
            assert list(v) == order


@pytest.mark.parametrize("name", ["uniform_u32", "normal_lognormal_u64", "zipf_dup_f32",
                                  "exponential_u32"])
def test_properties_on_workloads(name):
    dtype, keys, _ = inputs.workload(name, n=50000 + 13)
    vals = inputs.index_payload(len(keys))
    k, v = O.stable_sort(keys, vals, dtype)
    check_stable_sorted(keys, vals, k, v, dtype)
    assert multiset_digest(keys, vals) == multiset_digest(k, v)


def test_multiset_digest_detects_changes():
    keys = inputs.uniform_u32(1000, 5)
    vals = inputs.index_payload(1000)
    d = multiset_digest(keys, vals)
    k2 = keys.copy()
    k2[17] ^= 1
    assert multiset_digest(k2, vals) != d
    v2 = vals.copy()
    v2[3], v2[4] = v2[4], v2[3]
    assert multiset_digest(keys, v2) != d
