"""Pins of the oracle's lookups on sorted output: brute-force counts, float
total order, bucket ranges and provenance closed forms."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs
from tests.pins import golden_lines


def brute_count(keys_ord, q, inclusive):
    return sum(1 for k in keys_ord if (k <= q if inclusive else k < q))


@pytest.mark.parametrize("seed", range(5))
def test_search_counts_by_brute_force(seed):
    g = np.random.default_rng(seed)
    keys = np.sort(g.integers(0, 9, size=int(g.integers(0, 40))).astype(np.uint32))
    queries = g.integers(0, 10, size=30).astype(np.uint32)
    lo = O.search(keys, queries, "u32", "left")
    hi = O.search(keys, queries, "u32", "right")
    for q, a, b in zip(queries, lo, hi):
        assert a == brute_count(keys, q, False) and b == brute_count(keys, q, True)
        assert b - a == int(np.sum(keys == q))


def test_search_float_total_order():
    pats = np.array([int(ln.split()[0], 16) for ln in golden_lines("f32_total_order.txt")], np.uint32)
    # The golden list is in totalOrder: every pattern's lower bound is its index
    # among the distinct patterns, and -0 / +0 and the NaN signs are distinct keys.
    pos = O.search(pats, pats, "f32", "left")
    assert list(pos) == list(range(len(pats)))
    assert list(O.search(pats, pats, "f32", "right")) == list(range(1, len(pats) + 1))


def test_bucket_of_closed_form():
    e = np.array([0, 3, 3, 7, 10], np.int64)           # bucket 1 is empty
    pos = np.array([0, 2, 3, 6, 7, 9, 10], np.int64)
    assert list(O.bucket_of(pos, e)) == [0, 0, 2, 2, 3, 3, 4]


def test_search_on_a_sorted_workload_and_its_buckets():
    n, P = 20_000, 16
    keys = inputs.zipf_dup_f32(n, 7)
    res = O.sample_sort(keys, np.arange(n, dtype=np.uint32), P, "f32", threads=4)
    q = inputs.zipf_dup_f32(500, 8)
    pos = O.search(res["keys"], q, "f32", "left")
    b = O.bucket_of(pos, res["e"])
    o = O.ord_bits(res["keys"], "f32")
    qo = O.ord_bits(q, "f32")
    for p_, bb, qq in zip(pos, b, qo):
        assert (p_ == 0 or o[p_ - 1] < qq) and (p_ == n or o[p_] >= qq)
        assert (p_ == n and bb == P) or (res["e"][bb] <= p_ < res["e"][bb + 1])


def test_provenance_closed_form():
    r, i = O.provenance(np.arange(10, dtype=np.uint32), 10, 3)     # runs [0,3), [3,6), [6,10)
    assert list(r) == [0, 0, 0, 1, 1, 1, 2, 2, 2, 2]
    assert list(i) == [0, 1, 2, 0, 1, 2, 0, 1, 2, 3]
    r, i = O.provenance(np.array([4, 0], np.uint32), 5, 9)          # P clamps to 5: one key per run
    assert list(r) == [4, 0] and list(i) == [0, 0]
