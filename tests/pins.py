"""Checks that pin a sort result without re-running any implementation of it.

Used against the oracle (its pins) and against the CUDA path (properties that
hold at any size).  Nothing here imports the oracle or the CUDA binding.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_lines(name: str) -> list[str]:
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]


def total_order_key(bits: np.ndarray, dtype: str) -> np.ndarray:
    """An order-preserving integer image of the key, written independently of
    the oracle: for float32 a negative pattern maps to 0x7FFFFFFF - magnitude and a
    non-negative one to 0x80000000 + pattern (IEEE 754 totalOrder)."""
    if dtype != "f32":
        return bits
    b = bits.astype(np.uint64)
    neg = (b >> np.uint64(31)) & np.uint64(1)
    mag = b & np.uint64(0x7FFFFFFF)
    return np.where(neg == 1, np.uint64(0x7FFFFFFF) - mag, np.uint64(0x80000000) + b).astype(np.uint32)


def insertion_sort_order(keys: list) -> list[int]:
    """Textbook stable insertion sort; returns the input positions in output order."""
    order: list[int] = []
    for i, k in enumerate(keys):
        j = len(order)
        while j > 0 and keys[order[j - 1]] > k:     # strict: equal keys never pass each other
            j -= 1
        order.insert(j, i)
    return order


def mix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser, used to hash (key, val) pairs into a multiset digest."""
    z = x.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def multiset_digest(keys: np.ndarray, vals: np.ndarray | None) -> tuple[int, int]:
    """Order-independent digest (wrapping sum, xor) of the (key, val) pairs."""
    k = keys.astype(np.uint64)
    h = mix64(k)
    if vals is not None:
        with np.errstate(over="ignore"):
            h = mix64(h ^ (vals.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)))
    with np.errstate(over="ignore"):
        s = int(np.sum(h, dtype=np.uint64))
    x = int(np.bitwise_xor.reduce(h)) if len(h) else 0
    return s, x


def check_stable_sorted(in_keys, in_vals, out_keys, out_vals, dtype, index_payload=True):
    """Assert that (out_keys, out_vals) is THE stable sort of (in_keys, in_vals).

    With vals = original index the three properties below determine the stable
    sort uniquely: (1) keys ascend in total order, (2) vals are a permutation of
    0..N-1 and out_keys[i] == in_keys[out_vals[i]], (3) equal keys have
    ascending vals.  Otherwise the multiset digest and sortedness are checked.
    """
    n = len(in_keys)
    assert len(out_keys) == n
    o = total_order_key(out_keys, dtype)
    if n > 1:
        assert np.all(o[:-1] <= o[1:]), "keys not ascending"
    if in_vals is None:
        assert multiset_digest(in_keys, None) == multiset_digest(out_keys, None)
        return
    assert len(out_vals) == n
    if index_payload:
        seen = np.zeros(n, dtype=bool)
        assert out_vals.max(initial=0) < max(n, 1)
        seen[out_vals] = True
        assert seen.all(), "vals are not a permutation"
        assert np.array_equal(in_keys[out_vals], out_keys), "key/val pairs broken"
        if n > 1:
            eq = o[:-1] == o[1:]
            assert np.all(out_vals[:-1][eq] < out_vals[1:][eq]), "not stable"
    else:
        assert multiset_digest(in_keys, in_vals) == multiset_digest(out_keys, out_vals)
