"""Plant plausible mistakes in a copy of the oracle and check that its pins catch each.

The copy is built from the oracle's source text with one replacement applied;
the real oracle module is never modified.
"""
import os
import types

import numpy as np
import pytest

from paper_1611_00463_gb300 import inputs
from tests.pins import check_stable_sorted, golden_lines, insertion_sort_order

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "pgs_oracle.py")

MUTATIONS = {
    "drop_prefix_over_runs": ("- pre[:, 1:P]", ""),
    "lower_bound_as_upper": ('lb[r, 1:P] = np.searchsorted(run_ord[r], t, side="left")',
                             'lb[r, 1:P] = np.searchsorted(run_ord[r], t, side="right")'),
    "rank_target_off_by_one": ("e[b] = min(max((b * n) // P, L[b]), L[b] + G[b])",
                               "e[b] = min(max((b * n) // P + 1, L[b]), L[b] + G[b])"),
    "clamp_without_upper": ("e[b] = min(max((b * n) // P, L[b]), L[b] + G[b])",
                            "e[b] = max((b * n) // P, L[b])"),
    "sample_position_off_by_one": ("return (i * n_r) // s_r - 1", "return (i * n_r) // s_r - 1 - (i == s_r)"),
    "splitter_index_off_by_one": ("idx = [(b * S) // P - 1 for b in range(1, P)]",
                                  "idx = [(b * S) // P for b in range(1, P)]"),
    "float_sign_not_flipped": ("np.where(neg, ~b, b | np.uint32(0x80000000))",
                               "np.where(neg, b, b | np.uint32(0x80000000))"),
    "exchange_inclusive_prefix": ("before = np.cumsum(size, axis=0) - size",
                                  "before = np.cumsum(size, axis=0)"),
    "merge_ties_to_second_list": ("k = np.concatenate([ka, kb])\n    v = None if va is None else np.concatenate([va, vb])",
                                  "k = np.concatenate([kb, ka])\n    v = None if va is None else np.concatenate([vb, va])"),
    "schedule_wrong_stride": ("range(0, k, 2 * step)", "range(0, k, step + 1)"),
    "ceil_run_split": ("(r * n) // P for r in range(P + 1)", "(r * n + P - 1) // P for r in range(P + 1)"),
    "budget_counts_payload": ("SAMPLE_BUFFER_BYTES // (P * key_bytes)",
                              "SAMPLE_BUFFER_BYTES // (P * (key_bytes + 4))"),
    "local_divides_global_count": ("cut[:, b + i] = lb[:, b] + (cnt[:, b] * (i + 1)) // k",
                                   "cut[:, b + i] = lb[:, b] + (G[b] * (i + 1)) // k"),
    "local_one_part_too_many": ("cut[:, b + i] = lb[:, b] + (cnt[:, b] * (i + 1)) // k",
                                "cut[:, b + i] = lb[:, b] + (cnt[:, b] * (i + 1)) // (k + 1)"),
}


def load_oracle(mutation=None):
    src = open(SRC).read()
    if mutation is not None:
        old, new = MUTATIONS[mutation]
        assert src.count(old) == 1, mutation
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_copy")
    exec(compile(src, SRC, "exec"), mod.__dict__)
    return mod


def run_pins(O):
    """A compact pass over the pins of tests/test_oracle_*.py; raises on failure."""
    # Golden: IEEE totalOrder and the Fig. 2 schedule.
    pats = np.array([int(ln.split()[0], 16) for ln in golden_lines("f32_total_order.txt")], np.uint32)
    o = O.ord_bits(pats, "f32").astype(np.uint64)
    assert np.all(o[:-1] < o[1:])
    want = [[tuple(int(x) for x in p.split("<-")) for p in ln.split()]
            for ln in golden_lines("fig2_schedule_8.txt")]
    assert O.balanced_merge_schedule(8) == want
    # Closed forms.
    assert list(O.run_bounds(10, 3)) == [0, 3, 6, 10]
    assert list(O.regular_sample_positions(16, 4)) == [3, 7, 11, 15]
    assert O.paper_samples_per_run(128, 8) == 256
    # Brute-force bucket semantics and the balance bound.
    g = np.random.default_rng(5)
    for _ in range(60):
        P = int(g.integers(1, 9))
        s = int(g.integers(1, 5))
        n = s * int(g.integers(1, 5))
        keys = g.integers(0, int(g.integers(1, 5)), size=P * n).astype(np.uint32)
        res = O.buckets(keys, P, "u32", samples_per_run=s)
        e, cut = res["e"], res["cut"]
        d = e - np.arange(P + 1) * n
        assert np.all(d >= 0) and np.all(d * s < P * n)
        order = insertion_sort_order(list(keys))
        rank = np.empty(len(keys), np.int64)
        rank[order] = np.arange(len(keys))
        for r in range(P):
            rr = np.sort(rank[r * n:(r + 1) * n])
            for b in range(P):
                seg = rr[cut[r, b]:cut[r, b + 1]]
                assert np.array_equal(seg, rr[(rr >= e[b]) & (rr < e[b + 1])])
    # Unequal runs (n not a multiple of P, s not dividing n): bucket semantics
    # and sum over runs of the cuts == e_b.
    for _ in range(60):
        n = int(g.integers(1, 50))
        P = int(g.integers(1, 8))
        keys = g.integers(0, int(g.integers(1, 5)), size=n).astype(np.uint32)
        res = O.buckets(keys, P, "u32", samples_per_run=int(g.integers(1, 5)))
        assert np.array_equal(res["cut"].sum(axis=0), res["e"])
    # Runs of 3 with 2 samples each: blocks of sizes 1 and 2, and the target
    # floor(3 * 15 / 5) = 9 lies above every copy of splitter t_3 (L = 6, G = 2),
    # so only the upper clamp keeps e_3 consistent with the cuts.
    keys = np.array([4, 1, 3, 0, 2, 0, 2, 0, 4, 4, 0, 4, 3, 1, 3], np.uint32)
    res = O.buckets(keys, 5, "u32", samples_per_run=2)
    assert np.array_equal(res["cut"].sum(axis=0), res["e"]) and res["e"][3] == 8
    # Closed forms: all-equal keys cut exactly at floor(bN/P); with every element
    # sampled and distinct keys the splitters are the exact P-quantile keys.
    keys = np.full(50, 7, np.uint32)
    res = O.buckets(keys, 6, "u32", samples_per_run=3)
    assert list(res["e"]) == [(b * 50) // 6 for b in range(7)]
    keys = np.random.default_rng(4).permutation(48).astype(np.uint32) * 3
    res = O.buckets(keys, 6, "u32", samples_per_run=8)
    assert list(res["splitters"]) == list(np.sort(keys)[[8 * b - 1 for b in range(1, 6)]])
    # Fig. 5(c) with the per-run rule: every run splits its own copies of the
    # duplicated value into four equal parts.
    keys = np.full(40, 5, np.uint32)
    keys[0], keys[39] = 1, 9
    res = O.buckets(keys, 5, "u32", samples_per_run=8, variant=O.INVESTIGATOR_LOCAL)
    cnt_a, lb_a = [7, 8, 8, 8, 7], [1, 0, 0, 0, 0]
    for r in range(5):
        assert list(res["cut"][r]) == [0] + [lb_a[r] + (cnt_a[r] * (i + 1)) // 4 for i in range(4)] + [8]
    # The full pipeline against the stable-sort properties.
    for name, n, P in [("zipf_dup_f32", 3001, 16), ("normal_lognormal_u64", 2000, 8)]:
        dtype, keys, _ = inputs.workload(name, n=n)
        vals = inputs.index_payload(n)
        res = O.sample_sort(keys, vals, P, dtype, threads=4)
        check_stable_sorted(keys, vals, res["keys"], res["vals"], dtype)
        exch = res["dst"]
        assert exch.min() >= 0 and exch.max() <= n


def test_unmutated_oracle_passes_pins():
    run_pins(load_oracle())


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(mutation):
    O = load_oracle(mutation)
    with pytest.raises(Exception):
        run_pins(O)
