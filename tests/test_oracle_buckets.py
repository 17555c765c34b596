"""Pins of the oracle's Part 2: the method's steps (Section IV) and the bucket vector."""
import itertools

import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs
from tests.pins import check_stable_sorted, golden_lines, insertion_sort_order

VARIANTS = [O.INVESTIGATOR_RANK, O.INVESTIGATOR_EQUAL, O.INVESTIGATOR_OFF]


def test_fig2_schedule_golden():
    want = [[tuple(int(x) for x in pair.split("<-")) for pair in ln.split()]
            for ln in golden_lines("fig2_schedule_8.txt")]
    assert O.balanced_merge_schedule(8) == want


@pytest.mark.parametrize("k", range(1, 40))
def test_schedule_merges_every_list_once(k):
    # Every list but list 0 is a source exactly once, and only after it has
    # absorbed everything it will ever absorb; list 0 ends holding all.
    holds = {i: {i} for i in range(k)}
    done = set()
    for rnd in O.balanced_merge_schedule(k):
        assert len({d for d, _ in rnd} | {s for _, s in rnd}) == 2 * len(rnd)
        for d, s in rnd:
            assert s not in done and d not in done
            holds[d] |= holds.pop(s)
            done.add(s)
    assert holds == {0: set(range(k))}


def test_run_bounds_closed_form():
    assert list(O.run_bounds(10, 3)) == [0, 3, 6, 10]
    assert list(O.run_bounds(16, 4)) == [0, 4, 8, 12, 16]
    assert list(O.run_bounds(5, 5)) == [0, 1, 2, 3, 4, 5]


def test_sample_positions_closed_form():
    assert list(O.regular_sample_positions(16, 4)) == [3, 7, 11, 15]
    assert list(O.regular_sample_positions(10, 3)) == [2, 5, 9]
    assert list(O.regular_sample_positions(3, 8)) == [0, 1, 2]
    assert list(O.regular_sample_positions(0, 8)) == []


def test_paper_sample_budget():
    # Section IV-B: 256/p KB per processor.
    assert O.paper_samples_per_run(16, 4) == 4096
    assert O.paper_samples_per_run(128, 8) == 256
    assert O.paper_samples_per_run(256, 4) == 256
    assert O.paper_samples_per_run(1024, 4) == 64
    assert O.paper_samples_per_run(10, 8) == 3276


def test_local_sort_equals_stable_sort():
    for n in [0, 1, 5, 31, 32, 33, 1000]:
        keys = inputs.structured_u32("few", n) if n else np.zeros(0, np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        k, v = O.local_sort(keys, vals, "u32", threads=32)
        check_stable_sorted(keys, vals, k, v, "u32")


def _stable_ranks(ordkeys):
    order = insertion_sort_order(list(ordkeys))
    rank = np.empty(len(ordkeys), dtype=np.int64)
    rank[order] = np.arange(len(ordkeys))
    return rank


@pytest.mark.parametrize("variant", VARIANTS)
def test_cut_semantics_brute_force(variant):
    # For small inputs, bucket b of the cut matrix must hold exactly the
    # elements of global stable rank [e_b, e_{b+1}) from every run.
    g = np.random.default_rng(5)
    for trial in range(150):
        n = int(g.integers(1, 60))
        P = int(g.integers(1, 9))
        keys = g.integers(0, int(g.integers(1, 6)), size=n).astype(np.uint32)
        s = int(g.integers(1, 6))
        res = O.buckets(keys, P, "u32", samples_per_run=s, variant=variant)
        Pe, e, cut, bounds = res["P"], res["e"], res["cut"], res["bounds"]
        rank = _stable_ranks(keys)
        assert e[0] == 0 and e[Pe] == n and np.all(np.diff(e) >= 0)
        for r in range(Pe):
            lo, hi = bounds[r], bounds[r + 1]
            run_rank = np.sort(rank[lo:hi])      # stable order inside a run = rank order
            assert cut[r, 0] == 0 and cut[r, Pe] == hi - lo
            for b in range(Pe):
                seg = run_rank[cut[r, b]:cut[r, b + 1]]
                inside = (run_rank >= e[b]) & (run_rank < e[b + 1])
                assert np.array_equal(seg, run_rank[inside])


def _equal_runs_bound_check(keys, P, s, dtype="u32"):
    n = len(keys) // P
    assert n * P == len(keys) and n % s == 0
    res = O.buckets(keys, P, dtype, samples_per_run=s)
    e = res["e"]
    b = np.arange(P + 1)
    d = e - b * n
    # Balance bound: 0 <= e_b - b n < P n / s for any input.
    assert np.all(d >= 0)
    assert np.all(d * s < P * n)
    sizes = np.diff(e)
    assert np.all(sizes * s < n * (s + P)) and np.all(sizes * s > n * (s - P))
    return res


@pytest.mark.parametrize("kind", ["random", "few", "equal", "sorted", "reverse", "extremes"])
@pytest.mark.parametrize("P,s,n", [(4, 4, 64), (8, 16, 128), (16, 8, 64), (7, 5, 35), (32, 64, 256)])
def test_balance_bound_any_input(kind, P, s, n):
    N = P * n
    if kind == "random":
        keys = inputs.uniform_u32(N, 3)
    else:
        keys = inputs.structured_u32(kind, N, seed=P * 1000 + s)
    _equal_runs_bound_check(keys, P, s)


def test_balance_bound_heavy_duplicates_random():
    g = np.random.default_rng(9)
    for _ in range(200):
        P = int(g.integers(1, 12))
        s = int(g.integers(1, 9))
        n = s * int(g.integers(1, 9))
        distinct = int(g.integers(1, 5))
        keys = g.integers(0, distinct, size=P * n).astype(np.uint32)
        _equal_runs_bound_check(keys, P, s)


def _ragged_bound_check(keys, P, s, dtype="u32"):
    """Equal runs of n keys, s samples per run with s not dividing n (blocks of
    floor or ceil n/s keys).  The run's first floor(k n / s) keys are at or
    before its k-th sample and fewer than floor((k+1) n / s) are before the
    next, so t_b's stable rank R_b satisfies b n - P (s-1)/s <= R_b + 1 <=
    b n + P n / s, and the clamp keeps e_b between b n and R_b:
    -P (s-1)/s <= e_b - b n < P n / s, every bucket < (1 + P/s) n + P."""
    n = len(keys) // P
    assert n * P == len(keys) and s <= n
    res = O.buckets(keys, P, dtype, samples_per_run=s)
    d = res["e"] - np.arange(P + 1) * n
    assert np.all(d * s >= -P * (s - 1))
    assert np.all(d * s < P * n)
    sizes = np.diff(res["e"])
    assert np.all(sizes * s < n * s + P * n + P * (s - 1))
    assert np.all(sizes * s > n * s - P * n - P * (s - 1))
    return res


@pytest.mark.parametrize("kind", ["random", "few", "equal", "sorted", "reverse", "extremes"])
@pytest.mark.parametrize("P,s,n", [(4, 3, 64), (8, 5, 128), (16, 7, 64), (7, 6, 35), (32, 60, 256), (5, 64, 100)])
def test_balance_bound_ragged_blocks(kind, P, s, n):
    assert n % s != 0
    N = P * n
    keys = inputs.uniform_u32(N, 5) if kind == "random" else inputs.structured_u32(kind, N, seed=P * 100 + s)
    _ragged_bound_check(keys, P, s)


def test_balance_bound_ragged_blocks_adversarial():
    # Heavy duplicates, and keys that put each run's samples at the short end
    # of the blocks: the lower side of the bound is reached only when s does
    # not divide n, so a check written for s | n (e_b >= b n) would fail here.
    g = np.random.default_rng(17)
    below = 0
    for _ in range(400):
        P = int(g.integers(2, 12))
        n = int(g.integers(3, 40))
        s = int(g.integers(2, n + 1))
        if n % s == 0:
            continue
        distinct = int(g.integers(1, 6))
        keys = g.integers(0, distinct, size=P * n).astype(np.uint32)
        if g.random() < 0.5:
            keys = np.arange(P * n, dtype=np.uint32) % (n * P // max(1, distinct))
        res = _ragged_bound_check(keys, P, s)
        below += int(np.any(res["e"] - np.arange(P + 1) * n < 0))
    assert below > 0, "no case fell below b n: the test does not reach the ragged side of the bound"


def test_all_equal_keys_exact_sizes():
    for N, P in [(100, 7), (1000, 16), (12, 12), (5, 3)]:
        keys = np.full(N, 42, dtype=np.uint32)
        res = O.buckets(keys, P, "u32", samples_per_run=3)
        want = [((b + 1) * N) // P - (b * N) // P for b in range(P)]
        assert list(res["stats"]["sizes"]) == want


def test_single_partition():
    keys = inputs.uniform_u32(1000, 1)
    res = O.buckets(keys, 1, "u32")
    assert list(res["e"]) == [0, 1000]


def test_full_sampling_distinct_keys_is_exact():
    # Every element sampled (s = n) and distinct keys: bucket b = ranks [bn, (b+1)n).
    P, n = 8, 50
    keys = np.random.default_rng(2).permutation(P * n).astype(np.uint32)
    res = O.buckets(keys, P, "u32", samples_per_run=n)
    assert list(res["e"]) == [b * n for b in range(P + 1)]


def test_full_sampling_splitters_are_quantiles():
    # With every element sampled (s = n) the Master sees the whole data, so the
    # splitter t_b is the largest key of the first b n keys in sorted order.
    g = np.random.default_rng(8)
    for P, n in [(8, 50), (5, 7), (16, 3)]:
        keys = g.permutation(P * n).astype(np.uint32) * 7
        res = O.buckets(keys, P, "u32", samples_per_run=n)
        assert list(res["splitters"]) == list(np.sort(keys)[[b * n - 1 for b in range(1, P)]])


def test_cuts_sum_to_bucket_bounds_unequal_runs():
    g = np.random.default_rng(12)
    for variant in VARIANTS:
        for _ in range(100):
            n = int(g.integers(1, 80))
            P = int(g.integers(1, 10))
            keys = g.integers(0, int(g.integers(1, 6)), size=n).astype(np.uint32)
            res = O.buckets(keys, P, "u32", samples_per_run=int(g.integers(1, 6)), variant=variant)
            assert np.array_equal(res["cut"].sum(axis=0), res["e"])
            assert np.all(np.diff(res["cut"], axis=1) >= 0)


def test_upper_clamp_case():
    # Unequal blocks (runs of 3, 2 samples): the ideal rank 9 of splitter t_3
    # lies above all its copies (L = 6, G = 2), so e_3 = L + G = 8.
    keys = np.array([4, 1, 3, 0, 2, 0, 2, 0, 4, 4, 0, 4, 3, 1, 3], np.uint32)
    res = O.buckets(keys, 5, "u32", samples_per_run=2)
    assert res["e"][3] == 8
    assert np.array_equal(res["cut"].sum(axis=0), res["e"])


def test_fig5c_duplicated_splitters_divide_equally():
    # Fig. 5(c): four duplicated splitters with the same value a share the range
    # of a.  Five processors, mostly a, one smaller and one larger key.
    a = 5
    keys = np.full(40, a, dtype=np.uint32)
    keys[0] = 1
    keys[39] = 9
    rank_target = O.buckets(keys, 5, "u32", samples_per_run=8, variant=O.INVESTIGATOR_RANK)
    assert list(rank_target["splitters"]) == [a, a, a, a]
    assert list(rank_target["stats"]["sizes"]) == [8, 8, 8, 8, 8]
    equal = O.buckets(keys, 5, "u32", samples_per_run=8, variant=O.INVESTIGATOR_EQUAL)
    # L = 1 key below a, G = 38 copies of a split into 4 equal parts.
    assert list(equal["e"]) == [0, 1 + 9, 1 + 19, 1 + 28, 1 + 38, 40]
    # Fig. 5(b): plain binary search sends the whole range of a to one processor.
    naive = O.buckets(keys, 5, "u32", samples_per_run=8, variant=O.INVESTIGATOR_OFF)
    assert list(naive["stats"]["sizes"]) == [39, 0, 0, 0, 1]


def test_naive_fails_and_investigator_meets_bound_on_duplicates():
    _, keys, _ = inputs.workload("zipf_dup_f32", n=256 * 512)
    P, s = 256, 512
    naive = O.buckets(keys, P, "f32", samples_per_run=s, variant=O.INVESTIGATOR_OFF)
    rank = O.buckets(keys, P, "f32", samples_per_run=s)
    assert naive["stats"]["max_over_mean"] > 10.0
    assert rank["stats"]["max_over_mean"] < 1.0 + P / s


def test_table2_shares_consistent_with_budget_reading():
    # Table II: 10 processors.  With 8-byte keys the budget 256 KB / p gives
    # s = 3276 samples and the bound 1 + P/s = 1.00305; every printed share lies
    # inside it.  With 4-byte keys the bound (1.0015) would exclude 10.022 %.
    rows = [ln.split() for ln in golden_lines("table2_shares.txt")]
    shares = np.array([[float(x) for x in r[1:]] for r in rows])
    assert np.allclose(shares.sum(axis=1), 100.0, atol=0.01)
    P = 10
    s8 = O.paper_samples_per_run(P, 8)
    s4 = O.paper_samples_per_run(P, 4)
    assert np.all(shares / 10.0 < 1 + P / s8)
    assert shares.max() / 10.0 > 1 + P / s4


def test_table2_setting_reproduces_bound():
    # The same setting on synthetic stand-ins of the four distributions, with
    # equal runs and s | n, stays inside 1 + P/s.
    P = 10
    s = O.paper_samples_per_run(P, 8)
    N = P * s * 4
    for gen in [inputs.uniform_u64, inputs.normal_lognormal_u64, inputs.exponential_u64]:
        keys = gen(N, 21)
        res = _equal_runs_bound_check(keys, P, s, dtype="u64")
        assert res["stats"]["max_over_mean"] < 1 + P / s


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name,n,P", [("uniform_u32", 4099, 16), ("normal_lognormal_u64", 3000, 8),
                                      ("zipf_dup_f32", 5003, 32), ("exponential_u32", 2048, 64)])
def test_pipeline_equals_stable_sort(variant, name, n, P):
    dtype, keys, _ = inputs.workload(name, n=n)
    vals = inputs.index_payload(n)
    res = O.sample_sort(keys, vals, P, dtype, variant=variant, threads=4)
    k, v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(res["keys"], k) and np.array_equal(res["vals"], v)
    check_stable_sorted(keys, vals, res["keys"], res["vals"], dtype)


def test_pipeline_edge_shapes():
    for n, P in [(0, 4), (1, 1), (1, 8), (3, 8), (8, 8), (9, 8), (100, 1), (17, 16)]:
        keys = inputs.structured_u32("few", n) if n else np.zeros(0, np.uint32)
        vals = inputs.index_payload(n)
        res = O.sample_sort(keys, vals, P, "u32", samples_per_run=2, threads=3)
        check_stable_sorted(keys, vals, res["keys"], res["vals"], "u32")
        assert res["P"] == max(1, min(P, n))


def test_exchange_offsets_tile_the_output():
    _, keys, _ = inputs.workload("exponential_u32", n=3001)
    res = O.sample_sort(keys, None, 12, "u32", threads=2)
    cut, dst, e = res["cut"], res["dst"], res["e"]
    size = cut[:, 1:] - cut[:, :-1]
    # Segments of bucket b lie back to back in run order and fill [e_b, e_{b+1}).
    covered = np.zeros(e[-1], dtype=np.int64)
    for r in range(cut.shape[0]):
        for b in range(cut.shape[1] - 1):
            covered[dst[r, b]:dst[r, b] + size[r, b]] += 1
            assert e[b] <= dst[r, b] and dst[r, b] + size[r, b] <= e[b + 1]
    assert np.all(covered == 1)


def test_fig5c_local_rule_divides_every_run():
    # The text's literal rule: each processor divides its own range of the
    # duplicated value equally among the four duplicated splitters.
    a = 5
    keys = np.full(40, a, dtype=np.uint32)
    keys[0] = 1
    keys[39] = 9
    loc = O.buckets(keys, 5, "u32", samples_per_run=8, variant=O.INVESTIGATOR_LOCAL)
    assert list(loc["splitters"]) == [a, a, a, a]
    # Runs of 8 keys: run 0 holds 1 + seven a, runs 1-3 eight a, run 4 seven a + 9.
    cnt_a = [7, 8, 8, 8, 7]
    lb_a = [1, 0, 0, 0, 0]
    for r in range(5):
        want = [0] + [lb_a[r] + (cnt_a[r] * (i + 1)) // 4 for i in range(4)] + [8]
        assert list(loc["cut"][r]) == want
    assert list(loc["e"]) == list(loc["cut"].sum(axis=0))
    assert list(loc["e"]) == [0, 1 + 1 + 2 + 2 + 2 + 1, 1 + 3 + 4 + 4 + 4 + 3, 1 + 5 + 6 + 6 + 6 + 5,
                              1 + 38, 40]


@pytest.mark.parametrize("seed", range(6))
def test_local_rule_sorts_keys_and_stays_within_rounding_of_equal(seed):
    rng = np.random.default_rng(seed)
    n, P = int(rng.integers(50, 400)), int(rng.integers(2, 12))
    keys = rng.choice(np.array([3, 7, 7, 7, 7, 11, 20], np.uint32), size=n)
    vals = np.arange(n, dtype=np.uint32)
    s = int(rng.integers(1, 9))
    loc = O.sample_sort(keys, vals, P, "u32", samples_per_run=s, variant=O.INVESTIGATOR_LOCAL)
    want_k, _ = O.stable_sort(keys, vals, "u32")
    assert np.array_equal(loc["keys"], want_k)
    assert np.array_equal(np.sort(loc["vals"]), vals)
    assert np.array_equal(keys[loc["vals"]], loc["keys"])
    eq = O.buckets(keys, P, "u32", samples_per_run=s, variant=O.INVESTIGATOR_EQUAL)
    # Per-run floors against the floor of the sum: e_LOCAL <= e_EQUAL < e_LOCAL + R.
    R = loc["P"]
    assert np.all(loc["e"] <= eq["e"]) and np.all(eq["e"] - loc["e"] < R)
    # Inside each bucket, keys from run r precede equal keys from run r' > r.
    for b in range(R):
        seg = loc["vals"][loc["e"][b]:loc["e"][b + 1]]
        run_of = np.searchsorted(loc["bounds"], seg, side="right") - 1
        kk = keys[seg]
        for i in range(len(seg) - 1):
            if kk[i] == kk[i + 1]:
                assert (run_of[i], seg[i]) < (run_of[i + 1], seg[i + 1])


def test_local_rule_is_not_stable():
    # Three runs of three 7s under two duplicated splitters: each run sends
    # floor(3/2) = 1 of its 7s to bucket 0 and the other 2 to bucket 1, so run
    # 1's first 7 comes before run 0's second.
    keys = np.full(9, 7, np.uint32)
    vals = np.arange(9, dtype=np.uint32)
    loc = O.sample_sort(keys, vals, 3, "u32", samples_per_run=3, variant=O.INVESTIGATOR_LOCAL)
    assert list(loc["splitters"]) == [7, 7]
    assert [list(r) for r in loc["cut"]] == [[0, 1, 3, 3]] * 3
    assert list(loc["e"]) == [0, 3, 9, 9]
    assert list(loc["vals"]) == [0, 3, 6, 1, 2, 4, 5, 7, 8]
    assert list(O.stable_sort(keys, vals, "u32")[1]) == list(range(9))
