"""Parity with the oracle on both sides of every boundary between the
small-sort paths and the general ones.

The library picks, by size only: merge CTAs that search their own splits
(rounds of at most 4096 tiles) or a partition kernel; merge CTAs that work
out their pairs from the run or sample offsets (single sorts) or a planner;
bucket rounds planned by the offsets kernel (one instance, pairwise rounds,
ceil(n / 1088) + P^2 <= 4096) or one by one; cut searches by one warp per
(run, splitter) slot (P^2 <= 4096) or one thread; the bucket offsets in one
CTA (P^2 <= 4096) or a sizes kernel and a scan.  Each case sits just inside
or just outside one of those limits; every result must equal the oracle's
bit for bit (keys, payloads, bucket bounds, cut matrix, splitters).
"""
import numpy as np
import pytest

from paper_1611_00463_gb300 import inputs
from tests.test_gpu_parity import check_against_oracle

pytestmark = pytest.mark.gpu

MIN_TILE = 64 * 17          # the smallest merge tile shape
PRE_MAX = 4096              # tiles a pre-planned bucket round may hold


def pre_planned_limit(P):
    """The largest n whose bucket rounds the offsets kernel plans."""
    return (PRE_MAX - P * P) * MIN_TILE


@pytest.mark.parametrize("P", [64, 65])
@pytest.mark.parametrize("dtype", ["u32", "u64"])
def test_cut_search_and_offsets_either_side_of_4096_slots(P, dtype):
    n = 90_001
    gen = {"u32": inputs.exponential_u32, "u64": inputs.normal_lognormal_u64}[dtype]
    keys = gen(n, P)
    check_against_oracle(keys, inputs.index_payload(n), P, dtype)


@pytest.mark.parametrize("P,delta", [(16, 0), (16, 1), (63, 0), (63, 1), (2, 0)])
def test_pre_planned_bucket_rounds_limit(P, delta):
    n = pre_planned_limit(P) + delta
    keys = inputs.uniform_u32(n, P + delta)
    check_against_oracle(keys, inputs.index_payload(n), P, "u32", merge_ways=2)


@pytest.mark.parametrize("exchange", ["scatter", "fused"])
@pytest.mark.parametrize("P", [3, 16, 33])
def test_pre_planned_rounds_with_either_exchange(exchange, P):
    n = 123_457
    keys = inputs.zipf_dup_f32(n, P)
    check_against_oracle(keys, inputs.index_payload(n), P, "f32", exchange=exchange)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_job_mode_at_every_tile_shape(variant):
    n = 250_003
    keys = inputs.normal_lognormal_u64(n, variant)
    check_against_oracle(keys, inputs.index_payload(n), 16, "u64", tile_variant=variant)


@pytest.mark.parametrize("n", [7_000_000, 7_400_000])
def test_self_searching_rounds_up_to_4096_tiles(n):
    # One run level per round (pairwise): the first run round of P = 2 runs
    # has about 5 n / 8704 tiles, inside the 4096-tile limit at 7.0M keys and
    # outside at 7.4M.
    keys = inputs.exponential_u32(n, 3)
    check_against_oracle(keys, inputs.index_payload(n), 2, "u32", merge_ways=2)


@pytest.mark.parametrize("P", [5, 16, 100])
def test_inline_sample_rounds_with_ragged_runs(P):
    # n not a multiple of P: runs of two lengths, every run still gives s samples
    # (or every key when s reaches the run length).
    for n, s in [(P * 1000 + P - 1, None), (P * 37 + 3, 64), (P * 37 + 3, 37), (P * 37 + 3, 38)]:
        keys = inputs.uniform_u32(n, n)
        check_against_oracle(keys, inputs.index_payload(n), P, "u32", s=s)
