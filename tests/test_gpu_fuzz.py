"""Randomised parity: seeded random configurations of the sort (key type,
size, partitions, key distribution, investigator, exchange, merge ways, sample
count, guaranteed mode) and of batches, each against the oracle."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu

GENS = {
    "u32": [inputs.uniform_u32, inputs.exponential_u32, lambda n, s: inputs.structured_u32("few", n, s),
            lambda n, s: inputs.structured_u32("sorted", n, s), lambda n, s: inputs.structured_u32("reverse", n, s),
            lambda n, s: inputs.structured_u32("extremes", n, s)],
    "u64": [inputs.uniform_u64, inputs.normal_lognormal_u64, inputs.zipf_dup_u64,
            lambda n, s: inputs.exponential_u64(n, s, scale=1e3)],
    "f32": [inputs.zipf_dup_f32, lambda n, s: inputs.zipf_dup_f32(n, s, distinct=3)],
}


def random_case(seed):
    g = np.random.default_rng(seed)
    dtype = ["u32", "u64", "f32"][int(g.integers(0, 3))]
    n = int(g.choice([0, 1, 2, int(g.integers(3, 100)), int(g.integers(100, 5000)), int(g.integers(5000, 60000))]))
    P = int(g.choice([1, 2, int(g.integers(3, 40)), int(g.integers(40, 300))]))
    gen = GENS[dtype][int(g.integers(0, len(GENS[dtype])))]
    opts = {"investigator": ["rank", "equal", "off"][int(g.integers(0, 3))],
            "exchange": ["auto", "scatter"][int(g.integers(0, 2))],
            "merge_ways": [2, 4][int(g.integers(0, 2))]}
    s = None
    if g.random() < 0.4:
        s = int(g.integers(1, 64))
    elif g.random() < 0.2:
        opts["guaranteed"] = True
    return dtype, n, P, gen, opts, s, int(g.integers(0, 1 << 30))


@pytest.mark.parametrize("seed", range(200))
def test_random_configuration(seed):
    from tests.gpu_helpers import gpu_sort
    dtype, n, P, gen, opts, s, kseed = random_case(seed)
    keys = gen(n, kseed) if n else np.zeros(0, np.uint64 if dtype == "u64" else np.uint32)
    vals = inputs.index_payload(n)
    kw = dict(opts)
    if s is not None:
        kw["samples_per_run"] = s
    got = gpu_sort(keys, vals, P, dtype, **kw)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(got["keys"], want_k) and np.array_equal(got["vals"], want_v)
    if n == 0:
        return
    variant = {"rank": O.INVESTIGATOR_RANK, "equal": O.INVESTIGATOR_EQUAL, "off": O.INVESTIGATOR_OFF}[opts["investigator"]]
    ss = s
    if opts.get("guaranteed"):
        Pe = O.effective_partitions(n, P)
        ss = max(O.paper_samples_per_run(Pe, O.KEY_BYTES[dtype]), O.guaranteed_samples_per_run(Pe, 0.05))
    ref = O.buckets(keys, P, dtype, samples_per_run=ss, variant=variant)
    assert np.array_equal(got["e"], ref["e"])
    assert np.array_equal(got["cut"], ref["cut"])
    assert np.array_equal(O.ord_bits(got["splitters"], dtype), ref["splitters"])


@pytest.mark.parametrize("seed", range(16))
def test_random_batch(seed):
    import torch
    from paper_1611_00463_gb300 import pgs
    g = np.random.default_rng(100 + seed)
    dtype = ["u32", "u64", "f32"][seed % 3]
    num = int(g.integers(1, 60))
    sizes = g.integers(0, int(g.choice([50, 3000, 40000])), size=num)
    offsets = np.zeros(num + 1, np.uint64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    gen = GENS[dtype][int(g.integers(0, len(GENS[dtype])))]
    keys = np.concatenate([gen(int(m), int(g.integers(0, 1 << 30))) if m else
                           np.zeros(0, np.uint64 if dtype == "u64" else np.uint32) for m in sizes])
    vals = np.arange(n, dtype=np.uint32)
    Pv = None if g.random() < 0.5 else g.integers(1, 50, size=num).astype(np.uint32)
    bt = pgs.Batch(offsets, Pv, dtype=dtype, with_vals=True)
    k = pgs.as_device_keys(keys, dtype)
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    bt.sort_copy(k, v, ko, vo)
    torch.cuda.synchronize()
    got_k, got_v = pgs.to_numpy_keys(ko, dtype), vo.cpu().numpy().view(np.uint32)
    for i in range(num):
        a, b = int(offsets[i]), int(offsets[i + 1])
        wk, wv = O.stable_sort(keys[a:b], vals[a:b], dtype)
        assert np.array_equal(got_k[a:b], wk) and np.array_equal(got_v[a:b], wv), f"instance {i}"


def random_case_larger(seed):
    """Sizes up to 3M keys, every merge-width choice (0 = by size) and every
    merge tile shape: the rounds that plan themselves, by one CTA or by the
    partition kernel, and the bucket rounds planned by the offsets kernel."""
    g = np.random.default_rng(seed)
    dtype = ["u32", "u64", "f32"][int(g.integers(0, 3))]
    n = int(g.choice([int(g.integers(1, 5000)), int(g.integers(5000, 300000)), int(g.integers(300000, 3000000))]))
    P = int(g.choice([1, 2, int(g.integers(3, 70)), int(g.integers(70, 400))]))
    gen = GENS[dtype][int(g.integers(0, len(GENS[dtype])))]
    opts = {"investigator": ["rank", "equal", "off"][int(g.integers(0, 3))],
            "exchange": ["auto", "scatter"][int(g.integers(0, 2))],
            "merge_ways": [0, 2, 4][int(g.integers(0, 3))],
            "tile_variant": int(g.integers(0, 4))}
    s = int(g.integers(1, 300)) if g.random() < 0.3 else None
    return dtype, n, P, gen, opts, s, int(g.integers(0, 1 << 30))


@pytest.mark.parametrize("seed", range(10000, 10040))
def test_random_larger_configuration(seed):
    from tests.gpu_helpers import gpu_sort
    dtype, n, P, gen, opts, s, kseed = random_case_larger(seed)
    keys = gen(n, kseed)
    vals = inputs.index_payload(n)
    kw = dict(opts)
    if s is not None:
        kw["samples_per_run"] = s
    got = gpu_sort(keys, vals, P, dtype, **kw)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(got["keys"], want_k) and np.array_equal(got["vals"], want_v)
    variant = {"rank": O.INVESTIGATOR_RANK, "equal": O.INVESTIGATOR_EQUAL, "off": O.INVESTIGATOR_OFF}[opts["investigator"]]
    ref = O.buckets(keys, P, dtype, samples_per_run=s, variant=variant)
    assert np.array_equal(got["e"], ref["e"])
    assert np.array_equal(got["cut"], ref["cut"])
