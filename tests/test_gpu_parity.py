"""Parity of the CUDA path (through the C ABI) with the oracle, element by element.

Sorted keys and payloads must match the oracle's stable sort bit for bit; the
bucket vector e, the cut matrix and the splitters must match the oracle's
step-by-step computation (Section IV, steps 2-4) bit for bit.
"""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs
from tests.pins import check_stable_sorted

pytestmark = pytest.mark.gpu

TILE = 17 * 256


def _gpu(*a, **k):
    from tests.gpu_helpers import gpu_sort
    return gpu_sort(*a, **k)


def check_against_oracle(keys, vals, P, dtype, s=None, variant=0, **opts):
    kw = dict(opts)
    if s is not None:
        kw["samples_per_run"] = s
    inv = {0: "rank", 1: "equal", 2: "off"}[variant]
    got = _gpu(keys, vals, P, dtype, investigator=inv, **kw)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    assert np.array_equal(got["keys"], want_k), "keys differ"
    if vals is not None:
        assert np.array_equal(got["vals"], want_v), "payload differs"
    n = len(keys)
    if n:
        ref = O.buckets(keys, P, dtype, samples_per_run=s, variant=variant)
        Peff = ref["P"]
        assert np.array_equal(got["e"], ref["e"]), "bucket bounds differ"
        assert np.array_equal(got["cut"], ref["cut"]), "cut matrix differs"
        assert np.array_equal(O.ord_bits(got["splitters"], dtype), ref["splitters"]), "splitters differ"
        st = got["stats"]
        assert st["n"] == n and st["P"] == Peff
        assert st["max_bucket"] == ref["stats"]["max"] and st["min_bucket"] == ref["stats"]["min"]
    return got


SHAPES = [1, 2, 5, 100, TILE - 1, TILE, TILE + 1, 3 * TILE + 77, 40_009]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("P", [1, 3, 16])
def test_u32_shapes(n, P):
    keys = inputs.uniform_u32(n, seed=n)
    check_against_oracle(keys, inputs.index_payload(n), P, "u32")


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("P", [1, 7, 64])
def test_u64_shapes(n, P):
    keys = inputs.normal_lognormal_u64(n, seed=n + 1)
    check_against_oracle(keys, inputs.index_payload(n), P, "u64")


@pytest.mark.parametrize("n", [1, 77, TILE + 5, 50_001])
@pytest.mark.parametrize("P", [1, 2, 32])
def test_f32_duplicates_and_specials(n, P):
    keys = inputs.zipf_dup_f32(n, seed=n + 2)
    check_against_oracle(keys, inputs.index_payload(n), P, "f32")


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32"])
def test_keys_only(dtype):
    n = 3 * TILE + 11
    gen = {"u32": inputs.uniform_u32, "u64": inputs.uniform_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(n, 5)
    check_against_oracle(keys, None, 8, dtype)


@pytest.mark.parametrize("kind", ["sorted", "reverse", "equal", "few", "extremes"])
def test_structured(kind):
    n = 2 * TILE + 999
    keys = inputs.structured_u32(kind, n)
    check_against_oracle(keys, inputs.index_payload(n), 12, "u32")


@pytest.mark.parametrize("exchange", ["scatter", "fused"])
@pytest.mark.parametrize("dtype,P", [("u64", 7), ("f32", 33), ("u32", 128)])
def test_exchange_modes(exchange, dtype, P):
    n = 3 * TILE + 1234
    gen = {"u32": inputs.exponential_u32, "u64": inputs.normal_lognormal_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(n, P)
    got = check_against_oracle(keys, inputs.index_payload(n), P, dtype, exchange=exchange)
    passes = got["stats"]["passes"]
    other = _gpu(keys, inputs.index_payload(n), P, dtype, exchange="fused" if exchange == "scatter" else "scatter")
    fused, scatter = (passes, other["stats"]["passes"]) if exchange == "fused" else (other["stats"]["passes"], passes)
    assert scatter - 1 <= fused <= scatter          # the fused exchange never costs a pass
    assert np.array_equal(other["keys"], got["keys"]) and np.array_equal(other["vals"], got["vals"])


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_investigator_variants(variant):
    n = 60_000
    keys = inputs.zipf_dup_f32(n, seed=9)
    got = check_against_oracle(keys, inputs.index_payload(n), 64, "f32", s=32, variant=variant)
    if variant == 2:
        assert got["stats"]["max_bucket"] > 3 * n / 64


@pytest.mark.parametrize("P", [2, 5, 17, 100])
def test_many_partitions_small_runs(P):
    n = 1000
    keys = inputs.structured_u32("few", n, seed=P)
    check_against_oracle(keys, inputs.index_payload(n), P, "u32", s=3)


def test_more_partitions_than_keys():
    keys = inputs.uniform_u32(5, 1)
    got = check_against_oracle(keys, inputs.index_payload(5), 64, "u32")
    assert len(got["e"]) == 6


def test_every_key_sampled():
    n = 5000
    keys = inputs.uniform_u32(n, 3)
    check_against_oracle(keys, inputs.index_payload(n), 10, "u32", s=n)


def test_guaranteed_mode_bound():
    # s = ceil(P / eps) = 1024 divides the run length 4096, so every bucket is
    # below (1 + P/s) n/P = (1 + eps) n/P.
    n, P, eps = 1 << 18, 64, 0.0625
    keys = inputs.exponential_u32(n, 4)
    s = max(O.paper_samples_per_run(P, 4), O.guaranteed_samples_per_run(P, eps))
    got = _gpu(keys, inputs.index_payload(n), P, "u32", guaranteed=True, eps=eps)
    ref = O.buckets(keys, P, "u32", samples_per_run=s)
    assert np.array_equal(got["e"], ref["e"])
    assert got["stats"]["samples_per_run"] == s == 1024
    assert got["stats"]["max_bucket"] < (1 + eps) * n / P


@pytest.mark.parametrize("name", ["exponential_u32", "zipf_dup_f32"])
def test_guaranteed_mode_bound_ragged_blocks(name):
    # s = ceil(64 / 0.05) = 1280 does not divide the run length 32768: blocks
    # hold 25 or 26 keys and the bound is -P (s-1)/s <= e_b - b m < P m / s,
    # so every bucket < (1 + eps) m + P.
    n, P, eps = 1 << 21, 64, 0.05
    dtype = "f32" if name == "zipf_dup_f32" else "u32"
    keys = inputs.workload(name, n=n)[1]
    m = n // P
    s = max(O.paper_samples_per_run(P, 4), O.guaranteed_samples_per_run(P, eps))
    assert s == 1280 and m % s != 0
    got = _gpu(keys, inputs.index_payload(n), P, dtype, guaranteed=True)
    ref = O.buckets(keys, P, dtype, samples_per_run=s)
    assert np.array_equal(got["e"], ref["e"])
    d = got["e"].astype(np.int64) - np.arange(P + 1) * m
    assert np.all(d * s >= -P * (s - 1)) and np.all(d * s < P * m)
    assert got["stats"]["max_bucket"] < (1 + eps) * m + P


def test_in_place_equals_copy():
    from tests.gpu_helpers import gpu_sort
    n = 30_011
    keys = inputs.normal_lognormal_u64(n, 8)
    vals = inputs.index_payload(n)
    a = gpu_sort(keys, vals, 9, "u64")
    b = gpu_sort(keys, vals, 9, "u64", in_place=True)
    assert np.array_equal(a["keys"], b["keys"]) and np.array_equal(a["vals"], b["vals"])
    assert np.array_equal(b["input_keys_after"], b["keys"])
    assert np.array_equal(a["input_keys_after"], keys)      # out of place leaves the input alone


def test_arbitrary_payload_travels_with_keys():
    n = 20_000
    keys = inputs.structured_u32("few", n, seed=3)
    vals = np.random.default_rng(1).integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    check_against_oracle(keys, vals, 6, "u32")


def test_small_workload_full():
    # 1M uniform uint32 keys from seed 0, payload = index, P = 16.
    dtype, keys, P = inputs.workload("uniform_u32")
    got = check_against_oracle(keys, inputs.index_payload(len(keys)), P, dtype)
    check_stable_sorted(keys, inputs.index_payload(len(keys)), got["keys"], got["vals"], dtype)


def test_fit_splitters_matches_oracle():
    import torch
    from paper_1611_00463_gb300 import pgs
    for dtype, gen in [("u32", inputs.exponential_u32), ("u64", inputs.normal_lognormal_u64),
                       ("f32", inputs.zipf_dup_f32)]:
        m, P = 70_001, 100
        samples = gen(m, 11)
        dev_s = pgs.as_device_keys(samples, dtype)
        cfg0 = pgs.make_config(dtype=dtype)
        ws = torch.empty(pgs.pgs_fit_workspace_bytes(m, P, cfg0), dtype=torch.uint8, device="cuda")
        cfg = pgs.make_config(dtype=dtype, workspace=ws)
        out = torch.zeros(P - 1, dtype=dev_s.dtype, device="cuda")
        pgs.pgs_fit_splitters(dev_s, P, cfg, out)
        torch.cuda.synchronize()
        want = O.select_splitters(O.ord_bits(samples, dtype), P)
        got = O.ord_bits(pgs.to_numpy_keys(out, dtype), dtype)
        assert np.array_equal(got, want), dtype


def test_workspace_too_small_is_reported():
    import torch
    from paper_1611_00463_gb300 import pgs
    n = 10_000
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    cfg = pgs.make_config(workspace=ws)
    with pytest.raises(pgs.PgsError) as ei:
        pgs.pgs_sort(k, None, 4, cfg)
    assert ei.value.status == pgs.PGS_ERR_WORKSPACE


@pytest.mark.parametrize("dtype,n,P", [("u64", 5 * TILE + 3, 9), ("f32", 40 * TILE + 17, 37), ("u32", 9000, 300),
                                       ("u32", 64 * TILE + 1, 1)])
def test_four_way_and_pairwise_rounds_agree(dtype, n, P):
    gen = {"u32": inputs.exponential_u32, "u64": inputs.normal_lognormal_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(n, n % 97)
    vals = inputs.index_payload(n)
    four = check_against_oracle(keys, vals, P, dtype, merge_ways=4)
    two = check_against_oracle(keys, vals, P, dtype, merge_ways=2)
    assert four["stats"]["passes"] <= two["stats"]["passes"]


@pytest.mark.parametrize("f", [0.004, 0.04, 0.4, 1.0, 1.004, 1.04, 1.4])
def test_sample_size_sweep_points(f):
    """The sample sizes of the paper's sweep (Section V, Fig. 9 and 10):
    f X keys per run, X = 256 KB / P."""
    P = 128
    n = P * 3001 + 17
    keys = inputs.normal_lognormal_u64(n, seed=11)
    s = max(1, int(f * (262144 // (P * 8))))
    check_against_oracle(keys, inputs.index_payload(n), P, "u64", s=s)
    zipf = inputs.zipf_dup_f32(n, seed=12)
    check_against_oracle(zipf, inputs.index_payload(n), P, "f32", s=max(1, int(f * (262144 // (P * 4)))))


@pytest.mark.parametrize("dtype,n,P,s", [("f32", 40_009, 16, None), ("f32", 3 * TILE + 5, 64, 4), ("u64", 30_011, 7, 8),
                                         ("u32", 20_000, 40, 3)])
def test_local_investigator_matches_oracle_pipeline(dtype, n, P, s):
    """The paper-literal per-run division (not stable): keys, payloads, bucket
    vector and cut matrix equal the oracle's six steps with the same rule."""
    gen = {"f32": inputs.zipf_dup_f32, "u64": inputs.zipf_dup_u64, "u32": lambda m, seed: inputs.structured_u32("few", m)}
    keys = gen[dtype](n, 21)
    vals = inputs.index_payload(n)
    kw = {} if s is None else {"samples_per_run": s}
    got = _gpu(keys, vals, P, dtype, investigator="local", **kw)
    ref = O.sample_sort(keys, vals, P, dtype, samples_per_run=s, variant=O.INVESTIGATOR_LOCAL)
    assert np.array_equal(got["keys"], ref["keys"]) and np.array_equal(got["vals"], ref["vals"])
    assert np.array_equal(got["e"], ref["e"]) and np.array_equal(got["cut"], ref["cut"])
    assert np.array_equal(got["keys"], O.stable_sort(keys, vals, dtype)[0])


@pytest.mark.parametrize("dtype,n,P", [("u32", 1 << 20, 16), ("f32", 100_003, 7)])
def test_single_sort_replays_from_a_cuda_graph(dtype, n, P):
    """A single sort captured once into a CUDA graph (after one direct call has
    set the kernels' attributes) and replayed twice from fresh input."""
    import torch
    from paper_1611_00463_gb300 import pgs
    gen = {"u32": inputs.uniform_u32, "f32": inputs.zipf_dup_f32}[dtype]
    keys = gen(n, 77)
    vals = inputs.index_payload(n)
    kin = pgs.as_device_keys(keys, dtype)
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    cfg0 = pgs.make_config(dtype=dtype)
    ws = pgs.workspace(n, P, cfg0)
    bounds = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    cfg = pgs.make_config(dtype=dtype, workspace=ws, bucket_bounds=bounds)
    pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)           # first call on the device: attributes set here
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream=s)
    want_k, want_v = O.stable_sort(keys, vals, dtype)
    for _ in range(2):
        kout.zero_()
        vout.zero_()
        bounds.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(pgs.to_numpy_keys(kout, dtype), want_k)
        assert np.array_equal(vout.cpu().numpy().view(np.uint32), want_v)
        assert np.array_equal(bounds.cpu().numpy(), O.buckets(keys, P, dtype)["e"])
