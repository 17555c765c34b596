"""pgs_search and pgs_provenance against the oracle's lookups, on outputs of
the CUDA sort (themselves checked against the oracle's stable sort)."""
import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

pytestmark = pytest.mark.gpu


def queries_for(keys, dtype, m, seed):
    g = np.random.default_rng(seed)
    hits = keys[g.integers(0, len(keys), size=m // 2)] if len(keys) else keys[:0]
    if dtype == "u64":
        fresh = g.integers(0, 1 << 64, size=m - len(hits), dtype=np.uint64, endpoint=False)
        ext = np.array([0, (1 << 64) - 1], np.uint64)
    else:
        fresh = g.integers(0, 1 << 32, size=m - len(hits), dtype=np.uint64).astype(np.uint32)
        ext = np.array([0, 0x80000000, 0x7FC00000, 0xFFC00000, 0x7F800000, 0xFF800000, 0xFFFFFFFF], np.uint32)
    return np.concatenate([hits.astype(ext.dtype), fresh.astype(ext.dtype), ext])


@pytest.mark.parametrize("dtype,gen,n,P", [("u32", inputs.exponential_u32, 300_001, 16),
                                           ("u64", inputs.normal_lognormal_u64, 200_003, 128),
                                           ("f32", inputs.zipf_dup_f32, 250_000, 64),
                                           ("u32", inputs.uniform_u32, 400_009, 3000),     # bounds beyond smem
                                           ("u64", inputs.zipf_dup_u64, 9_000, 8)])        # one-level search
def test_search_and_buckets_match_oracle(dtype, gen, n, P):
    import torch
    from paper_1611_00463_gb300 import pgs
    from tests.gpu_helpers import gpu_sort
    keys = gen(n, 3)
    vals = inputs.index_payload(n)
    got = gpu_sort(keys, vals, P, dtype)
    assert np.array_equal(got["keys"], O.stable_sort(keys, vals, dtype)[0])
    q = queries_for(got["keys"], dtype, 70_001, 4)
    dk = pgs.as_device_keys(got["keys"], dtype)
    dq = pgs.as_device_keys(q, dtype)
    e = torch.from_numpy(got["e"]).cuda()
    nbytes = pgs.pgs_search_workspace_bytes(n, dtype)
    assert nbytes == (0 if n < 64 * 1024 else -(-n // 64) * (8 if dtype == "u64" else 4))
    for ws in (None, torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")):   # plain, indexed
        for side in ("left", "right"):
            pos = torch.empty(len(q), dtype=torch.int64, device="cuda")
            bkt = torch.empty(len(q), dtype=torch.int32, device="cuda")
            pgs.pgs_search(dk, dq, pos, side=side, dtype=dtype, bucket_bounds=e, bucket_out=bkt, workspace=ws)
            torch.cuda.synchronize()
            want = O.search(got["keys"], q, dtype, side)
            assert np.array_equal(pos.cpu().numpy(), want)
            assert np.array_equal(bkt.cpu().numpy(), O.bucket_of(want, got["e"]))


def test_provenance_matches_oracle():
    import torch
    from paper_1611_00463_gb300 import pgs
    from tests.gpu_helpers import gpu_sort
    for n, P in [(100_003, 37), (5, 9), (4096, 1)]:
        keys = inputs.uniform_u32(n, n)
        got = gpu_sort(keys, inputs.index_payload(n), P, "u32")
        v = got["vals"]
        v_ext = np.concatenate([v, np.array([n, n + 5], np.uint32)])      # two payloads that are not positions
        dv = torch.from_numpy(v_ext.view(np.int32)).cuda()
        run = torch.empty(len(v_ext), dtype=torch.int32, device="cuda")
        idx = torch.empty(len(v_ext), dtype=torch.int64, device="cuda")
        pgs.pgs_provenance(dv, n, P, run, idx)
        torch.cuda.synchronize()
        wr, wi = O.provenance(v_ext, n, P)
        assert np.array_equal(run.cpu().numpy(), wr) and np.array_equal(idx.cpu().numpy(), wi)


def test_search_edges():
    import torch
    from paper_1611_00463_gb300 import pgs
    q = torch.tensor([0, 5, -1], dtype=torch.int32, device="cuda")
    pos = torch.full((3,), 7, dtype=torch.int64, device="cuda")
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    pgs.pgs_search(empty, q, pos, side="left")                       # no keys: every query at 0
    torch.cuda.synchronize()
    assert pos.cpu().tolist() == [0, 0, 0]
    pgs.pgs_search(empty, q[:0], pos[:0])                            # no queries: nothing to do
    with pytest.raises(pgs.PgsError):
        pgs.load()
        pgs._check(pgs.load().pgs_search(None, 0, q.data_ptr(), 3, 2, None, 0, pos.data_ptr(), None, None, None),
                   "pgs_search")


@pytest.mark.parametrize("dtype,side", [("u64", "left"), ("f32", "right")])
def test_many_queries_lockstep_path(dtype, side):
    """1.5 million queries on 2 million keys (a ragged last block)."""
    import torch
    from paper_1611_00463_gb300 import pgs
    n = 2_000_003
    gen = {"u64": inputs.uniform_u64, "f32": inputs.zipf_dup_f32}[dtype]
    keys = np.sort(O.ord_bits(gen(n, 41), dtype))
    if dtype == "f32":                                  # back from order form to float bits
        keys = np.where(keys >> np.uint32(31) == 1, keys & np.uint32(0x7FFFFFFF), ~keys).astype(np.uint32)
    q = queries_for(keys, dtype, 1_500_007, 42)
    ws = torch.empty(pgs.pgs_search_workspace_bytes(n, dtype), dtype=torch.uint8, device="cuda")
    want = O.search(keys, q, dtype, side)
    for w in (None, ws):
        pos = torch.empty(len(q), dtype=torch.int64, device="cuda")
        pgs.pgs_search(pgs.as_device_keys(keys, dtype), pgs.as_device_keys(q, dtype), pos, side=side, dtype=dtype,
                       workspace=w)
        torch.cuda.synchronize()
        assert np.array_equal(pos.cpu().numpy(), want)
