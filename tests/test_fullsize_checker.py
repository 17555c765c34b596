"""The property checker of the full-size GPU tests, run on CPU tensors: it
accepts the oracle's stable sort and rejects each kind of wrong output."""
import numpy as np
import pytest
import torch

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs
from tests.test_gpu_fullsize import check_stable_sort_device


def as_t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if dtype == "u64" else np.int32).copy())


def sorted_pair(keys, dtype):
    vals = np.arange(len(keys), dtype=np.uint32)
    k, v = O.stable_sort(keys, vals, dtype)
    return as_t(keys, dtype), as_t(k, dtype), torch.from_numpy(v.view(np.int32).copy())


@pytest.mark.parametrize("dtype,gen", [("u64", inputs.normal_lognormal_u64), ("u32", inputs.exponential_u32),
                                       ("f32", inputs.zipf_dup_f32)])
def test_accepts_the_stable_sort_in_chunks(dtype, gen):
    keys = gen(50_000, 3)
    kin, kout, vout = sorted_pair(keys, dtype)
    check_stable_sort_device(kin, kout, vout, dtype, chunk=4096)


def test_rejects_each_kind_of_mistake():
    dtype = "f32"
    keys = inputs.zipf_dup_f32(20_000, 4)
    kin, kout, vout = sorted_pair(keys, dtype)
    o = O.ord_bits(kout.numpy().view(np.uint32), dtype)
    i = int(np.nonzero(o[:-1] == o[1:])[0][10])             # two equal neighbours
    bad = vout.clone()
    bad[i], bad[i + 1] = vout[i + 1], vout[i]               # stability broken
    with pytest.raises(AssertionError):
        check_stable_sort_device(kin, kout, bad, dtype, chunk=4096)
    bad = vout.clone()
    bad[5] = vout[6]                                        # not a permutation (and a wrong key)
    with pytest.raises(AssertionError):
        check_stable_sort_device(kin, kout, bad, dtype, chunk=4096)
    badk = kout.clone()
    badk[100] = badk[100] ^ 1                               # a key that is not its payload's input key
    with pytest.raises(AssertionError):
        check_stable_sort_device(kin, badk, vout, dtype, chunk=4096)
    j = int(np.nonzero(o[:-1] < o[1:])[0][7])               # two different neighbours swapped with payloads
    bk, bv = kout.clone(), vout.clone()
    bk[j], bk[j + 1] = kout[j + 1], kout[j]
    bv[j], bv[j + 1] = vout[j + 1], vout[j]
    with pytest.raises(AssertionError):
        check_stable_sort_device(kin, bk, bv, dtype, chunk=4096)


def test_batch_instances_are_checked_separately():
    sizes = [300, 0, 1, 4000, 77]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    keys = inputs.uniform_u64(int(offsets[-1]), 9)
    parts_k, parts_v = [], []
    for a, b in zip(offsets[:-1], offsets[1:]):
        k, v = O.stable_sort(keys[a:b], np.arange(a, b, dtype=np.uint32), "u64")
        parts_k.append(k)
        parts_v.append(v)
    kin = as_t(keys, "u64")
    kout = as_t(np.concatenate(parts_k), "u64")
    vout = torch.from_numpy(np.concatenate(parts_v).view(np.int32).copy())
    check_stable_sort_device(kin, kout, vout, "u64", offsets=offsets, chunk=1000)
    # The whole array sorted as one instance is not a valid batch output.
    k1, v1 = O.stable_sort(keys, np.arange(len(keys), dtype=np.uint32), "u64")
    with pytest.raises(AssertionError):
        check_stable_sort_device(kin, as_t(k1, "u64"), torch.from_numpy(v1.view(np.int32).copy()), "u64",
                                 offsets=offsets, chunk=1000)
