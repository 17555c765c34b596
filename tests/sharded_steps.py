"""Rank steps computed by the oracle on the host, for running the sharded
sort's collective choreography (paper_1611_00463_gb300.sharded) on CPU ranks.
Test infrastructure: the product uses the CUDA steps."""
from __future__ import annotations

import numpy as np
import torch

from oracle import pgs_oracle as O

NP = {"u32": np.uint32, "f32": np.uint32, "u64": np.uint64}
TORCH = {"u32": torch.int32, "f32": torch.int32, "u64": torch.int64}


def to_np(t, dtype):
    return t.numpy().view(NP[dtype])


def to_t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if dtype == "u64" else np.int32))


class OracleSteps:
    """Each step of Section IV for one rank, from the oracle's definitions.
    Splitters travel as order-form keys (the driver treats them as opaque)."""

    def __init__(self, dtype: str, s: int | None = None, variant: int = O.INVESTIGATOR_RANK):
        self.dtype, self.s, self.variant = dtype, s, variant

    def samples_per_run(self, G):
        return self.s or O.paper_samples_per_run(G, O.KEY_BYTES[self.dtype])

    def local_sort(self, keys, vals):
        k, v = O.stable_sort(to_np(keys, self.dtype), None if vals is None else vals.numpy().view(np.uint32),
                             self.dtype)
        return to_t(k, self.dtype), (None if v is None else torch.from_numpy(v.view(np.int32).copy()))

    def samples(self, sk, s):
        k = to_np(sk, self.dtype)
        return to_t(k[O.regular_sample_positions(len(k), s)], self.dtype)

    def splitters(self, all_samples, G):
        return to_t(O.select_splitters(O.ord_bits(to_np(all_samples, self.dtype), self.dtype), G), self.dtype)

    def counts(self, sk, spl, G):
        o = O.ord_bits(to_np(sk, self.dtype), self.dtype)
        t = to_np(spl, self.dtype)
        lb = np.searchsorted(o, t, side="left")
        ub = np.searchsorted(o, t, side="right")
        return torch.from_numpy(np.concatenate([lb, ub - lb]).astype(np.int64))

    def cuts(self, counts_all, sizes, spl, G):
        rows = counts_all.numpy().reshape(G, 2 * (G - 1))
        lb = np.zeros((G, G + 1), dtype=np.int64)
        cnt = np.zeros((G, G + 1), dtype=np.int64)
        lb[:, 1:G] = rows[:, :G - 1]
        cnt[:, 1:G] = rows[:, G - 1:]
        N = int(sum(sizes))
        L, Gs = lb.sum(axis=0), cnt.sum(axis=0)
        pre = np.cumsum(cnt, axis=0) - cnt
        e = np.zeros(G + 1, dtype=np.int64)
        e[G] = N
        for b in range(1, G):
            e[b] = min(max((b * N) // G, L[b]), L[b] + Gs[b])
        cut = np.zeros((G, G + 1), dtype=np.int64)
        cut[:, G] = sizes
        cut[:, 1:G] = lb[:, 1:G] + np.clip(e[None, 1:G] - L[None, 1:G] - pre[:, 1:G], 0, cnt[:, 1:G])
        return torch.from_numpy(cut), torch.from_numpy(e)

    def merge(self, rk, rv, off):
        k = to_np(rk, self.dtype)
        v = None if rv is None else rv.numpy().view(np.uint32)
        lists = [(k[off[j]:off[j + 1]], None if v is None else v[off[j]:off[j + 1]]) for j in range(len(off) - 1)]
        mk, mv = O.balanced_merge(lists, self.dtype)
        return to_t(mk, self.dtype), (None if mv is None else torch.from_numpy(mv.view(np.int32).copy()))
