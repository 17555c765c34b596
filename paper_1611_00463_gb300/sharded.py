"""The sort of one global array spread over the ranks of a process group.

Rank r holds shard r; the global input is the shards in rank order.  Every
rank runs the six steps of Section IV as one of the paper's processors, with
the library's CUDA kernels on its own GPU (`CudaSteps`, through the C ABI),
and the data moves between ranks by torch.distributed collectives:

1. local sort of the shard (pgs_sort_copy);
2. regular samples (pgs_rank_samples) -> all-gather (rank order);
3. splitters from all samples (pgs_fit_splitters), the same on every rank;
4. per-splitter counts (pgs_rank_counts) -> all-gather -> investigator cuts
   and bucket bounds (pgs_rank_cuts), the same on every rank;
5. all-to-all of the segments: rank r sends its sorted positions
   [cut[r][b], cut[r][b+1]) to rank b (sizes known on every rank);
6. merge of the received segments (pgs_merge_lists).

Rank b returns bucket b: the global stable ranks [e_b, e_{b+1}).  With NCCL
the collectives run on device tensors; with another backend (gloo) they are
staged through host memory.  There is no CPU fallback: the steps object is
the library unless a caller passes another one.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import pgs

KEY_DTYPE = {"u32": torch.int32, "f32": torch.int32, "u64": torch.int64}


class CudaSteps:
    """The rank steps on this rank's GPU (argument marshalling only)."""

    def __init__(self, dtype: str = "u32", device=None, P_local: int = 1, **opts):
        self.dtype = dtype
        self.device = torch.device(device or "cuda")
        self.P_local = P_local
        self.opts = opts

    def cfg(self, **extra):
        return pgs.make_config(dtype=self.dtype, **self.opts, **extra)

    def samples_per_run(self, G: int) -> int:
        return pgs.pgs_samples_per_run(G, self.cfg())

    def local_sort(self, keys, vals):
        n = keys.numel()
        kout, vout = torch.empty_like(keys), (torch.empty_like(vals) if vals is not None else None)
        if n:
            ws = pgs.workspace(n, self.P_local, self.cfg(), device=self.device)
            pgs.pgs_sort_copy(keys, vals, kout, vout, self.P_local, self.cfg(workspace=ws))
        return kout, vout

    def samples(self, sorted_keys, s: int):
        sr = min(s, sorted_keys.numel())
        out = torch.empty(sr, dtype=sorted_keys.dtype, device=self.device)
        if sr:
            pgs.pgs_rank_samples(sorted_keys, s, out, self.cfg())
        return out

    def splitters(self, all_samples, G: int):
        spl = torch.empty(max(G - 1, 1), dtype=all_samples.dtype, device=self.device)
        cfg0 = self.cfg()
        ws = torch.empty(pgs.pgs_fit_workspace_bytes(all_samples.numel(), G, cfg0), dtype=torch.uint8,
                         device=self.device)
        pgs.pgs_fit_splitters(all_samples, G, self.cfg(workspace=ws), spl)
        return spl[:G - 1]

    def counts(self, sorted_keys, splitters, G: int):
        out = torch.empty(2 * (G - 1), dtype=torch.int64, device=self.device)
        pgs.pgs_rank_counts(sorted_keys, splitters, G, out, self.cfg())
        return out

    def cuts(self, counts_all, sizes, splitters, G: int):
        cut = torch.empty((G, G + 1), dtype=torch.int64, device=self.device)
        e = torch.empty(G + 1, dtype=torch.int64, device=self.device)
        ws = torch.empty(pgs.pgs_rank_cuts_workspace_bytes(G, self.cfg()), dtype=torch.uint8, device=self.device)
        pgs.pgs_rank_cuts(counts_all, sizes, splitters, cut, e, self.cfg(workspace=ws))
        return cut, e

    def merge(self, keys, vals, offsets):
        n, k = int(offsets[-1]), len(offsets) - 1
        kout, vout = torch.empty_like(keys), (torch.empty_like(vals) if vals is not None else None)
        if n:
            ws = torch.empty(pgs.pgs_merge_workspace_bytes(n, k, self.cfg()), dtype=torch.uint8, device=self.device)
            pgs.pgs_merge_lists(keys, vals, offsets, kout, vout, self.cfg(workspace=ws))
        return kout, vout


class _Mover:
    """Collectives on the group: on device tensors for NCCL, else through host memory."""

    def __init__(self, group, device, stage_on_host: bool):
        self.group = group
        self.device = device
        self.stage = stage_on_host

    def _out(self, t):
        return t.cpu() if self.stage else t

    def _back(self, t):
        return t.to(self.device) if self.stage else t

    def all_gather_v(self, t, sizes):
        """Concatenation, in rank order, of every rank's 1-D tensor (rank q's has sizes[q] items)."""
        m = max(sizes) if sizes else 0
        pad = torch.zeros(max(m, 1), dtype=t.dtype, device=t.device)
        pad[:t.numel()] = t
        parts = [torch.empty_like(self._out(pad)) for _ in sizes]
        dist.all_gather(parts, self._out(pad), group=self.group)
        return self._back(torch.cat([p[:sz] for p, sz in zip(parts, sizes)]))

    def all_to_all_v(self, t, send, recv):
        out = torch.empty(int(sum(recv)), dtype=t.dtype, device=t.device)
        o = self._out(out)
        dist.all_to_all_single(o, self._out(t), [int(x) for x in recv], [int(x) for x in send], group=self.group)
        return self._back(o) if self.stage else o


def sharded_sort(keys: torch.Tensor, vals: torch.Tensor | None, group=None, dtype: str = "u32", steps=None,
                 stage_on_host: bool | None = None, **opts):
    """Sort the global array whose shard on this rank is `keys` (+ `vals`).

    Returns (bucket_keys, bucket_vals, bounds, cut): this rank's bucket of the
    stable sort of the concatenated shards, the bucket bounds e[0..G] (global
    stable ranks) and the cut matrix, both on every rank."""
    G = dist.get_world_size(group)
    r = dist.get_rank(group)
    steps = steps or CudaSteps(dtype, keys.device, **opts)
    if stage_on_host is None:
        stage_on_host = dist.get_backend(group) != "nccl"
    mv = _Mover(group, keys.device, stage_on_host)
    # Every rank's shard size.
    sizes = mv.all_gather_v(torch.tensor([keys.numel()], dtype=torch.int64, device=keys.device), [1] * G)
    sizes = [int(x) for x in sizes.cpu().tolist()]
    # Step 1.
    sk, sv = steps.local_sort(keys, vals)
    if G == 1:
        n = keys.numel()
        return sk, sv, torch.tensor([0, n], dtype=torch.int64), torch.tensor([[0, n]], dtype=torch.int64)
    # Step 2: samples, gathered in rank order.
    s = steps.samples_per_run(G)
    smp = steps.samples(sk, s)
    all_smp = mv.all_gather_v(smp, [min(s, sz) for sz in sizes])
    # Step 3: splitters, the same on every rank.
    spl = steps.splitters(all_smp, G)
    # Step 4: counts, gathered; the investigator's cuts, the same on every rank.
    cnt = steps.counts(sk, spl, G)
    cnt_all = mv.all_gather_v(cnt, [2 * (G - 1)] * G)
    cut, e = steps.cuts(cnt_all, sizes, spl, G)
    cut_h = np.asarray(cut.cpu()).astype(np.int64)
    # Step 5: the exchange.
    send = np.diff(cut_h[r])
    recv = cut_h[:, r + 1] - cut_h[:, r]
    rk = mv.all_to_all_v(sk, send, recv)
    rv = mv.all_to_all_v(sv, send, recv) if sv is not None else None
    # Step 6: merge what arrived, in rank order.
    off = np.concatenate([[0], np.cumsum(recv)]).astype(np.uint64)
    bk, bv = steps.merge(rk, rv, off)
    return bk, bv, e, cut
