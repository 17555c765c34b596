"""The paper's distributed form of the sort over torch.distributed ranks.

TEST INFRASTRUCTURE, NOT PRODUCT CODE (only the test suite imports it).  Each
rank is one of the paper's processors (Section IV): it sorts its own share
(step 1), contributes regular samples that every rank gathers (steps 2-3 with
the Master's choice made identically everywhere), binary-searches the
splitters in its sorted data and gathers everyone's counts so that the
investigator's cuts are the same on every rank (step 4, Section IV-B),
exchanges the segments (step 5, Section IV-C), and merges what it received
with the Fig. 2 schedule (step 6).  Local arithmetic comes from the oracle.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from oracle import pgs_oracle as O


def _allgather_array(x: np.ndarray) -> list[np.ndarray]:
    """All-gather a 1-D integer array of any length (lengths first, then padded data)."""
    world = dist.get_world_size()
    n = torch.tensor([len(x)], dtype=torch.int64)
    ns = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ns, n)
    m = max(int(v.item()) for v in ns)
    buf = torch.zeros(m, dtype=torch.int64)
    buf[:len(x)] = torch.from_numpy(x.astype(np.int64, copy=False).view(np.int64))
    out = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(out, buf)
    return [out[r][:int(ns[r].item())].numpy() for r in range(world)]


def sharded_sort(keys_local: np.ndarray, vals_local: np.ndarray, n_total: int, dtype: str, s: int,
                 variant: int = O.INVESTIGATOR_RANK):
    """Run steps 1-6 with this rank as processor `rank`; returns this rank's
    bucket (keys, vals) and the bucket vector e (identical on every rank)."""
    rank, P = dist.get_rank(), dist.get_world_size()
    kt = keys_local.dtype
    # Step 1.
    run_k, run_v = O.stable_sort(keys_local, vals_local, dtype)
    run_o = O.ord_bits(run_k, dtype).astype(np.uint64)
    # Step 2: regular samples to everyone (the Master's buffer on every rank).
    mine = run_o[O.regular_sample_positions(len(run_o), s)]
    gathered = _allgather_array(mine.view(np.int64))
    samples = np.concatenate([g.view(np.uint64) for g in gathered])
    # Step 3: every rank picks the same splitters.
    t = O.select_splitters(samples, P)
    # Step 4: local searches, everyone's counts, the same investigator cuts everywhere.
    lb = np.searchsorted(run_o, t, side="left").astype(np.int64)
    cnt = (np.searchsorted(run_o, t, side="right") - lb).astype(np.int64)
    lbs = _allgather_array(lb)
    cnts = _allgather_array(cnt)
    L = np.sum(lbs, axis=0)                     # the investigator needs only each run's counts
    G = np.sum(cnts, axis=0)
    e = np.zeros(P + 1, dtype=np.int64)
    e[P] = n_total
    for b in range(1, P):
        if variant == O.INVESTIGATOR_RANK:
            e[b] = min(max((b * n_total) // P, L[b - 1]), L[b - 1] + G[b - 1])
        elif variant == O.INVESTIGATOR_OFF:
            e[b] = L[b - 1] + G[b - 1]
        else:
            raise ValueError(variant)
    pre = np.cumsum(np.array(cnts), axis=0) - np.array(cnts)
    cut = np.zeros(P + 1, dtype=np.int64)
    cut[P] = len(run_o)
    for b in range(1, P):
        take = min(max(e[b] - L[b - 1] - pre[rank][b - 1], 0), cnts[rank][b - 1])
        cut[b] = lbs[rank][b - 1] + take
    # Step 5: every segment to its bucket's rank.
    send_k = [run_k[cut[b]:cut[b + 1]] for b in range(P)]
    send_v = [run_v[cut[b]:cut[b + 1]] for b in range(P)]
    recv_k, recv_v = [None] * P, [None] * P
    for b in range(P):                          # rank b gathers every rank's segment b
        got_k = _allgather_array(send_k[b].view(np.int64) if kt == np.uint64 else send_k[b].astype(np.int64))
        got_v = _allgather_array(send_v[b].astype(np.int64))
        if b == rank:
            recv_k = [g.view(np.uint64) if kt == np.uint64 else g.astype(kt) for g in got_k]
            recv_v = [g.astype(np.uint32) for g in got_v]
    # Step 6: the Fig. 2 merge of the received segments (run order = rank order).
    merged = O.balanced_merge(list(zip(recv_k, recv_v)), dtype)
    return merged[0], merged[1], e
