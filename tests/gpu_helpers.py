"""Call the CUDA path through the C ABI and bring its results back as numpy."""
from __future__ import annotations

import numpy as np
import torch

from paper_1611_00463_gb300 import pgs


def gpu_sort(keys: np.ndarray, vals: np.ndarray | None, P: int, dtype: str, in_place: bool = False,
             **opts) -> dict:
    """Run pgs_sort_copy (or pgs_sort) on device copies of keys/vals and return
    the sorted keys/vals, bucket bounds, cut matrix, splitters and stats."""
    dev = torch.device("cuda")
    n = len(keys)
    Peff = max(1, min(P, n)) if n else 1
    kin = pgs.as_device_keys(keys, dtype, dev)
    vin = torch.from_numpy(np.ascontiguousarray(vals).view(np.int32)).to(dev) if vals is not None else None
    cfg0 = pgs.make_config(dtype=dtype, **opts)
    ws = pgs.workspace(n, P, cfg0, device=dev)
    bounds = torch.full((Peff + 1,), -1, dtype=torch.int64, device=dev)
    cuts = torch.full((Peff * (Peff + 1),), -1, dtype=torch.int64, device=dev)
    spl = torch.zeros(max(Peff - 1, 1), dtype=kin.dtype, device=dev)
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device=dev)
    cfg = pgs.make_config(dtype=dtype, workspace=ws, bucket_bounds=bounds, cuts=cuts, splitters_out=spl,
                          stats=st, **opts)
    if in_place:
        kout, vout = kin, vin
        pgs.pgs_sort(kout, vout, P, cfg)
    else:
        kout = torch.empty_like(kin)
        vout = torch.empty_like(vin) if vin is not None else None
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg)
    torch.cuda.synchronize()
    out = {
        "keys": pgs.to_numpy_keys(kout, dtype),
        "vals": vout.cpu().numpy().view(np.uint32) if vout is not None else None,
        "e": bounds.cpu().numpy(),
        "cut": cuts.cpu().numpy().reshape(Peff, Peff + 1),
        "splitters": pgs.to_numpy_keys(spl, dtype)[:Peff - 1],
        "stats": pgs.pgs_get_stats(st) if n else None,
        "input_keys_after": pgs.to_numpy_keys(kin, dtype),
    }
    return out
