"""CPU oracle for the load-balanced sample sort of "A Load-Balanced Parallel and
Distributed Sorting Algorithm Implemented with PGX.D" (arXiv 1611.00463).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import or run this module.  It shares
no code with the CUDA path and never takes an input or an expected value from it.

Plain numpy, single threaded, written for a reader to check against the paper by
eye.  Library sorts (``numpy.argsort(kind="stable")``) and binary searches
(``numpy.searchsorted``) serve as steps; nothing is blocked, fused or reordered.

Two things are computed:

* Part 1, the sorted output.  The method reaches exactly the plain result: a
  stable ascending sort on the key's total order, payload carried along
  (Section IV: smaller entries end on lower-numbered processors, and each entry
  keeps where it came from, step 6).  ``stable_sort`` is that definition.
* Part 2, the method's own steps in the paper's order (Section IV, steps 1-6;
  Section IV-A, Fig. 2 balanced merge; Section IV-B, sample budget and the
  investigator), giving the bucket vector e[0..P], the per-run cut matrix, the
  exchange offsets and, after the per-bucket merges, again the sorted output.
  The investigator also has the text's literal per-run rule (LOCAL), whose
  output keys are sorted but not in stable order.
* Part 3, lookups on the sorted output (end of Section IV-C): lower and upper
  bounds of query keys, the bucket holding a position, and every entry's
  previous processor and index.

Readings of points the paper leaves open (each is listed in the design notes):
sample positions are the last element of s equal blocks of a sorted run; the
Master takes every (S/P)-th sample as a splitter; bucket b receives the
stable-rank range [e_b, e_{b+1}); the default investigator cuts every splitter
at its ideal rank floor(b*N/P) clamped into the splitter's duplicate range, and
it divides that range by global stable rank so the output stays stable.

Parity pins: every function below is pinned by tests that do not re-run its own
formula (brute force, closed forms, invariants and the balance bound); none is
"parity unpinned" except the learned-CDF training, which the tests pin only by
properties (see ``mlp_*``).
"""
from __future__ import annotations

import numpy as np

DTYPES = {"u32": np.uint32, "u64": np.uint64, "f32": np.uint32}
KEY_BYTES = {"u32": 4, "u64": 8, "f32": 4}

INVESTIGATOR_RANK = 0      # default: cut at rank floor(bN/P) clamped into [L_b, L_b+G_b]
INVESTIGATOR_EQUAL = 1     # a group of k equal splitters splits the value's range into k equal parts
INVESTIGATOR_OFF = 2       # plain binary search (upper bound), the failure mode of Fig. 5(b)
INVESTIGATOR_LOCAL = 3     # the text's literal rule: every run divides its own range of the value

SAMPLE_BUFFER_BYTES = 262144   # the 256 KB read buffer of Section IV-B


# ---------------------------------------------------------------------------
# Key order
# ---------------------------------------------------------------------------

def ord_bits(keys: np.ndarray, dtype: str) -> np.ndarray:
    """Unsigned integer whose natural order is the key order.

    Integer keys are their own order.  float32 keys (passed as uint32 bit
    patterns) follow IEEE-754 totalOrder: negative values have every bit
    flipped, non-negative ones get the sign bit set, so
    -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN.
    The paper only sorts integers; this ordering is the reading for floats.
    """
    if dtype in ("u32", "u64"):
        return keys
    if dtype != "f32":
        raise ValueError(dtype)
    b = keys.astype(np.uint32, copy=False)
    neg = (b >> np.uint32(31)) == 1
    return np.where(neg, ~b, b | np.uint32(0x80000000)).astype(np.uint32)


# ---------------------------------------------------------------------------
# Part 1: the sorted output (definition)
# ---------------------------------------------------------------------------

def stable_sort(keys: np.ndarray, vals: np.ndarray | None, dtype: str):
    """Stable ascending sort by ord(key); the payload travels with its key.

    Section IV (end of IV-C): after the sort smaller entries sit on processors
    with smaller IDs, and each entry's previous processor and index are kept
    (step 6).  Equal keys keep their input order.
    """
    order = np.argsort(ord_bits(keys, dtype), kind="stable")
    return keys[order], (None if vals is None else vals[order])


# ---------------------------------------------------------------------------
# Part 2: the method, step by step
# ---------------------------------------------------------------------------

def effective_partitions(n: int, P: int) -> int:
    """P logical processors; more processors than keys collapse to one per key."""
    if P < 1:
        raise ValueError("P must be >= 1")
    return max(1, min(P, n))


def run_bounds(n: int, P: int) -> np.ndarray:
    """Processor r owns input positions [floor(r n / P), floor((r+1) n / P)).

    Step 1 of Section IV gives every processor its own share of the data; the
    floor split is the reading for n not divisible by P.
    """
    return np.array([(r * n) // P for r in range(P + 1)], dtype=np.int64)


def balanced_merge_schedule(k: int) -> list[list[tuple[int, int]]]:
    """Rounds of the balanced pairwise merge of Fig. 2 (Section IV-A).

    Round j merges list i + 2^j into list i for every i that is a multiple of
    2^(j+1) with i + 2^j < k; each pair is (destination, source).  For k = 8:
    (0<-1, 2<-3, 4<-5, 6<-7), then (0<-2, 4<-6), then (0<-4).
    """
    rounds = []
    step = 1
    while step < k:
        rounds.append([(i, i + step) for i in range(0, k, 2 * step) if i + step < k])
        step *= 2
    return rounds


def merge_two(ka, va, kb, vb, dtype):
    """Stable merge of two sorted lists; on equal keys the first list wins."""
    k = np.concatenate([ka, kb])
    v = None if va is None else np.concatenate([va, vb])
    order = np.argsort(ord_bits(k, dtype), kind="stable")
    return k[order], (None if v is None else v[order])


def balanced_merge(lists, dtype):
    """Merge sorted (keys, vals) lists with the schedule of Fig. 2."""
    if not lists:
        return None
    cur = list(lists)
    for rnd in balanced_merge_schedule(len(cur)):
        for dst, src in rnd:
            ka, va = cur[dst]
            kb, vb = cur[src]
            cur[dst] = merge_two(ka, va, kb, vb, dtype)
    return cur[0]


def local_sort(keys, vals, dtype, threads: int = 32):
    """Step 1 of Section IV and Section IV-A: split a processor's data equally
    over worker threads, sort each piece, then merge the pieces with Fig. 2."""
    n = len(keys)
    t = max(1, min(threads, n))
    cuts = [(i * n) // t for i in range(t + 1)]
    pieces = []
    for i in range(t):
        pk, pv = stable_sort(keys[cuts[i]:cuts[i + 1]],
                             None if vals is None else vals[cuts[i]:cuts[i + 1]], dtype)
        pieces.append((pk, pv))
    if not pieces:
        return keys[:0], (None if vals is None else vals[:0])
    return balanced_merge(pieces, dtype)


def paper_samples_per_run(P: int, key_bytes: int) -> int:
    """Section IV-B: each processor sends 256/p KB of samples to the Master.

    Read as floor(262144 / (P * key_bytes)) keys per processor (keys only).
    """
    return max(1, SAMPLE_BUFFER_BYTES // (P * key_bytes))


def guaranteed_samples_per_run(P: int, eps: float) -> int:
    """Samples per run so that the balance bound 1 + P/s is at most 1 + eps."""
    return int(np.ceil(P / eps))


def regular_sample_positions(n_r: int, s: int) -> np.ndarray:
    """Step 2 of Section IV: regular samples of a sorted run.

    Reading: the run is cut into s_r = min(s, n_r) equal blocks and the last
    element of each block is sampled, local position floor((i+1) n_r / s_r) - 1.
    """
    s_r = min(s, n_r)
    if s_r == 0:
        return np.zeros(0, dtype=np.int64)
    i = np.arange(1, s_r + 1, dtype=np.int64)
    return (i * n_r) // s_r - 1


def select_splitters(samples_ord: np.ndarray, P: int) -> np.ndarray:
    """Step 3 of Section IV: the Master sorts the gathered samples and picks P-1
    final splitters.  Reading (regular sampling, as in PSRS): with S samples,
    splitter t_b is the sample at sorted index floor(b S / P) - 1, b = 1..P-1.
    The samples arrive in (run, position) order, so a stable sort orders them by
    (key, run, position)."""
    S = len(samples_ord)
    srt = samples_ord[np.argsort(samples_ord, kind="stable")]
    idx = [(b * S) // P - 1 for b in range(1, P)]
    if any(i < 0 for i in idx):
        raise ValueError("fewer samples than partitions")
    return srt[np.array(idx, dtype=np.int64)] if idx else srt[:0]


def investigator(run_ord: list[np.ndarray], t: np.ndarray, n: int, P: int,
                 variant: int = INVESTIGATOR_RANK):
    """Step 4 of Section IV with the investigator of Section IV-B (Fig. 5).

    For splitter t_b on sorted run r: lb[r,b] = #{x < t_b} and cnt[r,b] = #{x = t_b}
    (two binary searches).  Over all runs, L_b = sum_r lb, G_b = sum_r cnt and
    pre[r,b] = sum_{r'<r} cnt[r',b].  The global target e_b picks how many stable
    ranks go to buckets 0..b-1:

    * RANK (default): e_b = clamp(floor(b n / P), L_b, L_b + G_b).  A value that
      spans several splitters is split at each one's ideal rank, so its range is
      divided into equal N/P pieces.
    * EQUAL: a maximal group t_j = ... = t_{j+k-1} of k duplicated splitters gets
      e_{j+i} = L + floor(G (i+1) / k); a splitter that is not duplicated is cut
      by plain binary search (upper bound), as the paper states.
    * OFF: plain upper bound everywhere, e_b = L_b + G_b (Fig. 5(b)).

    Each run gives bucket b its elements of stable rank [e_b, e_{b+1}):
    cut[r,b] = lb[r,b] + clamp(e_b - L_b - pre[r,b], 0, cnt[r,b]), with
    cut[r,0] = 0 and cut[r,P] = n_r.

    * LOCAL, the rule as Section IV-B words it ("during searching for each
      splitter on local data entries"): every run divides its own range of a
      duplicated value, so for a group of k equal splitters starting at b,
      cut[r, b+i] = lb[r,b] + floor(cnt[r,b] (i+1) / k), i = 0..k-1, and a
      splitter that is not duplicated cuts at the upper bound; e is then the sum
      of the cuts over runs.  Keys end sorted, but equal keys are ordered by
      bucket, then run, not by input position (not stable).

    Returns (e, cut, lb, cnt).
    """
    R = len(run_ord)
    lb = np.zeros((R, P + 1), dtype=np.int64)
    cnt = np.zeros((R, P + 1), dtype=np.int64)
    for r in range(R):
        lb[r, 1:P] = np.searchsorted(run_ord[r], t, side="left")
        cnt[r, 1:P] = np.searchsorted(run_ord[r], t, side="right") - lb[r, 1:P]
    L = lb.sum(axis=0)
    G = cnt.sum(axis=0)
    pre = np.cumsum(cnt, axis=0) - cnt

    if variant == INVESTIGATOR_LOCAL:
        cut = np.zeros((R, P + 1), dtype=np.int64)
        cut[:, P] = [len(x) for x in run_ord]
        b = 1
        while b < P:
            k = 1
            while b + k < P and t[b + k - 1] == t[b - 1]:
                k += 1
            for i in range(k):
                cut[:, b + i] = lb[:, b] + (cnt[:, b] * (i + 1)) // k
            b += k
        return cut.sum(axis=0), cut, lb, cnt

    e = np.zeros(P + 1, dtype=np.int64)
    e[P] = n
    if variant == INVESTIGATOR_RANK:
        for b in range(1, P):
            e[b] = min(max((b * n) // P, L[b]), L[b] + G[b])
    elif variant == INVESTIGATOR_OFF:
        for b in range(1, P):
            e[b] = L[b] + G[b]
    elif variant == INVESTIGATOR_EQUAL:
        b = 1
        while b < P:
            k = 1
            while b + k < P and t[b + k - 1] == t[b - 1]:
                k += 1
            for i in range(k):
                e[b + i] = L[b] + (G[b] * (i + 1)) // k
            b += k
    else:
        raise ValueError(variant)

    cut = np.zeros((R, P + 1), dtype=np.int64)
    cut[:, P] = [len(x) for x in run_ord]
    take = np.clip(e[None, 1:P] - L[None, 1:P] - pre[:, 1:P], 0, cnt[:, 1:P])
    cut[:, 1:P] = lb[:, 1:P] + take
    return e, cut, lb, cnt


def exchange_offsets(cut: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Section IV-C: once the ranges are broadcast every receiver knows how much
    it gets from each sender and writes at an offset.  Segment (r, b) lands at
    dst[r,b] = e_b + sum_{r'<r} (cut[r',b+1] - cut[r',b])."""
    R, P1 = cut.shape
    P = P1 - 1
    size = cut[:, 1:] - cut[:, :-1]
    before = np.cumsum(size, axis=0) - size          # sum over r' < r
    dst = e[None, :P] + before
    return dst


def load_stats(e: np.ndarray) -> dict:
    """Per-processor data size after the sort (Table II): sizes and max/mean."""
    sizes = np.diff(e)
    P = len(sizes)
    n = int(e[-1])
    mean = n / P if P else 0.0
    return {
        "sizes": sizes,
        "max": int(sizes.max()) if P else 0,
        "min": int(sizes.min()) if P else 0,
        "max_over_mean": (float(sizes.max()) / mean) if mean > 0 else 1.0,
    }


def sample_sort(keys: np.ndarray, vals: np.ndarray | None, P: int, dtype: str,
                samples_per_run: int | None = None,
                variant: int = INVESTIGATOR_RANK, threads: int = 32) -> dict:
    """The six steps of Section IV on P logical processors.

    1. every processor sorts its run (``local_sort``);
    2. regular samples of each sorted run go to the Master;
    3. the Master picks P-1 splitters;
    4. binary searches plus the investigator give each run's send ranges;
    5. every segment is written at its receive offset (the exchange);
    6. each receiver merges its P segments with the Fig. 2 schedule.

    Returns every intermediate result and the final keys/vals, which equal
    ``stable_sort`` for the RANK, EQUAL and OFF variants; with LOCAL the keys
    equal it and equal keys are ordered by bucket, then run.
    """
    n = len(keys)
    P = effective_partitions(n, P)
    wbytes = KEY_BYTES[dtype]
    s = paper_samples_per_run(P, wbytes) if samples_per_run is None else samples_per_run
    bounds = run_bounds(n, P)

    # Step 1.
    runs = []
    for r in range(P):
        lo, hi = bounds[r], bounds[r + 1]
        runs.append(local_sort(keys[lo:hi], None if vals is None else vals[lo:hi], dtype, threads))
    run_ord = [ord_bits(k, dtype) for k, _ in runs]

    # Step 2.
    sample_list = [run_ord[r][regular_sample_positions(len(run_ord[r]), s)] for r in range(P)]
    samples = np.concatenate(sample_list) if sample_list else np.zeros(0, run_ord[0].dtype)

    # Step 3.
    t = select_splitters(samples, P)

    # Step 4.
    e, cut, lb, cnt = investigator(run_ord, t, n, P, variant)

    # Step 5.
    dst = exchange_offsets(cut, e)
    out_k = np.empty_like(keys)
    out_v = None if vals is None else np.empty_like(vals)
    for r in range(P):
        rk, rv = runs[r]
        for b in range(P):
            a, z = cut[r, b], cut[r, b + 1]
            out_k[dst[r, b]:dst[r, b] + (z - a)] = rk[a:z]
            if vals is not None:
                out_v[dst[r, b]:dst[r, b] + (z - a)] = rv[a:z]

    # Step 6.
    for b in range(P):
        segs = []
        for r in range(P):
            lo = dst[r, b]
            hi = lo + cut[r, b + 1] - cut[r, b]
            segs.append((out_k[lo:hi], None if vals is None else out_v[lo:hi]))
        mk, mv = balanced_merge(segs, dtype)
        out_k[e[b]:e[b + 1]] = mk
        if vals is not None:
            out_v[e[b]:e[b + 1]] = mv

    return {
        "P": P, "s": s, "bounds": bounds, "samples": samples, "splitters": t,
        "e": e, "cut": cut, "lb": lb, "cnt": cnt, "dst": dst,
        "keys": out_k, "vals": out_v, "stats": load_stats(e),
    }


def buckets(keys: np.ndarray, P: int, dtype: str, samples_per_run: int | None = None,
            variant: int = INVESTIGATOR_RANK) -> dict:
    """Steps 1-4 only (no exchange, no merge): the bucket vector and cut matrix.

    Step 1 here uses a plain stable sort of each run, which the local_sort tests
    show to be the same result as the Fig. 2 thread merge.
    """
    n = len(keys)
    P = effective_partitions(n, P)
    s = paper_samples_per_run(P, KEY_BYTES[dtype]) if samples_per_run is None else samples_per_run
    bounds = run_bounds(n, P)
    o = ord_bits(keys, dtype)
    run_ord = [np.sort(o[bounds[r]:bounds[r + 1]], kind="stable") for r in range(P)]
    samples = np.concatenate([run_ord[r][regular_sample_positions(len(run_ord[r]), s)]
                              for r in range(P)])
    t = select_splitters(samples, P)
    e, cut, lb, cnt = investigator(run_ord, t, n, P, variant)
    return {"P": P, "s": s, "bounds": bounds, "splitters": t, "e": e, "cut": cut,
            "stats": load_stats(e)}


# ---------------------------------------------------------------------------
# Learned-CDF splitters (not in the paper): a 1 -> 32 -> 32 -> 1 ReLU model of
# the key CDF, trained on the method's own sample, predicts bucket ids; the
# sampled splitters with the investigator judge its imbalance.
#
# Monotone by construction: units 0..15 see +x through positive weights and
# enter the output with positive weights (a rising convex part); units 16..31
# see -x and enter with negative weights (a rising concave part); layer 2 only
# connects units of the same half, with positive weights.  Every fp32
# operation of the evaluation is monotone in the right direction, so the fp32
# bucket id is non-decreasing in the key and the buckets are key ranges.
#
# Parity: bucket ids are pinned bit for bit (same fp32 operation order on both
# sides, no fused multiply-add); training is "parity unpinned" bit for bit and
# pinned by its properties (finite-difference gradients, loss decrease,
# monotonicity, loss close to this fp64 reference trainer).
# ---------------------------------------------------------------------------

MLP_H = 32
MLP_HALF = 16
MLP_FLOATS = 1 * 32 + 32 + 32 * 32 + 32 + 32 * 1 + 1
MLP_STEPS = 300
MLP_LR = 0.01
MLP_OFF_DIAG = -6.0


def mlp_block_mask() -> np.ndarray:
    """W2[k, j] exists only when units k and j are in the same half."""
    i = np.arange(MLP_H)
    return (i[:, None] < MLP_HALF) == (i[None, :] < MLP_HALF)


def mlp_sign() -> np.ndarray:
    return np.where(np.arange(MLP_H) < MLP_HALF, 1.0, -1.0)


def mlp_norm(sorted_sample_ord: np.ndarray):
    """Input normalisation: x = f32(f64(max(k, kmin) - kmin)) * scale with
    scale = f32(1) / f32(f64(kmax - kmin)) (0 when every sample is equal)."""
    kmin = int(sorted_sample_ord[0])
    span = int(sorted_sample_ord[-1]) - kmin
    scale = np.float32(0.0) if span == 0 else np.float32(1.0) / np.float32(np.float64(span))
    return kmin, np.float32(scale)


def mlp_inputs(keys_ord: np.ndarray, kmin: int, scale: np.float32) -> np.ndarray:
    d = np.maximum(keys_ord.astype(np.uint64), np.uint64(kmin)) - np.uint64(kmin)
    return d.astype(np.float64).astype(np.float32) * np.float32(scale)


def mlp_init(x_sorted: np.ndarray) -> dict:
    """Deterministic start: layer-1 knots at the training inputs of sorted index
    floor((j + 1/2) m / 16), layer 2 close to the identity inside each half."""
    m = len(x_sorted)
    q = np.array([float(x_sorted[((2 * j + 1) * m) // (2 * MLP_HALF)]) for j in range(MLP_HALF)])
    b1 = np.concatenate([-q, q])
    V2 = np.where(np.eye(MLP_H, dtype=bool), 0.0, MLP_OFF_DIAG)
    V2 = np.where(mlp_block_mask(), V2, 0.0)
    return {"v1": np.zeros(MLP_H), "b1": b1, "V2": V2, "b2": np.zeros(MLP_H),
            "v3": np.full(MLP_H, np.log(1.0 / MLP_H)), "b3": np.array(0.5)}


def mlp_effective(raw: dict) -> dict:
    """Signed, exponentiated weights of the monotone network."""
    s = mlp_sign()
    mask = mlp_block_mask()
    return {"w1": s * np.exp(raw["v1"]), "b1": raw["b1"],
            "W2": np.where(mask, np.exp(np.where(mask, raw["V2"], 0.0)), 0.0), "b2": raw["b2"],
            "w3": s * np.exp(raw["v3"]), "b3": raw["b3"]}


def mlp_forward64(eff: dict, x: np.ndarray):
    z1 = x[:, None] * eff["w1"] + eff["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ eff["W2"].T + eff["b2"]
    h2 = np.maximum(z2, 0.0)
    return h2 @ eff["w3"] + eff["b3"], (z1, h1, z2, h2)


def mlp_loss_grad(raw: dict, x: np.ndarray, t: np.ndarray):
    """Mean squared error of the CDF fit and its gradient in the raw parameters."""
    eff = mlp_effective(raw)
    y, (z1, h1, z2, h2) = mlp_forward64(eff, x)
    m = len(x)
    r = y - t
    dy = 2.0 * r / m
    g = {"b3": np.array(dy.sum())}
    g["v3"] = (h2.T @ dy) * eff["w3"]                       # d w3 / d v3 = w3
    dz2 = (dy[:, None] * eff["w3"]) * (z2 > 0)
    g["b2"] = dz2.sum(axis=0)
    g["V2"] = np.where(mlp_block_mask(), (dz2.T @ h1) * eff["W2"], 0.0)
    dz1 = (dz2 @ eff["W2"]) * (z1 > 0)
    g["b1"] = dz1.sum(axis=0)
    g["v1"] = (dz1 * x[:, None]).sum(axis=0) * eff["w1"]
    return float(np.mean(r * r)), g


def mlp_train(x_sorted: np.ndarray, steps: int = MLP_STEPS, lr: float = MLP_LR):
    """Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) on targets (i + 1/2)/m,
    in float64.  Returns the raw parameters and the loss before the last step."""
    x = np.asarray(x_sorted, dtype=np.float64)
    m = len(x)
    t = (np.arange(m) + 0.5) / m
    raw = mlp_init(x)
    mom = {k: np.zeros_like(v) for k, v in raw.items()}
    vel = {k: np.zeros_like(v) for k, v in raw.items()}
    mask = mlp_block_mask()
    loss = None
    for step in range(1, steps + 1):
        loss, g = mlp_loss_grad(raw, x, t)
        for k in raw:
            mom[k] = 0.9 * mom[k] + 0.1 * g[k]
            vel[k] = 0.999 * vel[k] + 0.001 * g[k] * g[k]
            upd = lr * (mom[k] / (1 - 0.9 ** step)) / (np.sqrt(vel[k] / (1 - 0.999 ** step)) + 1e-8)
            raw[k] = raw[k] - (np.where(mask, upd, 0.0) if k == "V2" else upd)
    return raw, loss


def mlp_pack(eff: dict) -> np.ndarray:
    """The 1153 float32 weights in library order: w1, b1, W2 (row k, column j), b2, w3, b3."""
    return np.concatenate([eff["w1"], eff["b1"], eff["W2"].reshape(-1), eff["b2"], eff["w3"],
                           np.atleast_1d(eff["b3"])]).astype(np.float32)


def mlp_unpack(w: np.ndarray) -> dict:
    w = np.asarray(w, dtype=np.float32)
    return {"w1": w[0:32], "b1": w[32:64], "W2": w[64:1088].reshape(32, 32), "b2": w[1088:1120],
            "w3": w[1120:1152], "b3": w[1152]}


def mlp_monotone(w: np.ndarray) -> bool:
    """Sign pattern that makes the network non-decreasing (off-half W2 entries are unused)."""
    e = mlp_unpack(w)
    A = slice(0, MLP_HALF)
    Bh = slice(MLP_HALF, MLP_H)
    return bool(np.all(e["w1"][A] >= 0) and np.all(e["w1"][Bh] <= 0) and np.all(e["W2"][A, A] >= 0)
                and np.all(e["W2"][Bh, Bh] >= 0) and np.all(e["w3"][A] >= 0) and np.all(e["w3"][Bh] <= 0))


def mlp_bucket_f32(w: np.ndarray, x32: np.ndarray, P: int) -> np.ndarray:
    """Bucket id min(P-1, floor(P * clamp(y, 0, 1))) with y evaluated in float32 in
    this exact order (every product and sum rounded, no fused multiply-add):
    h1_j = max(w1_j x + b1_j, 0); acc = b2_k, acc += W2_kj h1_j over j of k's half
    in increasing j, h2_k = max(acc, 0); y = b3, y += w3_k h2_k for k = 0..31."""
    e = mlp_unpack(w)
    f = np.float32
    x32 = np.asarray(x32, dtype=np.float32)
    h1 = [np.maximum(e["w1"][j] * x32 + e["b1"][j], f(0)) for j in range(MLP_H)]
    h2 = []
    for k in range(MLP_H):
        acc = np.full(x32.shape, e["b2"][k], dtype=np.float32)
        lo = 0 if k < MLP_HALF else MLP_HALF
        for j in range(lo, lo + MLP_HALF):
            acc = acc + e["W2"][k, j] * h1[j]
        h2.append(np.maximum(acc, f(0)))
    y = np.full(x32.shape, e["b3"], dtype=np.float32)
    for k in range(MLP_H):
        y = y + e["w3"][k] * h2[k]
    c = np.minimum(np.maximum(y, f(0)), f(1))
    b = np.floor(f(P) * c).astype(np.int64)
    return np.minimum(b, P - 1)


def learned_buckets(keys: np.ndarray, P: int, dtype: str, w: np.ndarray, kmin: int, scale) -> dict:
    """Steps 1 and 4 with model bucket ids: every run sorted, every key's bucket
    from the model, cut[r][b] = #keys of run r with bucket id < b, e_b = sum_r cut."""
    n = len(keys)
    P = effective_partitions(n, P)
    bounds = run_bounds(n, P)
    o = ord_bits(keys, dtype)
    cut = np.zeros((P, P + 1), dtype=np.int64)
    for r in range(P):
        run = np.sort(o[bounds[r]:bounds[r + 1]], kind="stable")
        ids = mlp_bucket_f32(w, mlp_inputs(run, kmin, scale), P)
        hist = np.bincount(ids, minlength=P)
        cut[r, 1:] = np.cumsum(hist)
    e = cut.sum(axis=0)
    return {"P": P, "cut": cut, "e": e, "stats": load_stats(e)}


# ---------------------------------------------------------------------------
# Lookups on the sorted output (Section IV-C: the library lets users binary
# search the sorted data and find every entry's previous processor and index).
# ---------------------------------------------------------------------------

def search(sorted_keys: np.ndarray, queries: np.ndarray, dtype: str, side: str = "left") -> np.ndarray:
    """Position of every query in the sorted keys, by key order: "left" gives
    the number of keys ordered before the query (lower bound), "right" the
    number ordered before or equal to it (upper bound)."""
    return np.searchsorted(ord_bits(sorted_keys, dtype), ord_bits(queries, dtype), side=side).astype(np.int64)


def bucket_of(pos: np.ndarray, e: np.ndarray) -> np.ndarray:
    """The bucket (processor) whose output range [e_b, e_{b+1}) holds position
    pos; a position equal to n (past the last key) maps to P, and an empty
    bucket holds no position."""
    P = len(e) - 1
    b = np.searchsorted(e, pos, side="right") - 1
    return np.where(pos >= e[P], P, b).astype(np.int64)


def provenance(vals: np.ndarray, n: int, P: int):
    """Previous processor and index of every entry whose payload is its input
    position: run r = the one with run_bounds[r] <= v < run_bounds[r+1]; the
    index inside it is v - run_bounds[r] (step 6 keeps this provenance)."""
    P = effective_partitions(n, P)
    bounds = run_bounds(n, P)
    v = vals.astype(np.int64)
    r = np.searchsorted(bounds, v, side="right") - 1
    return r.astype(np.int64), (v - bounds[r]).astype(np.int64)
