"""Seeded synthetic workloads for the load-balanced sample sort.

This module only draws random keys; it holds none of the sort's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  The paper measures on
one billion entries drawn from uniform, normal, right-skewed and exponential
distributions (Section V, "Different types of data distribution"); its
distribution parameters exist only in a figure, so the recipes below stand in
for them.

Every generator is deterministic in (n, seed) and independent of the number of
host threads: the key stream is cut into chunks of ``CHUNK`` keys and chunk c is
drawn from its own PCG64 stream seeded by ``SeedSequence(seed, spawn_key=(c,))``.
Per-workload constants (the 1000 distinct Zipf values, the instance sizes of the
batched workload) come from a separate "setup" stream, ``spawn_key=(SETUP,)``.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

CHUNK = 1 << 22
SETUP = 0xFFFFFFFF
U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)
U32_MAX = 0xFFFFFFFF

# IEEE-754 single bit patterns mixed into the duplicate-heavy workload.
F32_SPECIALS = np.array([0x00000000, 0x80000000, 0x7FC00000, 0xFFC00000], dtype=np.uint32)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(stream,))))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _chunked(n: int, seed: int, dtype, fill) -> np.ndarray:
    """Fill an n-vector chunk by chunk; ``fill(rng, m)`` returns m keys of ``dtype``."""
    out = np.empty(n, dtype=dtype)
    nchunks = (n + CHUNK - 1) // CHUNK

    def work(c: int) -> None:
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        out[lo:hi] = fill(_rng(seed, c), hi - lo)

    if nchunks <= 1:
        for c in range(nchunks):
            work(c)
    else:
        with _cf.ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(nchunks)))
    return out


def _f64_to_u64_clamped(x: np.ndarray) -> np.ndarray:
    """Round to nearest integer and clamp into [0, 2^64 - 1] (values >= 2^64 saturate)."""
    x = np.rint(x)
    out = np.empty(x.shape, dtype=np.uint64)
    hi = x >= 2.0**63
    lo = ~hi
    # float64 -> uint64 is done in two halves so no platform conversion rule matters.
    out[lo] = np.maximum(x[lo], 0.0).astype(np.int64).astype(np.uint64)
    top = x[hi]
    sat = top >= 2.0**64
    part = np.where(sat, 0.0, top - 2.0**63).astype(np.int64).astype(np.uint64)
    part = part + np.uint64(1 << 63)
    part[sat] = U64_MAX
    out[hi] = part
    return out


# ---------------------------------------------------------------------------
# Key distributions
# ---------------------------------------------------------------------------

def uniform_u32(n: int, seed: int = 0) -> np.ndarray:
    """Uniform uint32 keys on [0, 2^32)."""
    return _chunked(n, seed, np.uint32,
                    lambda g, m: g.integers(0, 1 << 32, size=m, dtype=np.uint64).astype(np.uint32))


def uniform_u64(n: int, seed: int = 0) -> np.ndarray:
    """Uniform uint64 keys on [0, 2^64)."""
    return _chunked(n, seed, np.uint64,
                    lambda g, m: g.integers(0, 1 << 64, size=m, dtype=np.uint64, endpoint=False))


def normal_lognormal_u64(n: int, seed: int = 1) -> np.ndarray:
    """Half normal (mean 2^63, sigma 2^60), half right-skewed lognormal (mu 40, sigma 2).

    Per key a fair coin picks the branch; both are rounded and clamped into uint64,
    so about 1.5 % of the lognormal half saturates at 2^64 - 1 (a long duplicate run).
    """
    def fill(g, m):
        heads = g.random(m) < 0.5
        nrm = 2.0**63 + 2.0**60 * g.standard_normal(m)
        lgn = g.lognormal(mean=40.0, sigma=2.0, size=m)
        return _f64_to_u64_clamped(np.where(heads, nrm, lgn))
    return _chunked(n, seed, np.uint64, fill)


def zipf_values_f32(seed: int, distinct: int = 1000) -> np.ndarray:
    """The distinct finite non-zero float32 values of the Zipf workload, in rank order."""
    g = _rng(seed, SETUP)
    vals: list[float] = []
    seen: set[int] = set()
    while len(vals) < distinct:
        cand = (1000.0 * g.standard_normal(distinct - len(vals))).astype(np.float32)
        for v in cand:
            b = int(v.view(np.uint32))
            if not np.isfinite(v) or v == 0.0 or b in seen:
                continue
            seen.add(b)
            vals.append(float(v))
    table = np.array(vals, dtype=np.float32)
    return table[g.permutation(distinct)]


def zipf_cdf(distinct: int, s: float) -> np.ndarray:
    w = np.arange(1, distinct + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_dup_f32(n: int, seed: int = 2, distinct: int = 1000, s: float = 1.1,
                 special_rate: float = 0.05) -> np.ndarray:
    """Duplicate-heavy float32 keys (returned as their uint32 bit patterns).

    Keys take one of ``distinct`` values with Zipf(s) frequencies (rank k has
    weight k^-s); with probability ``special_rate`` a key is replaced by one of
    +0.0, -0.0, +NaN (0x7FC00000) or -NaN (0xFFC00000), chosen uniformly.
    """
    table = zipf_values_f32(seed, distinct).view(np.uint32)
    cdf = zipf_cdf(distinct, s)

    def fill(g, m):
        rank = np.searchsorted(cdf, g.random(m), side="right")
        np.minimum(rank, distinct - 1, out=rank)
        keys = table[rank]
        mask = g.random(m) < special_rate
        pick = g.integers(0, 4, size=m)
        keys[mask] = F32_SPECIALS[pick[mask]]
        return keys
    return _chunked(n, seed, np.uint32, fill)


def exponential_u32(n: int, seed: int = 3, scale: float = 1e8) -> np.ndarray:
    """uint32 keys rint(Exp(scale)) clamped to 2^32 - 1 (lambda = 1/scale)."""
    def fill(g, m):
        x = np.rint(g.exponential(scale, size=m))
        return np.minimum(x, float(U32_MAX)).astype(np.uint32)
    return _chunked(n, seed, np.uint32, fill)


def exponential_u64(n: int, seed: int, scale: float = 2.0**40) -> np.ndarray:
    def fill(g, m):
        return _f64_to_u64_clamped(g.exponential(scale, size=m))
    return _chunked(n, seed, np.uint64, fill)


def zipf_dup_u64(n: int, seed: int, distinct: int = 1000, s: float = 1.1) -> np.ndarray:
    """Zipf(s) frequencies over ``distinct`` uniform uint64 values."""
    table = _rng(seed, SETUP).integers(0, 1 << 64, size=distinct, dtype=np.uint64, endpoint=False)
    cdf = zipf_cdf(distinct, s)

    def fill(g, m):
        rank = np.searchsorted(cdf, g.random(m), side="right")
        np.minimum(rank, distinct - 1, out=rank)
        return table[rank]
    return _chunked(n, seed, np.uint64, fill)


def index_payload(n: int) -> np.ndarray:
    """uint32 payload = original index (the provenance the paper keeps)."""
    return np.arange(n, dtype=np.uint32)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    # name: (dtype, default n, default P, generator, seed)
    "uniform_u32": ("u32", 1 << 20, 16, uniform_u32, 0),
    "normal_lognormal_u64": ("u64", 1 << 28, 128, normal_lognormal_u64, 1),
    "zipf_dup_f32": ("f32", 1 << 29, 256, zipf_dup_f32, 2),
    "exponential_u32": ("u32", 1 << 30, 1024, exponential_u32, 3),
}


def workload(name: str, n: int | None = None, seed: int | None = None):
    """Return (dtype, keys, P) for a named workload, optionally at another size/seed."""
    dtype, n0, P, gen, seed0 = WORKLOADS[name]
    return dtype, gen(n0 if n is None else n, seed0 if seed is None else seed), P


def batched_sizes(num: int = 10000, seed: int = 4, lo: int = 1024, hi: int = 1 << 24,
                  mu: float = 10.65, sigma: float = 1.8) -> np.ndarray:
    """Instance sizes of the batched workload: clip(rint(lognormal(mu, sigma)), lo, hi)."""
    g = _rng(seed, SETUP)
    x = np.rint(g.lognormal(mu, sigma, size=num))
    return np.clip(x, lo, hi).astype(np.int64)


def batched_partitions(sizes: np.ndarray, unit: int = 1 << 16, pmax: int = 256) -> np.ndarray:
    """Logical partitions per instance: clamp(2^floor(log2(n/unit)), 1, pmax)."""
    out = np.ones(len(sizes), dtype=np.int64)
    big = sizes >= unit
    out[big] = 1 << np.floor(np.log2(sizes[big] / unit)).astype(np.int64)
    return np.clip(out, 1, pmax)


def batched_instance_keys(i: int, n: int) -> np.ndarray:
    """uint64 keys of batched instance i; its distribution is picked by (1000 + i) mod 4."""
    seed = 1000 + i
    kind = seed % 4
    if kind == 0:
        return uniform_u64(n, seed)
    if kind == 1:
        return normal_lognormal_u64(n, seed)
    if kind == 2:
        return zipf_dup_u64(n, seed)
    return exponential_u64(n, seed)


def batched(num: int = 10000, seed: int = 4, **size_kw):
    """(offsets[num+1] uint64, keys uint64, P[num]) of the batched workload."""
    sizes = batched_sizes(num, seed, **size_kw)
    offsets = np.zeros(num + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes).astype(np.uint64)
    keys = np.empty(int(offsets[-1]), dtype=np.uint64)

    def work(i: int) -> None:
        keys[int(offsets[i]):int(offsets[i + 1])] = batched_instance_keys(i, int(sizes[i]))

    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(num)))
    return offsets, keys, batched_partitions(sizes)


# Small structured cases for edge tests.
def structured_u32(kind: str, n: int, seed: int = 7) -> np.ndarray:
    g = _rng(seed, 0)
    if kind == "sorted":
        return np.sort(g.integers(0, 1 << 32, size=n, dtype=np.uint64)).astype(np.uint32)
    if kind == "reverse":
        return np.sort(g.integers(0, 1 << 32, size=n, dtype=np.uint64))[::-1].astype(np.uint32)
    if kind == "equal":
        return np.full(n, 12345, dtype=np.uint32)
    if kind == "few":
        return g.integers(0, 3, size=n).astype(np.uint32)
    if kind == "extremes":
        return g.choice(np.array([0, 1, U32_MAX - 1, U32_MAX], dtype=np.uint32), size=n)
    raise ValueError(kind)
