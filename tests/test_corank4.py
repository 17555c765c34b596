"""The four-way round's tile boundaries (`k_corank4`), in the kernel's own
integer steps, checked by brute force.

A quad is four adjacent sorted lists; the key index holds the keys at global
multiples of the stride S (64 in the kernel).  The round merges the index
samples I_0 + I_1 -> X' and I_2 + I_3 -> Y', and boundary j sits just before
the sample at position j Q of merge(X', Y').  Its co-rank is that sample's
position in its own list and a bounded bisection (a window of at most S keys
fixed by the sample counts) in the other three.  Checked here against the
stable four-way merge (key, list, position) written out from its definition,
for small S so that every alignment, tie pattern and list end is reached:
each boundary's co-ranks are exactly the elements before its sample; the
boundaries rise; every tile holds S Q +- 3 (S - 1) outputs and the first and
last at most S Q + 4 (S - 1), so with S = 64 a tile never exceeds the outputs
a CTA holds: Q = 34 and 2432 (128 x 19) for 8-byte keys, Q = 64 and 4352
(256 x 17) for 4-byte keys."""
import math

import numpy as np
import pytest


def merge_path(a, b, d):
    lo, hi = max(0, d - len(b)), min(d, len(a))
    while lo < hi:
        mid = (lo + hi) // 2
        if a[mid] <= b[d - 1 - mid]:
            lo = mid + 1
        else:
            hi = mid
    return lo


def merge(a, b):
    out, i, j = [], 0, 0
    while i < len(a) or j < len(b):
        if j >= len(b) or (i < len(a) and a[i] <= b[j]):
            out.append(a[i])
            i += 1
        else:
            out.append(b[j])
            j += 1
    return out


def ceil_div(a, b):
    return (a + b - 1) // b


def tiles(src, s, n, S, Q):
    """Number of tiles of a quad: ceil(M / Q) for its M index samples, 1 for a
    non-empty quad without samples, 0 for an empty one."""
    E0, E4 = ceil_div(s[0], S), ceil_div(s[3] + n[3], S)
    M = E4 - E0
    return 0 if sum(n) == 0 else (1 if M == 0 else ceil_div(M, Q))


def corank(src, s, n, S, Q, j):
    """Co-ranks of boundary j (j >= 1), in the kernel's steps; also the number
    of bisection steps the widest window took."""
    E = [ceil_div(s[i], S) for i in range(4)] + [ceil_div(s[3] + n[3], S)]
    m = [E[i + 1] - E[i] for i in range(4)]
    o = [E[i] * S - s[i] for i in range(4)]
    I = [[src[(E[i] + k) * S] for k in range(m[i])] for i in range(4)]
    X, Y = merge(I[0], I[1]), merge(I[2], I[3])
    qpos = j * Q
    assert qpos < E[4] - E[0]
    x = merge_path(X, Y, qpos)
    y = qpos - x
    a = merge_path(I[0], I[1], x)
    cc = merge_path(I[2], I[3], y)
    kap = [a, x - a, cc, y - cc]
    from_x = x < len(X) and (y >= len(Y) or X[x] <= Y[y])
    if from_x:
        v = X[x]
        own = 0 if (a < m[0] and (x - a >= m[1] or I[0][a] <= I[1][x - a])) else 1
    else:
        v = Y[y]
        own = 2 if (cc < m[2] and (y - cc >= m[3] or I[2][cc] <= I[3][y - cc])) else 3
    assert v == I[own][kap[own]]
    c, steps = [], 0
    for i in range(4):
        if i == own:
            c.append(o[i] + S * kap[i])
            continue
        lo = o[i] + S * (kap[i] - 1) + 1 if kap[i] else 0
        hi = o[i] + S * kap[i] if kap[i] < m[i] else n[i]
        assert 0 <= lo <= hi <= n[i] and hi - lo <= S - 1
        k = 0
        while lo < hi:
            mid = (lo + hi) // 2
            kv = src[s[i] + mid]
            if (kv <= v) if i < own else (kv < v):
                lo = mid + 1
            else:
                hi = mid
            k += 1
        steps = max(steps, k)
        c.append(lo)
    return c, (v, own, o[own] + S * kap[own]), steps


def definition_prefix(src, s, n, elem):
    """Elements of each list before `elem` = (key, list, position) in the stable order."""
    v, own, p = elem
    out = []
    for i in range(4):
        lst = src[s[i]:s[i] + n[i]]
        out.append(sum(1 for k, x in enumerate(lst) if (x, i, k) < (v, own, p)))
    return out


def make_quad(g, S, max_len, vmax):
    n = [int(g.integers(0, max_len + 1)) for _ in range(4)]
    s0 = int(g.integers(0, 3 * S))
    s = [s0, s0 + n[0], s0 + n[0] + n[1], s0 + n[0] + n[1] + n[2]]
    src = [int(x) for x in g.integers(0, vmax, size=s[3] + n[3] + S)]
    for i in range(4):
        src[s[i]:s[i] + n[i]] = sorted(src[s[i]:s[i] + n[i]])
    return src, s, n


def check_quad(src, s, n, S, Q):
    T = tiles(src, s, n, S, Q)
    total = sum(n)
    bounds = [[0, 0, 0, 0]]
    for j in range(1, T):
        c, elem, steps = corank(src, s, n, S, Q, j)
        assert c == definition_prefix(src, s, n, elem), (s, n, j)
        assert steps <= math.ceil(math.log2(S)) if S > 1 else steps == 0
        bounds.append(c)
    bounds.append(list(n))
    sizes = []
    for b0, b1 in zip(bounds, bounds[1:]):
        assert all(x <= y for x, y in zip(b0, b1)), "boundaries must rise in every list"
        sizes.append(sum(b1) - sum(b0))
    if total == 0:
        return sizes
    assert sum(sizes) == total
    for k, sz in enumerate(sizes):
        assert sz <= S * Q + 4 * (S - 1), (k, sz)
        if 0 < k < len(sizes) - 1:
            assert S * Q - 3 * (S - 1) <= sz <= S * Q + 3 * (S - 1), (k, sz)
    return sizes


@pytest.mark.parametrize("S,Q", [(1, 1), (1, 3), (2, 1), (2, 3), (3, 2), (4, 1), (4, 5), (8, 2), (8, 7)])
def test_boundaries_are_exact_and_tiles_bounded(S, Q):
    g = np.random.default_rng(100 * S + Q)
    for _ in range(150):
        vmax = int(g.choice([1, 2, 3, 10, 1000]))
        src, s, n = make_quad(g, S, 5 * S + 6, vmax)
        check_quad(src, s, n, S, Q)


@pytest.mark.parametrize("Q,tile", [(30, 128 * 17), (34, 128 * 19), (64, 256 * 17)])
def test_kernel_stride_and_tile(Q, tile):
    """S = 64 and the kernel's Q for each key width (2176- and 4352-output
    tiles) on lists of thousands of keys, with heavy ties, one-sided lists and
    empty lists."""
    S = 64
    assert S * Q + 4 * (S - 1) <= tile
    g = np.random.default_rng(64)
    for vmax, lens in [(2, (3000, 2500, 0, 4100)), (7, (5000, 10, 3000, 3000)), (1 << 40, (4096, 4096, 4096, 4096)),
                       (1 << 40, (1, 0, 0, 9000)), (50, (2000, 2000, 2000, 2000))]:
        n = list(lens)
        s0 = int(g.integers(0, 200))
        s = [s0, s0 + n[0], s0 + n[0] + n[1], s0 + n[0] + n[1] + n[2]]
        src = [int(x) for x in g.integers(0, vmax, size=s[3] + n[3] + S)]
        for i in range(4):
            src[s[i]:s[i] + n[i]] = sorted(src[s[i]:s[i] + n[i]])
        sizes = check_quad(src, s, n, S, Q)
        assert max(sizes) <= tile
