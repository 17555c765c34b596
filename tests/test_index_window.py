"""The partition kernel's two searches, in its own integer steps, checked by
brute force: the window bound of the indexed merge-path search
(`merge_path_indexed`) and the pair search that starts from a guess
(`last_le_from`).

Lists A = src[pa, pa + na) and B = src[pb, pb + nb) are sorted; the index
holds the keys at global multiples of the stride S (64 in the kernel).  The
search bisects the merge of the two index samples at diagonal ceil((d - o)/S)
(o = the two lists' offsets to their first indexed position), takes one more
comparison for the next diagonal, and then bisects the keys only inside the
window the two bound.  Here the same integer arithmetic runs for small S (so
that ties, list ends and offsets hit every alignment) against the split of the
stable merge computed from its definition."""
import numpy as np
import pytest


def split_by_definition(a, b, d):
    """Number of A items among the first d outputs of the stable merge (ties: A first)."""
    tagged = sorted([(x, 0, i) for i, x in enumerate(a)] + [(x, 1, j) for j, x in enumerate(b)])
    return sum(1 for t in tagged[:d] if t[1] == 0)


def sample_merge_path(ia, ib, D):
    lo, hi = max(0, D - len(ib)), min(D, len(ia))
    while lo < hi:
        mid = (lo + hi) // 2
        if ia[mid] <= ib[D - 1 - mid]:
            lo = mid + 1
        else:
            hi = mid
    return lo


def ceil_div_signed(t, S):
    return (t + S - 1) // S if t >= 0 else -((-t) // S)


def window(src, pa, na, pb, nb, d, S):
    """[lo, hi] of the kernel's fine search, in the kernel's arithmetic."""
    lo, hi = max(0, d - nb), min(d, na)
    ea, eb = (pa + S - 1) // S, (pb + S - 1) // S
    ca = (pa + na + S - 1) // S - ea
    cb = (pb + nb + S - 1) // S - eb
    oa, ob = ea * S - pa, eb * S - pb
    t = d - (oa + ob)
    cmax = ca + cb
    dl = min(max(ceil_div_signed(t, S), 0), cmax)
    dh = min(max(ceil_div_signed(t + S - 1, S), 0), cmax)
    ia = [src[(ea + i) * S] for i in range(ca)]
    ib = [src[(eb + j) * S] for j in range(cb)]
    alo = sample_merge_path(ia, ib, dl)
    ahi = alo
    if dh > dl and alo < ca and (dl - alo >= cb or ia[alo] <= ib[dl - alo]):
        ahi = alo + 1
    if alo >= 1:
        lo = max(lo, oa + S * (alo - 1) + 1)
    if ahi < ca:
        hi = min(hi, oa + S * ahi)
    return lo, hi


@pytest.mark.parametrize("S", [1, 2, 3, 4, 8])
def test_window_holds_the_split(S):
    g = np.random.default_rng(1000 + S)
    for _ in range(300):
        na, nb = int(g.integers(0, 40)), int(g.integers(0, 40))
        gap = int(g.integers(0, 2 * S + 1))
        pa = int(g.integers(0, 3 * S + 1))
        pb = pa + na + gap
        n = pb + nb + int(g.integers(0, S + 1))
        vmax = int(g.choice([1, 3, 10, 1000]))
        src = [int(x) for x in g.integers(0, vmax, size=n)]
        src[pa:pa + na] = sorted(src[pa:pa + na])
        src[pb:pb + nb] = sorted(src[pb:pb + nb])
        a, b = src[pa:pa + na], src[pb:pb + nb]
        for d in range(na + nb + 1):
            want = split_by_definition(a, b, d)
            lo, hi = window(src, pa, na, pb, nb, d, S)
            assert lo <= want <= hi, (S, pa, na, pb, nb, d, lo, hi, want)
            assert hi - lo <= 2 * S - 1


def test_window_is_narrow_at_the_kernel_stride():
    """S = 64 on lists of thousands of keys with heavy ties: the window never
    exceeds 127 positions and always holds the split."""
    S = 64
    g = np.random.default_rng(7)
    for vmax in (2, 50, 1 << 30):
        na, nb = 3000 + int(g.integers(0, 500)), 2000 + int(g.integers(0, 500))
        pa = int(g.integers(0, 200))
        pb = pa + na
        src = [int(x) for x in g.integers(0, vmax, size=pb + nb)]
        src[pa:pa + na] = sorted(src[pa:pa + na])
        src[pb:pb + nb] = sorted(src[pb:pb + nb])
        a, b = np.array(src[pa:pa + na]), np.array(src[pb:pb + nb])
        for d in list(range(0, na + nb + 1, 97)) + [na + nb]:
            # the stable-merge split from its definition: the A item at index i goes to
            # i + #(B < a_i), so the split is the number of A items placed before d
            posA = np.arange(na) + np.searchsorted(b, a, side="left")
            want = int(np.sum(posA < d))
            lo, hi = window(src, pa, na, pb, nb, d, S)
            assert lo <= want <= hi and hi - lo <= 2 * S - 1


def last_le_from(t, n, i, g):
    """The partition kernel's pair search (gallop from a guess, then bisect),
    in the kernel's steps."""
    if t[g] <= i:
        lo, step = g, 1
        while True:
            nx = lo + step
            if nx >= n:
                hi = n
                break
            if t[nx] > i:
                hi = nx
                break
            lo, step = nx, step * 2
    else:
        hi, step = g, 1
        while True:
            if hi <= step:
                lo = 0
                break
            nx = hi - step
            if t[nx] <= i:
                lo = nx
                break
            hi, step = nx, step * 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if t[mid] <= i:
            lo = mid
        else:
            hi = mid
    return lo


def test_pair_search_from_any_guess():
    """For tile i the search returns the last pair p with tbegin[p] <= i (empty
    pairs repeat a tbegin value) from any starting guess."""
    g = np.random.default_rng(11)
    for _ in range(200):
        n = int(g.integers(1, 60))
        counts = g.integers(0, 4, size=n) * (g.random(n) < 0.7)
        t = np.concatenate([[0], np.cumsum(counts)]).astype(int)
        total = int(t[-1])
        for i in range(total):
            want = max(p for p in range(n) if t[p] <= i)
            for guess in {0, n - 1, (i * n) // total, int(g.integers(0, n))}:
                assert last_le_from(t, n, i, guess) == want
