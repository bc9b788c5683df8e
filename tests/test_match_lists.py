"""The precision-form matcher's per-thread top lists, restated on the host.

After the runs a thread holds NBIN bins of T ascending keys (distance bits with the candidate's index in
the low bits, ~0 for an empty slot).  The kernel takes the LH smallest of them in ascending order with a
bitonic merge tree: bins padded to TP = 2^ceil(log2 T) slots, runs merged pairwise (the second reversed
against the first, then both halves cleaned) up to length LS = 2^ceil(log2 LH), then the chunks of LS
folded into the first (element i against element LS - 1 - i of the next chunk keeps the LS smallest as
a bitonic sequence, which one more clean sorts).  These tests restate that network and check it against
a plain sort for every bin shape the library builds, including empty bins and bins whose keys all
beat the other bins'.
"""

import numpy as np
import pytest

EMPTY = 0xFFFFFFFF


def _cmpx(v, i, j):
    if v[j] < v[i]:
        v[i], v[j] = v[j], v[i]


def _clean(v, base, n):
    h = n // 2
    while h >= 1:
        for i in range(n):
            if (i & h) == 0:
                _cmpx(v, base + i, base + i + h)
        h //= 2


def _smallest_sorted(v, r, s):
    """The kernel's network on the list v (len a power of two, ascending runs of length r)."""
    n = len(v)
    ln = r
    while ln < s and ln < n:
        for base in range(0, n, 2 * ln):
            for i in range(ln):
                _cmpx(v, base + i, base + 2 * ln - 1 - i)
            h = ln // 2
            while h >= 1:
                for i in range(2 * ln):
                    if (i & h) == 0:
                        _cmpx(v, base + i, base + i + h)
                h //= 2
        ln *= 2
    for c in range(1, n // s):
        for i in range(s):
            v[i] = min(v[i], v[c * s + s - 1 - i])
        _clean(v, 0, s)
    return v


def _pow2(n):
    p = 1
    while p < n:
        p *= 2
    return p


def _shape(k):
    # the kernel's ListCfg: LH = max(2K, K + 8), 32 bins of 3 for K <= 16, else 16 bins of 6
    lh = max(2 * k, k + 8)
    return (32, 3, lh) if k <= 16 else (16, 6, lh)


@pytest.mark.parametrize("k", [2, 4, 8, 16, 32])
def test_top_list_network_is_the_sorted_prefix(k):
    nbin, t, lh = _shape(k)
    tp, ls = _pow2(t), _pow2(lh)
    assert (nbin * tp) % ls == 0 and ls >= tp
    rng = np.random.default_rng(40 + k)
    for trial in range(200):
        bins = []
        for g in range(nbin):
            n = int(rng.integers(0, t + 1))
            if trial % 7 == 0 and g < 2:  # two bins holding every one of the best keys
                keys = sorted(int(x) for x in rng.integers(0, 1000, n))
            else:
                keys = sorted(int(x) for x in rng.integers(1 << 20, 1 << 31, n))
            bins.append(keys + [EMPTY] * (t - n))
        v = []
        for b in bins:
            v += b + [EMPTY] * (tp - t)
        got = _smallest_sorted(v, tp, ls)[:lh]
        want = sorted(x for b in bins for x in b)[:lh]
        assert got == want, (k, trial)


def test_all_empty_bins_give_empty_list():
    nbin, t, lh = _shape(16)
    v = [EMPTY] * (nbin * _pow2(t))
    assert _smallest_sorted(v, _pow2(t), _pow2(lh))[:lh] == [EMPTY] * lh
