"""The precision-form matcher's per-thread bins and their row pitch, restated on the host.

The tensor-core matcher numbers the candidates of a tile's region p = y * Wq + x and keeps, per
reference, the T = 3 smallest keys of each cell (p - band start) mod 64 (bin and half-run).  A
reference whose cells pushed out a key below its (K+3)-th smallest kept one is matched again
exhaustively.  Equally good candidates lie along lattice directions (edges, stripes); the pitch Wq in
[Wc, Wc + 7] is chosen so that the short directions spread over many cells (`bench._match_pitch`
restates the kernel's rule).  These tests pin the rule's choices and show, with exact FP64 distances on
a seeded image, that the padded pitch lists far fewer references than the region width itself.
"""

import numpy as np

import bench
from paper_2512_23569_gb300 import synth

PS, STEP = 8, 4


def _cells(w, dy, dx):
    d = (dy * w + dx) & 63
    return 64 >> ((d & -d).bit_length() - 1) if d else 1


def test_pitch_rule():
    assert bench._match_pitch(49) == 51  # 49 maps the anti-diagonal (48 = -16 mod 64) onto 4 cells
    assert bench._match_pitch(59) == 59
    for wc in range(2, 120):
        wq = bench._match_pitch(wc)
        assert wc <= wq <= wc + 7
        dirs = [(dy, dx) for dy in range(5) for dx in range(-4, 5) if not (dy == 0 and dx <= 0)]
        score = min(_cells(wq, dy, dx) ** 2 * (dy * dy + dx * dx) for dy, dx in dirs)
        assert score >= min(_cells(wc, dy, dx) ** 2 * (dy * dy + dx * dx) for dy, dx in dirs)


def _grid(n):
    g = list(range(0, n - PS + 1, STEP))
    if g[-1] != n - PS:
        g.append(n - PS)
    return g


def _listed(pl, R, K, T, pad):
    """References the bins would list for the exhaustive matcher (exact FP64 distances)."""
    H, W = pl.shape
    KC = K + 3
    ys, xs = _grid(H), _grid(W)
    P = np.lib.stride_tricks.sliding_window_view(pl, (PS, PS)).reshape(H - PS + 1, W - PS + 1, PS * PS)
    listed = total = 0
    for gy0 in range(0, len(ys), 16):
        for gx0 in range(0, len(xs), 8):
            gy1, gx1 = min(len(ys), gy0 + 16) - 1, min(len(xs), gx0 + 8) - 1
            cy0, cx0 = max(0, ys[gy0] - R), max(0, xs[gx0] - R)
            wc = min(W - PS, xs[gx1] + R) - cx0 + 1
            wq = bench._match_pitch(wc) if pad else wc
            for q in range(4):
                refs = [(gy0 + 4 * q + j // 8, gx0 + j % 8) for j in range(32)
                        if gy0 + 4 * q + j // 8 <= gy1 and gx0 + j % 8 <= gx1]
                if not refs:
                    continue
                start = ((max(0, ys[refs[0][0]] - R) - cy0) * wq) & ~31
                for ry, rx in refs:
                    yr, xr = ys[ry], xs[rx]
                    yy, xx = np.mgrid[max(0, yr - R):min(H - PS, yr + R) + 1, max(0, xr - R):min(W - PS, xr + R) + 1]
                    keep = ~((yy == yr) & (xx == xr))
                    yy, xx = yy[keep], xx[keep]
                    d = ((P[yy, xx] - P[yr, xr]) ** 2).sum(1)
                    p = (yy - cy0) * wq + (xx - cx0)
                    rank = np.empty(len(p), int)
                    rank[np.lexsort((p, d))] = np.arange(len(p))
                    cell = (p - start) % 64
                    kept = np.zeros(len(p), bool)
                    for c in np.unique(cell):
                        members = np.nonzero(cell == c)[0]
                        kept[members[np.argsort(rank[members])[:T]]] = True
                    kr = np.sort(rank[kept])
                    pushed = rank[~kept].min() if (~kept).any() else len(p)
                    listed += int(pushed < (kr[KC - 1] if len(kr) >= KC else len(p)))
                    total += 1
    return listed, total


def test_padded_pitch_lists_few_references():
    _, noisy = synth.make_pg_correlated_image(192, 192, 1, 3000)
    pl = noisy[0].astype(np.float64)
    raw, n = _listed(pl, 10, 16, 3, pad=False)
    padded, _ = _listed(pl, 10, 16, 3, pad=True)
    assert padded <= 0.005 * n
    assert raw >= 5 * max(padded, 1)
