"""Precision form: grouping by BF16 tensor-core distances with an FP32 re-rank of the nearest
(references whose nearest may have been dropped by the per-thread bins are matched exhaustively in
FP32), filtering with FP16 tensor-core projections and FP32 threshold decisions.

Its groups are not bit-exact by design: BF16 rounding may reorder near
neighbours.  What is checked: every group is valid (the reference first, K
distinct members inside its search window, the K-1 others in ascending FP32
distance), nearly all groups equal the FP64 definition's, the denoised
image is within 0.05 dB PSNR of the FP64 oracle, on AWGN and on
spatially correlated Poisson-Gaussian noise, and the tensor-core filter
gives the image back at a zero threshold and zero at a huge one.
"""

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hts():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2512_23569_gb300 import build, hts as h

    build.build()
    h.load()
    return h


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _plane(noisy, green):
    if noisy.shape[0] == 1:
        return noisy[0].astype(np.float64)
    return noisy[1].astype(np.float64) if green else (noisy[0].astype(np.float64) + noisy[1] + noisy[2])


CASES = [
    # H, W, C, win, K, sigma, seed
    (128, 128, 1, 21, 16, 25.0, 1000),
    (77, 93, 1, 21, 16, 25.0, 11),
    (96, 112, 3, 31, 16, 50.0, 2000),
    (45, 61, 3, 15, 8, 30.0, 12),
    (48, 56, 3, 11, 32, 20.0, 14),
    (40, 40, 1, 7, 4, 10.0, 13),
]


@pytest.mark.parametrize("H,W,C,win,K,sigma,seed", CASES)
def test_groups_valid_and_close_to_exact(oracle, hts, H, W, C, win, K, sigma, seed):
    _, noisy = synth.make_config_image(H, W, C, sigma, seed)
    _check_groups(oracle, hts, noisy, K, win)


def test_rescue_of_crowded_bins(oracle, hts):
    # stripes of constant x + 3y (period 16) put the equally good candidates of a reference on the lattice
    # direction (1, -3), which the row pitch 51 of a 49-column region maps onto 4 of the 64 bins: those
    # references are matched again exhaustively (FP32), and every group must still be valid and nearly all
    # equal the FP64 definition's
    H = W = 96
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    clean = 128.0 + 60.0 * np.sin(2.0 * np.pi * (xx + 3.0 * yy) / 16.0)
    noisy = (clean + np.random.default_rng(17).normal(0.0, 5.0, clean.shape))[None].astype(np.float32)
    _check_groups(oracle, hts, noisy, 16, 21)
    assert hts.last_stats()["match_fallback"] >= 50


def test_rescue_of_crowded_bins_colour(oracle, hts):
    # colour: stripes of constant 3x + y (period 16) lie along (3, -1), which the 59-column regions of a
    # 31x31 window map onto 4 bins; the channel gains differ between the halves of the image so that
    # both Eq. 9 planes occur -- the rescued references must be matched on their own plane
    H = W = 128
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    base = 120.0 + 60.0 * np.sin(2.0 * np.pi * (3.0 * xx + yy) / 16.0)
    left = xx < W / 2
    gains = [np.where(left, 1.3, 0.7), np.ones_like(xx), np.where(left, 0.8, 0.6)]  # R, G, B
    rng = np.random.default_rng(23)
    noisy = np.stack([base * g_ + rng.normal(0.0, 5.0, base.shape) for g_ in gains]).astype(np.float32)
    _check_groups(oracle, hts, noisy, 16, 31)
    assert hts.last_stats()["match_fallback"] >= 50
    green = hts.match(_dev(noisy), hts.params(K=16, win=31, precision=1))[1].cpu().numpy()
    assert 0 < int(green.sum()) < green.size  # both planes


def _check_groups(oracle, hts, noisy, K, win):
    C, H, W = noisy.shape
    p1 = hts.params(K=K, win=win, precision=1)
    idx, green = hts.match(_dev(noisy), p1)
    idx, green = idx.cpu().numpy(), green.cpu().numpy()
    want, green_o, _ = oracle.match(noisy, oracle.Params(K=K, win=win))
    if C == 3:
        np.testing.assert_array_equal(green, green_o)
    R = (win - 1) // 2
    ys = oracle.grid(H, 8, 4)
    xs = oracle.grid(W, 8, 4)
    same = 0
    for r in range(idx.shape[0]):
        yr, xr = ys[r // len(xs)], xs[r % len(xs)]
        g = idx[r]
        assert g[0] == yr * W + xr
        assert len(set(g.tolist())) == K
        pl = _plane(noisy, green[r] if C == 3 else 1)
        a = pl[yr:yr + 8, xr:xr + 8]
        d = []
        for q in g[1:]:
            y, x = divmod(int(q), W)
            assert abs(y - yr) <= R and abs(x - xr) <= R and 0 <= y <= H - 8 and 0 <= x <= W - 8
            d.append(np.sum((a - pl[y:y + 8, x:x + 8]) ** 2))
        d = np.array(d)
        assert np.all(np.diff(d) >= -1e-4 * (1.0 + d[1:]))  # ascending up to FP32 rounding
        same += int(set(g.tolist()) == set(want[r].tolist()))
    assert same >= 0.9 * idx.shape[0]


@pytest.mark.parametrize("H,W,C,win,K,sigma,seed", CASES[:4])
def test_denoise_within_005_db_of_oracle(oracle, hts, H, W, C, win, K, sigma, seed):
    clean, noisy = synth.make_config_image(H, W, C, sigma, seed)
    out = hts.denoise(_dev(noisy), sigma=sigma, p=hts.params(K=K, win=win, precision=1)).cpu().numpy()
    want, _ = oracle.denoise(noisy, oracle.Params(K=K, win=win), sigma=sigma)
    assert abs(synth.psnr(out, clean) - synth.psnr(want, clean)) <= 0.05


def test_correlated_poisson_gaussian_256(oracle, hts):
    # the precision-form workload's noise on a 256x256 colour image, sigma estimated on both sides
    clean, noisy = synth.make_pg_correlated_image(256, 256, 3, 3000)
    out = hts.denoise(_dev(noisy), sigma=None, p=hts.params(win=31, precision=1)).cpu().numpy()
    want, info = oracle.denoise(noisy, oracle.Params(win=31))
    assert abs(synth.psnr(out, clean) - synth.psnr(want, clean)) <= 0.05


def test_precision_validation(hts):
    x = _dev(synth.make_config_image(256, 256, 1, 10.0, 5)[1])
    with pytest.raises(hts.HtsError):
        hts.denoise(x, sigma=10.0, p=hts.params(precision=3))
    with pytest.raises(hts.HtsError):  # 63x63 window: the staged search region does not fit on chip
        hts.denoise(x, sigma=10.0, p=hts.params(win=63, precision=1))


@pytest.mark.parametrize("C,K,win", [(1, 16, 21), (3, 16, 31), (3, 8, 15), (1, 32, 11), (3, 32, 11)])
def test_tensor_core_filter_reconstructs_and_thresholds(hts, C, K, win):
    # sigma = 0 keeps every coefficient: the FP16 forward and inverse projections must give the noisy
    # image back up to their rounding (FP16 input: half a unit in the last place, 0.125 at 256, plus the
    # FP16 coefficients); a huge sigma drops every coefficient: the output is exactly zero
    clean, noisy = synth.make_config_image(70, 83, C, 20.0, 31 + C + K)
    x = _dev(noisy)
    p = hts.params(K=K, win=win, precision=1)
    out = hts.denoise(x, sigma=0.0, p=p).cpu().numpy()
    err = np.abs(out.astype(np.float64) - noisy.astype(np.float64))
    assert np.max(err) <= 0.5
    assert np.mean(err) <= 0.05
    assert hts.last_stats()["tau"] == 0.0
    zero = hts.denoise(x, sigma=1e6, p=p).cpu().numpy()
    assert np.all(zero == 0.0)


@pytest.mark.parametrize("H,W,C,win,K,sigma,seed", CASES[:3])
def test_exact_groups_with_tensor_core_filter(oracle, hts, H, W, C, win, K, sigma, seed):
    # precision 2: the grouping of the plain form (bit-exact groups) and the filter of the precision form
    clean, noisy = synth.make_config_image(H, W, C, sigma, seed)
    x = _dev(noisy)
    p2 = hts.params(K=K, win=win, precision=2)
    idx2, green2 = hts.match(x, p2)
    idx0, green0 = hts.match(x, hts.params(K=K, win=win))
    assert torch.equal(idx2, idx0) and torch.equal(green2, green0)
    out = hts.denoise(x, sigma=sigma, p=p2).cpu().numpy()
    want, _ = oracle.denoise(noisy, oracle.Params(K=K, win=win), sigma=sigma)
    assert abs(synth.psnr(out, clean) - synth.psnr(want, clean)) <= 0.05
    # same groups: the filters differ only by FP16 rounding and the threshold decisions it moves
    assert np.mean(np.abs(out.astype(np.float64) - want)) <= 0.05
