"""Parity at the workloads' full sizes, in the launch configuration the benchmark times, pixel by pixel.

* Plain form on the colour 512x512x3 workload (AWGN sigma = 50 estimated, K = 16, 31x31 window): groups
  bit-exact, sigma to 1e-9, denoised pixels within 1e-3 of the FP64 oracle and 0.01 dB.
* Precision form (BF16 tensor-core grouping, FP16 tensor-core filter) on the colour 1024x1024x3 workload
  (correlated Poisson-Gaussian noise, sigma estimated): at this size the filter runs its 8x8-group tiles and
  the matcher its full (tile, plane pass) work queue.  Groups valid and >= 90 % equal to the FP64
  definition's; with the GPU's own groups, basis and threshold the oracle's filter (Eq. 19-21, FP64) and
  the tensor-core filter differ only by FP16 rounding and the threshold decisions it moves:
  max |diff| <= PREC_MAX_ABS, 99.9th percentile <= PREC_P999, mean <= PREC_MEAN; end to end (each side its
  own groups, basis and sigma) within 0.05 dB and the 99.9th percentile <= E2E_P999.
* Learned form's filter (network map as per-reference noise levels) in the precision form, against the
  oracle fed the same levels, groups and basis: the same per-pixel bounds.

The bounds on the tensor-core filter follow from its arithmetic: FP16 operands carry a relative rounding of
2^-11 (0.125 grey levels at 255; the zero-threshold reconstruction test bounds the round trip by 0.5),
and a coefficient within that rounding of the threshold may be kept on one side and dropped on the other;
one such flip moves each pixel of the 16 patches of its group by at most |s| |u_a v_b| |h_k| <= tau / 32
before the average over the estimates covering the pixel, a few grey levels at tau ~ 4 sigma.  Flips are
rare (a coefficient must fall within ~1e-3 tau of tau), so the 99.9th percentile stays small.
"""

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC_MAX_ABS = 12.0
PREC_P999 = 1.0
PREC_MEAN = 0.05
E2E_P999 = 4.0


@pytest.fixture(scope="module")
def hts():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2512_23569_gb300 import build, hts as h

    build.build()
    h.load()
    return h


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _errors(got, want):
    d = np.abs(got.astype(np.float64) - want)
    return float(d.max()), float(np.quantile(d, 0.999)), float(d.mean())


def _groups_valid(noisy, idx, green, K, win, want):
    """Vectorised validity of every group (reference first, K distinct members inside the window, the others
    ascending in distance up to FP32 rounding); returns the fraction equal (as sets) to the FP64 groups."""
    C, H, W = noisy.shape
    n = idx.shape[0]
    ys = np.arange(0, H - 8 + 1, 4)
    ys = np.unique(np.append(ys, H - 8))
    xs = np.unique(np.append(np.arange(0, W - 8 + 1, 4), W - 8))
    yr = np.repeat(ys, len(xs))
    xr = np.tile(xs, len(ys))
    assert np.array_equal(idx[:, 0], yr * W + xr)
    srt = np.sort(idx, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0)  # distinct
    y, x = np.divmod(idx, W)
    R = (win - 1) // 2
    assert np.all(np.abs(y - yr[:, None]) <= R) and np.all(np.abs(x - xr[:, None]) <= R)
    assert np.all((y >= 0) & (y <= H - 8) & (x >= 0) & (x <= W - 8))
    if C == 1:
        planes = [noisy[0].astype(np.float64)]
        sel = np.zeros(n, dtype=int)
    else:
        planes = [noisy.astype(np.float64).sum(0), noisy[1].astype(np.float64)]
        sel = green.astype(int)
    d = np.zeros((n, K))
    for pi, pl in enumerate(planes):
        rows = np.nonzero(sel == pi)[0]
        if rows.size == 0:
            continue
        for u in range(8):
            for v in range(8):
                a = pl[yr[rows] + u, xr[rows] + v]
                b = pl[y[rows] + u, x[rows] + v]
                d[rows] += (a[:, None] - b) ** 2
    assert np.all(np.diff(d[:, 1:], axis=1) >= -1e-4 * (1.0 + d[:, 2:]))
    same = np.mean([set(a_) == set(b_) for a_, b_ in zip(idx.tolist(), want.tolist())])
    return float(same)


def test_plain_colour512_full_size(oracle, hts):
    clean, noisy = synth.make_config_image(512, 512, 3, 50.0, 2000)
    po = oracle.Params(K=16, win=31)
    ph = hts.params(K=16, win=31)
    x = _dev(noisy)
    idx, green = hts.match(x, ph)
    want_idx, want_green, _ = oracle.match(noisy, po)
    np.testing.assert_array_equal(idx.cpu().numpy(), want_idx)
    np.testing.assert_array_equal(green.cpu().numpy(), want_green)
    out = hts.denoise(x, sigma=None, p=ph).cpu().numpy()
    st = hts.last_stats()
    want, info = oracle.denoise(noisy, po)
    assert abs(st["sigma"] / info["sigma"] - 1) < 1e-9
    mx, p999, mean = _errors(out, want)
    assert mx <= 1e-3, (mx, p999, mean)
    assert abs(synth.psnr(out, clean) - synth.psnr(want, clean)) <= 0.01


def test_precision_colour1024_full_size(oracle, hts):
    clean, noisy = synth.make_pg_correlated_image(1024, 1024, 3, 3000)
    po = oracle.Params(K=16, win=31)
    p1 = hts.params(K=16, win=31, precision=1)
    x = _dev(noisy)
    out = hts.denoise(x, sigma=None, p=p1).cpu().numpy()
    st = hts.last_stats()
    idx, green = hts.match(x, p1)
    idx, green = idx.cpu().numpy(), green.cpu().numpy()
    want_idx, want_green, _ = oracle.match(noisy, po)
    np.testing.assert_array_equal(green, want_green)
    same = _groups_valid(noisy, idx, green, 16, 31, want_idx)
    assert same >= 0.9, same
    # the filter alone: the GPU's groups, basis and threshold on both sides
    b, _ = hts.estimate_basis(x, p1).read()
    want_f, _ = oracle.denoise_groups(noisy, po, b, st["tau"], idx)
    mx, p999, mean = _errors(out, want_f)
    print("precision 1024 same-groups errors: max %.4g p99.9 %.4g mean %.4g" % (mx, p999, mean))
    assert mx <= PREC_MAX_ABS and p999 <= PREC_P999 and mean <= PREC_MEAN, (mx, p999, mean)
    # end to end against the oracle's own groups, basis and sigma
    want, info = oracle.denoise(noisy, po)
    mx, p999, mean = _errors(out, want)
    dp = synth.psnr(out, clean) - synth.psnr(want, clean)
    print("precision 1024 end-to-end: max %.4g p99.9 %.4g mean %.4g dPSNR %.3g dB, sigma %.6g vs %.6g"
          % (mx, p999, mean, dp, st["sigma"], info["sigma"]))
    assert abs(dp) <= 0.05 and p999 <= E2E_P999, (dp, mx, p999, mean)
    # the plain form on the same low-noise image (sigma-hat about 0.86: most coefficients lie near the
    # threshold, the certified FP32 difference evaluation and the FP64 passes decide them): the oracle's
    # groups bit for bit, its noise level, pixels within 1e-3
    p0 = hts.params(K=16, win=31)
    out0 = hts.denoise(x, sigma=None, p=p0).cpu().numpy()
    st0 = hts.last_stats()
    np.testing.assert_array_equal(hts.match(x, p0)[0].cpu().numpy(), want_idx)
    assert abs(st0["sigma"] / info["sigma"] - 1) < 1e-9, (st0["sigma"], info["sigma"])
    mx, p999, mean = _errors(out0, want)
    print("plain 1024 low noise: max %.4g p99.9 %.4g mean %.4g" % (mx, p999, mean))
    assert mx <= 1e-3, (mx, p999, mean)


def test_learned_map_precision_filter_per_pixel(oracle, hts):
    # a (random-weight) network's map as the per-reference noise levels, precision form, 384x320x3
    clean, noisy, _ = synth.make_varying_noise_image(384, 320, 3, 6600, gain=0.01, levels=(2.0, 28.0))
    p1 = hts.params(K=16, win=31, precision=1)
    po = oracle.Params(K=16, win=31)
    x = _dev(noisy)
    net = hts.Cnn(3, seed=9)
    net.window = 64
    sref = net.sigma_refs(x, p1)
    out = hts.denoise_sigma_map(x, sref, p=p1).cpu().numpy()
    idx, _ = hts.match(x, p1)
    b, _ = hts.estimate_basis(x, p1).read()
    s = sref.cpu().numpy().astype(np.float64)
    taus = np.array([oracle.tau(float(v), 3, po) for v in s])
    want, _ = oracle.denoise_groups(noisy, po, b, taus, idx.cpu().numpy())
    mx, p999, mean = _errors(out, want)
    print("learned map, precision filter: max %.4g p99.9 %.4g mean %.4g" % (mx, p999, mean))
    assert mx <= PREC_MAX_ABS and p999 <= PREC_P999 and mean <= PREC_MEAN, (mx, p999, mean)
