"""Batched form: many images of mixed sizes and channel counts in one graph launch.

The batch must give, image by image, exactly (bit for bit) what hts_denoise
gives -- the tuning (tile shape, number of concurrent streams) may change only
the speed -- and so the same parity with the FP64 oracle.  Graph reuse is
checked through the schedule counters and the library's launch counter.
"""

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# H, W, C, sigma (None = estimated), seed: gray and colour, known and estimated,
# ragged grids, one geometry twice
BATCH = [
    (40, 48, 1, 20.0, 501),
    (64, 56, 3, None, 502),
    (72, 61, 1, None, 503),
    (48, 48, 3, 30.0, 504),
    (40, 48, 1, 25.0, 505),
    (96, 80, 3, 15.0, 506),
    (33, 90, 3, None, 507),
]


@pytest.fixture(scope="module")
def hts():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2512_23569_gb300 import build, hts as h

    build.build()
    h.load()
    return h


def _images():
    out = []
    for H, W, C, s, seed in BATCH:
        clean, noisy = synth.make_config_image(H, W, C, 20.0 if s is None else s, seed)
        out.append((clean, noisy, s))
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_batch_equals_single_calls(hts):
    p = hts.params(win=15)
    imgs = _images()
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    single = [hts.denoise(x, sigma=s, p=p).cpu().numpy() for x, s in zip(xs, sig)]
    outs = hts.denoise_batch(xs, sig, p)
    for a, b in zip(single, outs):
        np.testing.assert_array_equal(a, b.cpu().numpy())
    per, info = hts.last_batch_stats(len(imgs))
    assert info["images"] == len(imgs)
    assert info["lanes"] in (1, 2, 4, 8)
    assert info["kernels"] > 0
    for (H, W, C, s, _), st in zip(BATCH, per):
        assert st["nref"] == hts.num_refs(H, W, p)
        if s is not None:
            assert st["sigma"] == pytest.approx(s, rel=0, abs=1e-6)
    # every geometry of the batch was tuned to a valid shape
    for H, W, C, _, _ in BATCH:
        t = hts.tuned_tile(H, W, C, p)
        assert t is not None and t[0] >= 0 and t[1] >= 0


def test_batch_matches_oracle(oracle, hts):
    p = hts.params(win=15)
    po = oracle.Params(win=15)
    imgs = _images()
    outs = hts.denoise_batch([_dev(n) for _, n, _ in imgs], [s for _, _, s in imgs], p)
    for (clean, noisy, s), o in zip(imgs, outs):
        want, _ = oracle.denoise(noisy, po, sigma=s)
        got = o.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - want)) <= 1e-3
        assert abs(synth.psnr(got, clean) - synth.psnr(want, clean)) <= 0.01


def test_graph_reuse_and_rebinding(hts):
    p = hts.params(win=11, K=8)
    imgs = _images()[:4]
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    outs = [torch.empty_like(x) for x in xs]
    hts.denoise_batch(xs, sig, p, outs=outs)
    first = [o.cpu().numpy() for o in outs]
    _, info0 = hts.last_batch_stats(len(xs))
    # same signature and pointers: the graph is launched as it is
    n0 = hts.launch_count()
    hts.denoise_batch(xs, sig, p, outs=outs)
    torch.cuda.synchronize()
    _, info1 = hts.last_batch_stats(len(xs))
    assert info1["captures"] == info0["captures"]
    assert hts.launch_count() - n0 == info1["kernels"]
    for a, o in zip(first, outs):
        np.testing.assert_array_equal(a, o.cpu().numpy())
    # new output buffers and a changed known sigma: re-captured and updated in place
    outs2 = [torch.zeros_like(x) for x in xs]
    sig2 = list(sig)
    sig2[0] = sig[0] + 5.0
    hts.denoise_batch(xs, sig2, p, outs=outs2)
    _, info2 = hts.last_batch_stats(len(xs))
    assert info2["captures"] == info1["captures"] + 1
    want0 = hts.denoise(xs[0], sigma=sig2[0], p=p).cpu().numpy()
    np.testing.assert_array_equal(want0, outs2[0].cpu().numpy())
    for a, o in zip(first[1:], outs2[1:]):
        np.testing.assert_array_equal(a, o.cpu().numpy())


def test_batch_rejects_bad_input_before_work(hts):
    p = hts.params()
    x = _dev(synth.make_config_image(32, 32, 1, 10.0, 9)[1])
    n0 = hts.launch_count()
    with pytest.raises(hts.HtsError):
        hts.denoise_batch([x, x[:, :4, :4].contiguous()], [10.0, 10.0], p)  # 4x4 is smaller than a patch
    assert hts.launch_count() == n0
    assert hts.denoise_batch([], [], p) == []


def test_per_image_parameters(hts):
    # gray images with a 11x11 window and K=8, colour with 15x15 and K=16, in one graph
    pg, pc = hts.params(win=11, K=8), hts.params(win=15)
    imgs = _images()
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    per = [pg if C == 1 else pc for (_, _, C, _, _) in BATCH]
    outs = hts.denoise_batch(xs, sig, hts.params(), per_image=per)
    for x, s, pi, o in zip(xs, sig, per, outs):
        np.testing.assert_array_equal(hts.denoise(x, sigma=s, p=pi).cpu().numpy(), o.cpu().numpy())


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_tensor_core_forms_equal_single_calls(hts, precision):
    # the tensor-core forms in the graph (precision 1: BF16 tensor-core grouping with its exhaustive rescue;
    # precision 2: exact groups) equal the per-image calls bit for bit
    pg, pc = hts.params(win=11, K=8, precision=precision), hts.params(win=15, precision=precision)
    imgs = _images()
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    per = [pg if C == 1 else pc for (_, _, C, _, _) in BATCH]
    outs = hts.denoise_batch(xs, sig, hts.params(), per_image=per)
    for x, s, pi, o in zip(xs, sig, per, outs):
        np.testing.assert_array_equal(hts.denoise(x, sigma=s, p=pi).cpu().numpy(), o.cpu().numpy())
