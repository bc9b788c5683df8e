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


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_sigma_maps_equal_single_calls(oracle, hts, precision):
    # a caller's noise level per reference patch (hts_image.sigma_map) in the graph: per image equal to
    # hts_denoise_sigma_map bit for bit, mixed with images that have none; against the oracle fed the
    # same levels (plain form: <= 1e-3 max-abs)
    pg, pc = hts.params(win=11, K=8, precision=precision), hts.params(win=15, precision=precision)
    imgs = _images()
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    per = [pg if C == 1 else pc for (_, _, C, _, _) in BATCH]
    rng = np.random.default_rng(77)
    maps = []
    for i, ((H, W, C, _, _), pi) in enumerate(zip(BATCH, per)):
        if i % 3 == 1:
            maps.append(None)
            continue
        n = hts.num_refs(H, W, pi)
        maps.append(_dev(rng.uniform(8.0, 40.0, size=n)))
    outs = hts.denoise_batch(xs, sig, hts.params(), per_image=per, sigma_maps=maps)
    for x, s, pi, m, o in zip(xs, sig, per, maps, outs):
        want = (hts.denoise(x, sigma=s, p=pi) if m is None else hts.denoise_sigma_map(x, m, p=pi)).cpu().numpy()
        np.testing.assert_array_equal(want, o.cpu().numpy())
    if precision == 0:
        for (clean, noisy, s), (H, W, C, _, _), m, o in zip(imgs, BATCH, maps, outs):
            if m is None:
                continue
            po = oracle.Params(win=11, K=8) if C == 1 else oracle.Params(win=15)
            basis = hts.estimate_basis(_dev(noisy), hts.params(win=11, K=8) if C == 1 else hts.params(win=15))
            b, _ = basis.read()
            want, _ = oracle.denoise(noisy, po, sigma=m.cpu().numpy().astype(np.float64), basis=b)
            got = o.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - want)) <= 1e-3


def test_batch_learned_equals_single_calls(hts):
    # the network's maps inside the graph launch (its forwards on a stream of their own): per image equal
    # to hts_denoise_learned bit for bit, the fallback decisions included; training between calls is seen
    imgs = [(c, n, s) for (c, n, s), (_, _, C, _, _) in zip(_images(), BATCH) if C == 3]
    xs = [_dev(n) for _, n, _ in imgs]
    net = hts.Cnn(3, seed=5)
    net.window = 16
    for prec in (1, 2):
        p = hts.params(win=15, precision=prec)
        for factor in (2.0, 50.0):  # 2: the untrained map may be judged off and fall back; 50: used
            outs = hts.denoise_batch_learned(xs, net, p, fallback_factor=factor)
            per, _ = hts.last_batch_stats(len(xs))
            for x, o, st in zip(xs, outs, per):
                want = hts.denoise_learned(x, net, p, fallback_factor=factor).cpu().numpy()
                single = hts.last_stats()
                np.testing.assert_array_equal(want, o.cpu().numpy())
                assert st["learned"] == single["learned"]
                assert st["learned_ratio"] == pytest.approx(single["learned_ratio"], rel=1e-12)
            if factor == 50.0:
                assert all(st["learned"] == 1 for st in per)
    # new weights: the same plan reads them at its next launch
    theta = net.get_params()
    theta[-1] += 0.5  # the output bias: log sigma + 0.5 everywhere
    net.set_params(theta)
    p = hts.params(win=15, precision=1)
    outs = hts.denoise_batch_learned(xs, net, p, fallback_factor=50.0)
    for x, o in zip(xs, outs):
        np.testing.assert_array_equal(hts.denoise_learned(x, net, p, fallback_factor=50.0).cpu().numpy(),
                                      o.cpu().numpy())
    with pytest.raises(hts.HtsError):  # a gray image with a colour network
        hts.denoise_batch_learned([_dev(_images()[0][1])], net, p)


def test_phased_batch_uses_single_launches_over_all_images(oracle, hts):
    # every image in a tensor-core form: the matcher and the filter run once per group of images over a work
    # queue of (image, tile) items; mixed sizes, gray and colour, K 8 and 16, precision 1 and 2 together
    imgs = _images()
    xs = [_dev(n) for _, n, _ in imgs]
    sig = [s for _, _, s in imgs]
    per = []
    for i, (_, _, C, _, _) in enumerate(BATCH):
        per.append(hts.params(win=11, K=8, precision=1 + (i % 2)) if C == 1 else hts.params(win=15, precision=1))
    outs = hts.denoise_batch(xs, sig, hts.params(), per_image=per)
    per_stats, info = hts.last_batch_stats(len(xs))
    assert info["phased"] == 1
    for x, s, pi, o in zip(xs, sig, per, outs):
        np.testing.assert_array_equal(hts.denoise(x, sigma=s, p=pi).cpu().numpy(), o.cpu().numpy())
    # the graph holds far fewer heavy launches than one pipeline per image would
    n0 = hts.launch_count()
    hts.denoise_batch(xs, sig, hts.params(), per_image=per)
    torch.cuda.synchronize()
    assert hts.launch_count() - n0 == info["kernels"]
    # a plain-form image in the batch: one pipeline per image
    per2 = list(per)
    per2[0] = hts.params(win=11, K=8)
    hts.denoise_batch(xs, sig, hts.params(), per_image=per2)
    assert hts.last_batch_stats(len(xs))[1]["phased"] == 0
