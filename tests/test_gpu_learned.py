"""Spatially varying noise: per-reference thresholds and the learned noise-level map.

* hts_denoise_sigma_map with one sigma per reference patch against the FP64
  oracle fed the same sigmas (same tolerances as the global-sigma parity);
* the network's denoising forward (tensor cores, FP16 activations) against
  the oracle's FP16-activation forward, and the training forward's loss,
  gradient and Adam step against the FP64 oracle of cnn_oracle.py, from the
  same (FP16-rounded) parameters;
* training on images whose noise level varies across the frame, with targets
  the method generates itself (best-PSNR threshold level, train.py), gives a
  map whose denoising beats one global estimated sigma;
* a map far from the estimate falls back to the estimate.
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


@pytest.mark.parametrize("H,W,C,seed", [(64, 72, 1, 41), (64, 56, 3, 42), (45, 61, 3, 43)])
def test_sigma_map_matches_oracle(oracle, hts, H, W, C, seed):
    p = hts.params(win=11)
    po = oracle.Params(win=11)
    clean, noisy = synth.make_config_image(H, W, C, 20.0, seed)
    n = hts.num_refs(H, W, p)
    smap = np.random.default_rng(seed).uniform(8.0, 40.0, size=n).astype(np.float32)
    got = hts.denoise_sigma_map(_dev(noisy), _dev(smap), p=p).cpu().numpy().astype(np.float64)
    want, _ = oracle.denoise(noisy, po, sigma=smap.astype(np.float64))
    assert np.max(np.abs(got - want)) <= 1e-3
    assert abs(synth.psnr(got, clean) - synth.psnr(want, clean)) <= 0.01
    # a constant map is the global-sigma call, bit for bit
    const = hts.denoise_sigma_map(_dev(noisy), _dev(np.full(n, 20.0, np.float32)), p=p).cpu().numpy()
    np.testing.assert_array_equal(const, hts.denoise(_dev(noisy), sigma=20.0, p=p).cpu().numpy())


def _layer_slices(co, C):
    out, o = [], 0
    for cout, cin in co.layer_shapes(C):
        out.append(slice(o, o + cout * cin * 9))
        out.append(slice(o + cout * cin * 9, o + cout * cin * 9 + cout))
        o += cout * cin * 9 + cout
    return out


@pytest.mark.parametrize("C,H,W", [(1, 24, 28), (3, 24, 28), (3, 45, 150)])
def test_network_matches_oracle(hts, C, H, W):
    # 45 x 150 spans three strips of 16 x 64 pixels each way, with ragged last ones
    from oracle import cnn_oracle as co

    p = hts.params()
    net = hts.Cnn(C, seed=5)
    rng = np.random.default_rng(100 + C)
    theta = (rng.standard_normal(co.num_params(C)) * 0.2).astype(np.float32)
    net.set_params(theta)
    np.testing.assert_array_equal(net.get_params(), theta)
    img = rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)
    th16 = co.fp16(theta)
    out, cache = co.forward(th16, img)
    # the denoising forward (tensor cores, FP16 activations): FP32 accumulation against FP64 can move
    # an activation across an FP16 rounding boundary (one unit, 2^-11 relative) now and then
    out16 = co.forward_act16(th16, img)
    got = net.log_sigma_map(_dev(img)).cpu().numpy()
    tol = 4e-3 * (1.0 + np.max(np.abs(out16)))
    assert np.max(np.abs(got - out16)) <= tol
    assert np.mean(np.abs(got - out16)) <= 0.1 * tol
    # sigma of every reference through the readout window, against the oracle's map and window
    cen = co.ref_centres(H, W)
    for S in (1, 8, 128):
        net.window = S
        np.testing.assert_allclose(net.sigma_refs(_dev(img), p).cpu().numpy(), co.window_sigma(out16, cen, S),
                                   rtol=2 * tol)
    # loss and gradient of the FP32 training kernels
    tgt = rng.uniform(1.0, 3.5, size=len(cen)).astype(np.float32)
    L, dout = co.loss_and_dout(out, cen, tgt)
    g = co.backward(th16, cache, dout)
    net.train_fp16 = False
    net.zero_grad()
    net.accumulate_grad(_dev(img), _dev(tgt), p)
    assert net.take_loss() == pytest.approx(L, rel=1e-4)
    gg = net.get_grad()
    for sl in _layer_slices(co, C):
        ref = g[sl]
        assert np.linalg.norm(gg[sl] - ref) <= 1e-3 * np.linalg.norm(ref) + 1e-9
    # Adam from the library's own gradient (first step: closed form of the oracle)
    net.adam_step(1e-2)
    want, _, _ = co.adam_step(theta.astype(np.float64), 0.0, 0.0, gg.astype(np.float64), 1, 1e-2)
    np.testing.assert_allclose(net.get_params(), want, rtol=1e-5, atol=1e-7)


def _he_params(co, C, rng):
    # He-scaled weights (the library's initialisation) and small biases: activations stay O(1)
    parts = []
    for cout, cin in co.layer_shapes(C):
        parts.append(rng.standard_normal(cout * cin * 9) * np.sqrt(2.0 / (9 * cin)))
        parts.append(rng.standard_normal(cout) * 0.05)
    return np.concatenate(parts).astype(np.float32)


@pytest.mark.parametrize("C,H,W", [(1, 24, 28), (3, 24, 28), (3, 45, 150)])
def test_fp16_training_step_matches_oracle(hts, C, H, W):
    # the tensor-core training step (the default): FP16 activations and input gradients, FP32 weight
    # gradients; against the oracle that rounds the same values (grad_act16), and near the exact FP64
    # gradient.  45 x 150 spans 6 x 3 strips of 8 x 64 pixels of the weight-gradient kernel, ragged ones last
    from oracle import cnn_oracle as co

    p = hts.params()
    rng = np.random.default_rng(200 + C)
    net = hts.Cnn(C, seed=5)
    assert net.train_fp16
    theta = _he_params(co, C, rng)
    net.set_params(theta)
    th16 = co.fp16(theta)
    cen = co.ref_centres(H, W)
    imgs = [rng.uniform(0, 255, size=(C, H, W)).astype(np.float32) for _ in range(2)]
    tgts = [rng.uniform(1.0, 3.5, size=len(cen)).astype(np.float32) for _ in range(2)]
    net.zero_grad()
    L16, g16, gex = 0.0, 0.0, 0.0
    for img, tgt in zip(imgs, tgts):  # two images: the gradients add up
        net.accumulate_grad(_dev(img), _dev(tgt), p)
        l16, gi = co.grad_act16(th16, img, cen, tgt)
        out, cache = co.forward(th16, img)
        L16 += l16
        g16 = g16 + gi
        gex = gex + co.backward(th16, cache, co.loss_and_dout(out, cen, tgt)[1])
    assert net.take_loss() == pytest.approx(L16, rel=1e-4)
    gg = net.get_grad()
    assert np.all(np.isfinite(gg))
    for sl in _layer_slices(co, C):
        # FP32 against FP64 accumulation can move a stored FP16 value by one unit (2^-11) now and then
        assert np.linalg.norm(gg[sl] - g16[sl]) <= 2e-3 * np.linalg.norm(g16[sl]) + 1e-9
        assert np.linalg.norm(gg[sl] - gex[sl]) <= 3e-2 * np.linalg.norm(gex[sl]) + 1e-9
    # the same step on the FP32 kernels agrees with the exact gradient; both settings train the same net
    net.train_fp16 = False
    net.zero_grad()
    for img, tgt in zip(imgs, tgts):
        net.accumulate_grad(_dev(img), _dev(tgt), p)
    net.take_loss()
    g32 = net.get_grad()
    for sl in _layer_slices(co, C):
        assert np.linalg.norm(g32[sl] - gex[sl]) <= 1e-3 * np.linalg.norm(gex[sl]) + 1e-9


def test_denoising_forward_full_size_samples(hts):
    # 3840 x 2160 x 3: a map pixel depends on the 11 x 11 input pixels around it (five 3x3 layers), so
    # the oracle's forward of a crop with 5 pixels of margin gives the map exactly inside the margin;
    # crops at the image corners check the zero padding of the real border
    from oracle import cnn_oracle as co

    H, W, C = 2160, 3840, 3
    net = hts.Cnn(C, seed=21)
    th16 = co.fp16(net.get_params().astype(np.float64))
    rng = np.random.default_rng(22)
    img = rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)
    got = net.log_sigma_map(_dev(img)).cpu().numpy()
    for y0, x0 in ((0, 0), (H - 24, W - 40), (1031, 1917), (0, W - 40), (H - 24, 0)):
        ylo, xlo = max(0, y0 - 5), max(0, x0 - 5)
        yhi, xhi = min(H, y0 + 24 + 5), min(W, x0 + 40 + 5)
        want = co.forward_act16(th16, img[:, ylo:yhi, xlo:xhi].astype(np.float64))
        sub = want[y0 - ylo:y0 - ylo + 24, x0 - xlo:x0 - xlo + 40]
        g = got[y0:y0 + 24, x0:x0 + 40]
        tol = 4e-3 * (1.0 + np.max(np.abs(sub)))
        assert np.max(np.abs(g - sub)) <= tol, (y0, x0)


def _images(n, size, seed):
    return [synth.make_varying_noise_image(size, size, 1, seed + 7 * i, sb_min=2.0) for i in range(n)]


def test_training_beats_one_global_sigma(hts):
    from paper_2512_23569_gb300 import train

    p = hts.params(win=15)
    data = [train.targets(n, c, s, p) for c, n, s in _images(48, 96, 1000)]
    net = hts.Cnn(1, seed=3)
    hist = train.fit(net, [d[0] for d in data], [d[1] for d in data], p, steps=1200, batch=8, lr0=2e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    net.window = 64
    gains, err_net, err_est = [], [], []
    for clean, noisy, spx in _images(6, 192, 9000):
        x = _dev(noisy)
        a = hts.denoise_learned(x, net, p, fallback_factor=3.0).cpu().numpy()
        assert hts.last_stats()["learned"] == 1
        b = hts.denoise(x, p=p).cpu().numpy()
        gains.append(synth.psnr(a, clean) - synth.psnr(b, clean))
        # the map's shape against the generator's per-patch levels: the network learns log(m* sigma) with the
        # best-PSNR multiplier m*, so both are compared up to a constant; one global level (any constant)
        # leaves at best the spread of the true levels about their mean
        truth = synth.ref_log_sigma(spx, 8, 4).astype(np.float64)
        lmap = np.log(net.sigma_refs(x, p).cpu().numpy().astype(np.float64))
        d = lmap - truth
        err_net.append(np.sqrt(np.mean((d - d.mean()) ** 2)))
        err_est.append(np.sqrt(np.mean((truth - truth.mean()) ** 2)))
    # measured: about +1 dB, and a map that follows the per-patch levels
    assert np.mean(gains) > 0.3, gains
    assert np.mean(err_net) < np.mean(err_est), (err_net, err_est)


def test_far_map_falls_back_to_the_estimate(hts):
    from oracle import cnn_oracle as co

    p = hts.params(win=11)
    net = hts.Cnn(1, seed=2)
    theta = net.get_params()
    theta[-1] = 9.0  # output bias: sigma ~ e^9, far from any estimate
    net.set_params(theta)
    clean, noisy = synth.make_config_image(64, 64, 1, 20.0, 77)
    x = _dev(noisy)
    got = hts.denoise_learned(x, net, p, fallback_factor=2.0).cpu().numpy()
    st = hts.last_stats()
    assert st["learned"] == 0 and st["learned_ratio"] > 2.0
    # the fallback is the estimated global threshold: the plain call, bit for bit
    np.testing.assert_array_equal(got, hts.denoise(x, p=p).cpu().numpy())
    assert co.num_params(1) == net.nparams


def test_network_save_load_roundtrip(hts, tmp_path):
    net = hts.Cnn(3, seed=11)
    net.window = 40
    path = str(tmp_path / "net.bin")
    net.save(path)
    back = hts.Cnn.load_file(path)
    assert back.C == 3 and back.window == 40
    np.testing.assert_array_equal(back.get_params(), net.get_params())


def test_learned_host_buffers_equal_device_call(hts):
    # hts_denoise_learned_host: copies in, the learned call, copies out -- the device call's result
    p = hts.params(win=15, precision=1)
    net = hts.Cnn(3, seed=4)
    net.window = 32
    clean, noisy, _ = synth.make_varying_noise_image(80, 96, 3, 321, sb_min=2.0)
    want = hts.denoise_learned(_dev(noisy), net, p, fallback_factor=50.0).cpu().numpy()
    got = hts.denoise_learned_host(noisy, net, p, fallback_factor=50.0)
    np.testing.assert_array_equal(want, got)
