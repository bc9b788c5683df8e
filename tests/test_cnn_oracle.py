"""Pins of the learned noise-level map's FP64 oracle (oracle/cnn_oracle.py).

The convolution is pinned to scipy's 2-D correlation, the backward pass to
central finite differences of the forward pass (every layer, weights and
biases), the loss gradient to finite differences, and the first Adam step to
its closed form lr * g / (|g| + eps).
"""

import numpy as np
import pytest

from oracle import cnn_oracle as co

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_is_2d_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 9, 11))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = co.conv3x3(x, w, b)
    for o in range(4):
        want = b[o] + sum(scipy_signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(got[o], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("C", [1, 3])
def test_backward_matches_finite_differences(C):
    rng = np.random.default_rng(10 + C)
    theta = rng.standard_normal(co.num_params(C)) * 0.3
    img = rng.uniform(0, 255, size=(C, 6, 7))
    dout = rng.standard_normal((6, 7))
    out, cache = co.forward(theta, img)
    g = co.backward(theta, cache, dout)
    # a sample of parameters from every layer (weights and biases)
    offs, o = [], 0
    for cout, cin in co.layer_shapes(C):
        offs += [o, o + cout * cin * 9 - 1, o + cout * cin * 9 + cout - 1]
        o += cout * cin * 9 + cout
    offs += list(rng.choice(co.num_params(C), 20, replace=False))
    eps = 1e-6
    for i in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fp = np.sum(co.forward(tp, img)[0] * dout)
        fm = np.sum(co.forward(tm, img)[0] * dout)
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * (1.0 + abs(fd)), (i, fd, g[i])


def test_loss_gradient():
    rng = np.random.default_rng(3)
    out = rng.standard_normal((20, 24))
    cen = co.ref_centres(20, 24)
    tgt = rng.standard_normal(len(cen))
    L, d = co.loss_and_dout(out, cen, tgt)
    eps = 1e-7
    for (y, x) in cen[:5]:
        op, om = out.copy(), out.copy()
        op[y, x] += eps
        om[y, x] -= eps
        fd = (co.loss_and_dout(op, cen, tgt)[0] - co.loss_and_dout(om, cen, tgt)[0]) / (2 * eps)
        assert abs(fd - d[y, x]) <= 1e-6


def test_first_adam_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = co.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + co.ADAM_EPS), rtol=1e-12)


def test_reference_centres_follow_the_grid():
    c = co.ref_centres(21, 17)
    # grid {0, 4, 8, 12, 13} x {0, 4, 8, 9}: centres shifted by 4
    assert c[0].tolist() == [4, 4] and c[-1].tolist() == [13 + 4, 9 + 4]
    assert len(c) == 5 * 4


def test_window_readout_special_cases():
    rng = np.random.default_rng(4)
    H, W = 40, 36
    cen = co.ref_centres(H, W)
    out = rng.standard_normal((H, W))
    # S = 1 is the centre readout used in training
    np.testing.assert_allclose(co.window_sigma(out, cen, 1), np.exp(out[cen[:, 0], cen[:, 1]]), rtol=1e-14)
    # a constant map gives the constant everywhere, whatever the window
    np.testing.assert_allclose(co.window_sigma(np.full((H, W), 2.5), cen, 16), np.exp(2.5), rtol=1e-14)
    # a linear map averages to its value at the window's mean index: for an even S inside the image
    # the window [c - S/2, c + S/2) has mean index c - 1/2; for an odd S, [c - (S-1)/2, c + (S+1)/2) has c
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    lin = 0.03 * yy - 0.02 * xx
    for S, shift in ((8, -0.5), (5, 0.0)):
        got = np.log(co.window_sigma(lin, cen, S))
        for (cy, cx), g in zip(cen, got):
            if cy - S // 2 >= 0 and cx - S // 2 >= 0 and cy + S - S // 2 <= H and cx + S - S // 2 <= W:
                assert abs(g - (0.03 * (cy + shift) - 0.02 * (cx + shift))) <= 1e-12
    # a window cut by the border: centre (4, 4) of a 40 x 36 map with S = 16 covers rows and columns 0..11
    got = np.log(co.window_sigma(lin, np.array([[4, 4]]), 16))[0]
    assert abs(got - (0.03 * 5.5 - 0.02 * 5.5)) <= 1e-12


def test_fp16_activation_forward():
    # exact case: input k * 255 / 256 (x / 255 = k / 256), centre-tap weights +-1 from one input
    # channel each and biases in multiples of 1/256: every activation is a small multiple of 1/256,
    # exactly representable in FP16, so both forwards agree exactly
    rng = np.random.default_rng(8)
    C = 3
    theta = np.zeros(co.num_params(C))
    o = 0
    for cout, cin in co.layer_shapes(C):
        w = np.zeros((cout, cin, 3, 3))
        for c in range(cout):
            w[c, c % cin, 1, 1] = rng.choice([-1.0, 1.0])
        theta[o:o + w.size] = w.reshape(-1)
        theta[o + w.size:o + w.size + cout] = rng.integers(-4, 5, size=cout) / 256.0
        o += w.size + cout
    img = rng.integers(0, 256, size=(C, 7, 9)) * (255.0 / 256.0)
    np.testing.assert_array_equal(co.forward_act16(theta, img), co.forward(theta, img)[0])
    # generic case: rounding happens (results differ) but stays within a small multiple of the FP16
    # unit roundoff 2^-11 relative to the activations' scale
    theta = co.fp16(rng.standard_normal(co.num_params(C)) * 0.2)
    img = rng.uniform(0, 255, size=(C, 12, 10))
    a, b = co.forward_act16(theta, img), co.forward(theta, img)[0]
    assert np.max(np.abs(a - b)) > 0
    assert np.max(np.abs(a - b)) <= 50 * 2.0 ** -11 * (1.0 + np.max(np.abs(b)))


@pytest.mark.parametrize("C", [1, 3])
def test_fp16_training_gradient(C):
    # structure: with the rounding replaced by the identity, the tensor-core training step's gradient is
    # the FP64 gradient of backward() (pinned above by finite differences) at any loss scale
    rng = np.random.default_rng(20 + C)
    theta = co.fp16(rng.standard_normal(co.num_params(C)) * 0.2)
    img = rng.uniform(0, 255, size=(C, 12, 16))
    cen = co.ref_centres(12, 16)
    tgt = rng.standard_normal(len(cen))
    out, cache = co.forward(theta, img)
    L, dout = co.loss_and_dout(out, cen, tgt)
    want = co.backward(theta, cache, dout)
    for scale in (1.0, 16384.0):
        L2, got = co.grad_act16(theta, img, cen, tgt, scale=scale, rnd=lambda v: v)
        assert abs(L2 - L) <= 1e-12 * (1 + L)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))
    # with FP16 rounding (He-scaled weights, as the library initialises them) every layer's gradient stays
    # within a few FP16 roundoffs of the exact one
    theta = np.concatenate([np.concatenate([rng.standard_normal(co_ * ci * 9) * np.sqrt(2.0 / (9 * ci)),
                                            np.zeros(co_)]) for co_, ci in co.layer_shapes(C)])
    theta = co.fp16(theta)
    out, cache = co.forward(theta, img)
    want = co.backward(theta, cache, co.loss_and_dout(out, cen, tgt)[1])
    L3, g16 = co.grad_act16(theta, img, cen, tgt)
    assert len(cen) == 6 and co.loss_scale(len(cen)) == 16.0  # 2 x 3 references: 2^(2 + 2)
    o = 0
    for cout, cin in co.layer_shapes(C):
        n = cout * cin * 9 + cout
        a, b = g16[o:o + n], want[o:o + n]
        assert np.linalg.norm(a - b) <= 0.02 * np.linalg.norm(b), (cout, cin)
        o += n
