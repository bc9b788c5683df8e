"""Pins of the enhancement strategy's oracle (Eq. 24-25): the network (oracle/fcn_oracle.py) and the
RA filter of the C oracle (the first Haar row of each group replaced by a refined mean patch).

The network's backward pass is pinned to central finite differences of its forward pass, a zero
output layer to the identity refinement, the first Adam step to its closed form.  The RA filter is
pinned where the result is known without the transform: given the groups' own noisy mean patches
and a zero threshold the image comes back exactly (Haar and the projections are orthonormal); with a
threshold above every coefficient only the replaced row survives, so every member of group r is
estimated by its refined mean patch and the output is the plain average of those patches over the
members covering each pixel, computed here by brute force.
"""

import numpy as np
import pytest

from oracle import fcn_oracle as fo
from paper_2512_23569_gb300 import synth


@pytest.mark.parametrize("C", [1, 3])
def test_backward_matches_finite_differences(C):
    rng = np.random.default_rng(20 + C)
    theta = rng.standard_normal(fo.num_params(C)) * 0.1
    X = fo.features(rng.uniform(-255, 255, size=(5, C * 64)), rng.uniform(30, 80, size=5), C, 16)
    dout = rng.standard_normal((5, C * 64))
    out, cache = fo.forward(theta, X, C)
    g = fo.backward(theta, cache, dout, C)
    offs, o = [], 0
    for n_out, n_in in fo.layer_shapes(C):
        offs += [o, o + n_out * n_in - 1, o + n_out * n_in + n_out - 1]
        o += n_out * n_in + n_out
    offs += list(rng.choice(fo.num_params(C), 20, replace=False))
    eps = 1e-6
    for i in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (np.sum(fo.forward(tp, X, C)[0] * dout) - np.sum(fo.forward(tm, X, C)[0] * dout)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * (1.0 + abs(fd)), (i, fd, g[i])


def test_loss_gradient_and_layout():
    rng = np.random.default_rng(4)
    noisy, clean = rng.uniform(0, 255, size=(3, 192)), rng.uniform(0, 255, size=(3, 192))
    out = rng.standard_normal((3, 192)) * 0.1
    sig = np.array([30.0, 50.0, 70.0])
    L, d = fo.loss_and_dout(out, noisy, clean, sig, 16)
    eps = 1e-7
    for (i, j) in ((0, 0), (2, 191), (1, 77)):
        op, om = out.copy(), out.copy()
        op[i, j] += eps
        om[i, j] -= eps
        fd = (fo.loss_and_dout(op, noisy, clean, sig, 16)[0] - fo.loss_and_dout(om, noisy, clean, sig, 16)[0]) / (2 * eps)
        assert abs(fd - d[i, j]) <= 1e-6 * (1 + abs(fd))
    # features: g(c / s) with s = sigma / sqrt(K), then sigma, then zeros up to a multiple of 16;
    # g is odd, g(16) = 8, g(x) -> 16 for large x
    X = fo.features(np.array([[16 * 12.5, -16 * 12.5, 0.0] + [1e9] * 189]), 50.0, 3, 16)
    assert X.shape == (1, 208)
    np.testing.assert_allclose(X[0, :3], [8.0, -8.0, 0.0], rtol=1e-12)
    assert abs(X[0, 3] - 16.0) < 1e-5
    assert X[0, 192] == 50.0 / 255.0 and np.all(X[:, 193:] == 0.0)


def test_zero_output_layer_refines_to_the_input_and_adam():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(fo.num_params(1))
    n_last = 64 * fo.HIDDEN + 64
    theta[-n_last:] = 0.0
    means = rng.uniform(0, 255, size=(4, 64))
    np.testing.assert_array_equal(fo.refine(theta, means, 40.0, 1, 16), means)
    g = np.array([0.5, -2.0, 1e-3])
    th, _, _ = fo.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + fo.ADAM_EPS), rtol=1e-12)


@pytest.mark.parametrize("C", [1, 3])
def test_ra_filter_special_cases(oracle, C):
    clean, noisy = synth.make_config_image(28, 33, C, 40.0, 70 + C)
    p = oracle.Params(K=8, win=9)
    basis, _, _ = oracle.estimate_basis(noisy, p)
    idx, _, _ = oracle.match(noisy, p)
    means = oracle.group_means(noisy, idx, p.ps)
    # own means, zero threshold: perfect reconstruction
    out, _ = oracle.denoise_groups_ra(noisy, p, basis, 0.0, idx, means)
    np.testing.assert_allclose(out, noisy.astype(np.float64), atol=1e-9)
    # threshold above everything: every member becomes its group's (arbitrary) refined mean
    est = np.random.default_rng(3).uniform(0, 255, size=means.shape)
    out, _ = oracle.denoise_groups_ra(noisy, p, basis, 1e12, idx, est)
    H, W = noisy.shape[1:]
    num, cnt = np.zeros((C, H, W)), np.zeros((H, W))
    for r in range(idx.shape[0]):
        e = est[r].reshape(C, 8, 8)
        for pos in idx[r]:
            y, x = pos // W, pos % W
            num[:, y:y + 8, x:x + 8] += e
            cnt[y:y + 8, x:x + 8] += 1
    np.testing.assert_allclose(out, num / cnt, rtol=1e-12, atol=1e-9)


def test_group_means_brute_force(oracle):
    _, noisy = synth.make_config_image(20, 21, 3, 20.0, 9)
    idx = np.array([[0, 5, 21 * 3 + 2], [21 * 12 + 13, 7, 21 * 4]], dtype=np.int32)
    m = oracle.group_means(noisy, idx)
    for r in range(2):
        want = np.mean([noisy[:, q // 21:q // 21 + 8, q % 21:q % 21 + 8].astype(np.float64) for q in idx[r]], axis=0)
        np.testing.assert_allclose(m[r], want.reshape(-1), rtol=1e-12)


@pytest.mark.parametrize("C", [1, 3])
def test_mean_coefs_orthonormal_round_trip(oracle, C):
    # the coordinates keep the norm (Parseval: unitary DFT along the channels, orthonormal bases, the
    # conjugate slice counted by sqrt(2)) and the inverse gives the patches back
    clean, noisy = synth.make_config_image(30, 35, C, 30.0, 80 + C)
    p = oracle.Params(K=8, win=9)
    basis, _, _ = oracle.estimate_basis(noisy, p)
    x = np.random.default_rng(C).uniform(0, 255, size=(6, C * 64))
    c = oracle.mean_coefs(x, basis, C)
    np.testing.assert_allclose(np.linalg.norm(c, axis=1), np.linalg.norm(x, axis=1), rtol=1e-12)
    np.testing.assert_allclose(oracle.coefs_to_patch(c, basis, C), x, rtol=1e-12, atol=1e-9)


def test_coordinates_do_not_depend_on_eigenvector_phases(oracle):
    # multiplying eigenvectors by arbitrary phases (signs for the real slice) leaves the coordinates unchanged
    clean, noisy = synth.make_config_image(30, 35, 3, 30.0, 85)
    basis, _, _ = oracle.estimate_basis(noisy, oracle.Params(K=8, win=9))
    rng = np.random.default_rng(8)
    b2 = np.array(basis)
    b2[0] *= rng.choice([-1.0, 1.0], size=(2, 1, 8))
    b2[1] *= np.exp(1j * rng.uniform(0, 2 * np.pi, size=(2, 1, 8)))
    x = rng.uniform(0, 255, size=(4, 192))
    np.testing.assert_allclose(oracle.mean_coefs(x, b2, 3), oracle.mean_coefs(x, basis, 3), rtol=1e-10, atol=1e-9)
