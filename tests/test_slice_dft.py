"""The tensor-core filter's channel DFT in its real orthonormal form, restated on the host (Eq. 4-5).

The filter's gather turns a pixel's R, G, B into the slice values s0 = P^(1), s1 = sqrt2 Re P^(2),
s2 = sqrt2 Im P^(2) of the unitary DFT along the channels, P^(j) = sum_t c_t w^{(j-1) t} / sqrt3 with
w = exp(-2 pi i / 3) (slice 3 is the conjugate of slice 2), written with the constants 1/sqrt3, sqrt(2/3)
and 1/sqrt2:
    s0 = (r + (g + b)) / sqrt3,   s1 = sqrt(2/3) (r - (g + b) / 2),   s2 = (b - g) / sqrt2,
and the normalisation of the per-slice sums turns them back with the transpose:
    R = s0 / sqrt3 + sqrt(2/3) s1,   t = s0 / sqrt3 - sqrt(2/3) s1 / 2,   G = t - s2 / sqrt2,   B = t + s2 / sqrt2.
These tests check the forward map against the DFT's definition, that it is orthonormal, and that the
inverse undoes it.
"""

import numpy as np

K3F = 1.0 / np.sqrt(3.0)
K23F = np.sqrt(2.0 / 3.0)
R2F = 1.0 / np.sqrt(2.0)


def _forward(r, g, b):
    gb = g + b
    return K3F * (r + gb), K23F * (r - 0.5 * gb), R2F * (b - g)


def _inverse(s0, s1, s2):
    t = K3F * s0 - 0.5 * K23F * s1
    return K3F * s0 + K23F * s1, t - R2F * s2, t + R2F * s2


def test_forward_is_the_unitary_channel_dft():
    rng = np.random.default_rng(11)
    w = np.exp(-2j * np.pi / 3.0)
    for _ in range(200):
        c = rng.normal(0.0, 100.0, 3)
        p1 = np.sum(c) / np.sqrt(3.0)
        p2 = np.sum(c * w ** np.arange(3)) / np.sqrt(3.0)
        s0, s1, s2 = _forward(*c)
        assert abs(s0 - p1) <= 1e-12 * (1 + abs(p1))
        assert abs(s1 - np.sqrt(2.0) * p2.real) <= 1e-12 * (1 + abs(p2))
        assert abs(s2 - np.sqrt(2.0) * p2.imag) <= 1e-12 * (1 + abs(p2))


def test_forward_is_orthonormal_and_the_inverse_its_transpose():
    m = np.array([_forward(*e) for e in np.eye(3)]).T  # columns: images of R, G, B
    assert np.allclose(m @ m.T, np.eye(3), atol=1e-14)
    inv = np.array([_inverse(*e) for e in np.eye(3)]).T
    assert np.allclose(inv, m.T, atol=1e-14)


def test_inverse_undoes_forward_and_keeps_the_energy():
    rng = np.random.default_rng(12)
    for _ in range(200):
        c = rng.uniform(-50.0, 300.0, 3)
        s = np.array(_forward(*c))
        assert np.allclose(_inverse(*s), c, rtol=0, atol=1e-10)
        assert abs(np.sum(s * s) - np.sum(c * c)) <= 1e-9 * np.sum(c * c)
