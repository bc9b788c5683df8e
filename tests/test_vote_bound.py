"""The rank vote's FP32 evaluation stays inside the error bound it is certified with (Eq. 16-18, 22).

The vote kernel computes X_m = sum_k q_k w^{mk} (w = exp(-2 pi i / K), q_k = p_k - p_0 in FP32) by
pairing k with K - k: (q_k + q_{K-k}) cos and (q_k - q_{K-k}) (-sin) accumulated with fused
multiply-adds over FP32-rounded twiddles, the quarter turns as plain sums and the K/2 term as
(-1)^m q_{K/2}.  Its decisions are certified with the per-component bound
|X_hat - X| <= sqrt(2) (K + 3) u sum_k |q_hat_k| (u = 2^-24); the pairing's own error analysis gives
sqrt(2) (K/2 + 5/2) u sum_k |q_k|.  This test restates that arithmetic in NumPy (a fused multiply-add
as the exact FP64 product-sum rounded once to FP32) and checks the error against the tighter bound
on random and adversarial patches, for every group size the library builds.
"""

import numpy as np
import pytest

U = 2.0 ** -24
F = np.float32


def _fma32(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _twiddles():
    j = np.arange(32)
    return (np.cos(2.0 * np.pi * j / 32.0).astype(np.float32),
            (-np.sin(2.0 * np.pi * j / 32.0)).astype(np.float32))


def _paired(q, K, m, tc, ts):
    sp = {k: F(q[k] + q[K - k]) for k in range(1, K // 2)}
    dm = {k: F(q[k] - q[K - k]) for k in range(1, K // 2)}
    xr = F(-q[K // 2]) if m & 1 else F(q[K // 2])
    xi = F(0.0)
    for k in range(1, K // 2):
        j = ((m * k) % K) * (32 // K)
        if j == 0:
            xr = F(xr + sp[k])
        elif j == 8:
            xi = F(xi - dm[k])
        elif j == 16:
            xr = F(xr - sp[k])
        elif j == 24:
            xi = F(xi + dm[k])
        else:
            xr = _fma32(sp[k], tc[j], xr)
            xi = _fma32(dm[k], ts[j], xi)
    return complex(float(xr), float(xi))


def _patches(K, rng):
    yield rng.uniform(0.0, 255.0, K)                          # noise
    yield 200.0 + rng.normal(0.0, 1e-3, K)                    # near-constant at a large offset
    yield np.where(np.arange(K) % 2 == 0, 255.0, 0.0)         # alternating extremes
    yield 765.0 * rng.random(K) ** 8                          # sum-plane range, skewed
    yield np.full(K, 123.456)                                 # constant


@pytest.mark.parametrize("K", [2, 4, 8, 16, 32])
def test_paired_dft_within_certified_bound(K):
    tc, ts = _twiddles()
    rng = np.random.default_rng(900 + K)
    worst = 0.0
    for _ in range(40):
        for p in _patches(K, rng):
            p = p.astype(np.float32)
            q_hat = np.array([F(p[k] - p[0]) for k in range(K)], dtype=np.float32)
            q = p.astype(np.float64) - np.float64(p[0])          # exact differences
            l1 = float(np.sum(np.abs(q)))
            for m in range(1, K // 2 + 1):
                exact = complex(np.sum(q * np.exp(-2j * np.pi * m * np.arange(K) / K)))
                got = _paired(q_hat, K, m, tc, ts)
                err = abs(got - exact)
                tight = np.sqrt(2.0) * (K / 2 + 2.5) * U * l1 * 1.01 + 1e-30
                certified = np.sqrt(2.0) * (K + 3) * U * float(np.sum(np.abs(q_hat))) * 1.01 + 1e-30
                assert err <= tight, (K, m, err, tight)
                assert tight <= certified * (1.0 + 1e-6)
                worst = max(worst, err / tight)
    assert worst > 0.0  # the emulation rounds at all


def test_quarter_turn_sums_equal_fma():
    # fmaf with an exact 0 or +-1 twiddle rounds like the plain sum or difference
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a = F(rng.normal() * 10.0 ** rng.integers(-3, 4))
        c = F(rng.normal() * 10.0 ** rng.integers(-3, 4))
        assert _fma32(a, F(1.0), c) == F(c + a)
        assert _fma32(a, F(-1.0), c) == F(c - a)
        assert _fma32(a, F(0.0), c) == c
