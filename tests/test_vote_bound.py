"""The rank vote's FP32 evaluation stays inside the error bound it is certified with (Eq. 16-18, 22).

The vote kernel computes the half spectrum X_m = sum_k q_k w^{mk} (w = exp(-2 pi i / K), q_k = p_k - p_0
in FP32, m = 0..K/2) by a radix-2 split per level: a_k = x_k + x_{k+N/2} carries the even outputs (the
same split again), d_k = x_k - x_{k+N/2} the odd ones, which are evaluated directly with d_k paired with
d_{N/2-k}: X_{2j+1} = d_0 + sum_{0<k<N/4} [(d_k - d_{N/2-k}) cos t - i (d_k + d_{N/2-k}) sin t]
+ (-i)^{2j+1} d_{N/4}, t = 2 pi (2j+1) k / N, fused multiply-adds over FP32-rounded twiddles, the quarter
turns as plain sums.  Each input reaches an output part along one path with constants of modulus at most
1 through at most N/4 + 2 roundings (log2 N for X_0), so with the subtraction |X_hat - X| <=
sqrt(2) gamma_(K/4+3) sum_k |q_k| for m != 0, and X_0(p) = X_0(q) + K p_0 (one more fused multiply-add)
errs by at most gamma_(log2 K + 2) (sum_k |q_k| + K |p_0|).  The kernel certifies its decisions with the
wider sqrt(2) (K + 3) u times these sums (u = 2^-24).  This test restates that arithmetic in NumPy (a fused
multiply-add as the exact FP64 product-sum rounded once to FP32), checks the recursion's formula against
the definition in FP64, and checks the FP32 errors against the tight bounds on random and adversarial
patches, for every group size the library builds.
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


def _half_spectrum(x, N, tc, ts, f):
    """X_m, m = 0..N/2, of the N values x by the kernel's recursion; f rounds every operation (F for the
    kernel's FP32, float for the FP64 check of the formula).  Returns {m: (re, im)}."""
    def fma(a, b, c):
        return _fma32(a, b, c) if f is F else a * b + c
    if N == 2:
        return {0: (f(x[0] + x[1]), f(0.0)), 1: (f(x[0] - x[1]), f(0.0))}
    n = N // 2
    a = [f(x[k] + x[k + n]) for k in range(n)]
    d = [f(x[k] - x[k + n]) for k in range(n)]
    out = {2 * j: v for j, v in _half_spectrum(a, n, tc, ts, f).items()}
    dd = {k: f(d[k] - d[n - k]) for k in range(1, n // 2)}
    ss = {k: f(d[k] + d[n - k]) for k in range(1, n // 2)}
    for j in range(n // 2):
        r = d[0]
        i = d[n // 2] if j & 1 else f(-d[n // 2])
        for k in range(1, n // 2):
            t = ((2 * j + 1) * k * (32 // N)) & 31
            if t == 0:
                r = f(r + dd[k])
            elif t == 8:
                i = f(i - ss[k])
            elif t == 16:
                r = f(r - dd[k])
            elif t == 24:
                i = f(i + ss[k])
            else:
                r = fma(dd[k], tc[t] if f is F else np.cos(2 * np.pi * t / 32), r)
                i = fma(ss[k], ts[t] if f is F else -np.sin(2 * np.pi * t / 32), i)
        out[2 * j + 1] = (r, i)
    return out


def _patches(K, rng):
    yield rng.uniform(0.0, 255.0, K)                          # noise
    yield 200.0 + rng.normal(0.0, 1e-3, K)                    # near-constant at a large offset
    yield np.where(np.arange(K) % 2 == 0, 255.0, 0.0)         # alternating extremes
    yield 765.0 * rng.random(K) ** 8                          # sum-plane range, skewed
    yield np.full(K, 123.456)                                 # constant


def _gamma(n):
    return n * U / (1.0 - n * U)


@pytest.mark.parametrize("K", [2, 4, 8, 16, 32])
def test_recursion_is_the_dft(K):
    # the formula in FP64 against the definition sum_k x_k w^{mk}
    rng = np.random.default_rng(700 + K)
    for _ in range(20):
        x = rng.normal(0.0, 50.0, K)
        got = _half_spectrum(list(x), K, None, None, float)
        assert sorted(got) == list(range(K // 2 + 1))
        for m, (re, im) in got.items():
            exact = complex(np.sum(x * np.exp(-2j * np.pi * m * np.arange(K) / K)))
            assert abs(complex(re, im) - exact) <= 1e-9 * (1.0 + np.sum(np.abs(x))), (K, m)


@pytest.mark.parametrize("K", [2, 4, 8, 16, 32])
def test_radix2_dft_within_certified_bound(K):
    tc, ts = _twiddles()
    rng = np.random.default_rng(900 + K)
    logk = int(np.log2(K))
    worst = 0.0
    for _ in range(40):
        for p in _patches(K, rng):
            p = p.astype(np.float32)
            q_hat = [F(0.0)] + [F(p[k] - p[0]) for k in range(1, K)]
            q = p.astype(np.float64) - np.float64(p[0])          # exact differences
            l1 = float(np.sum(np.abs(q)))
            l1_hat = float(np.sum(np.abs(np.array(q_hat, dtype=np.float64))))
            got = _half_spectrum(q_hat, K, tc, ts, F)
            for m in range(1, K // 2 + 1):
                exact = complex(np.sum(q * np.exp(-2j * np.pi * m * np.arange(K) / K)))
                err = abs(complex(float(got[m][0]), float(got[m][1])) - exact)
                tight = np.sqrt(2.0) * _gamma(K // 4 + 3) * l1 + 1e-30
                certified = np.sqrt(2.0) * (K + 3) * U * l1_hat * 1.01 + 1e-30
                assert err <= tight, (K, m, err, tight)
                assert tight <= certified * (1.0 + 1e-6)
                worst = max(worst, err / tight)
            # X_0(p) = X_0(q) + K p_0, one fused multiply-add
            x0 = float(_fma32(F(K), p[0], got[0][0]))
            exact0 = float(np.sum(p.astype(np.float64)))
            e0 = l1 + K * abs(float(p[0]))
            assert abs(x0 - exact0) <= _gamma(logk + 2) * e0 + 1e-30, (K, x0, exact0)
            assert _gamma(logk + 2) * e0 <= np.sqrt(2.0) * (K + 3) * U * e0 * 1.01 + 1e-30
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
