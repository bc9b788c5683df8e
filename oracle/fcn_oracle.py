"""FP64 CPU oracle of the enhancement strategy's network -- TEST INFRASTRUCTURE ONLY.

Only the test-suite and the benchmark may import this module; the CUDA
library never calls it and shares no code with it.

RA-Haar-tSVD (Eq. 24-25) refines the mean patch of every group with a plain
fully connected network trained by residual learning.  The mean patch enters
in the image's transform (hts_oracle.mean_coefs: the orthonormal coordinates
of Eq. 19 without the Haar factor, C * 64 values), where it is sparse, and in
units of its noise level s = sigma / sqrt(K) (the mean of K patches): the
input is g(c / s) with g(x) = x / (1 + |x| / 16) (noise-only coordinates
stay near x, strong ones saturate), then sigma / 255, zero-padded to a
multiple of 16 features; two hidden layers of 128 units with ReLU; a linear
output of C * 64 values, the residual in noise units: refined = c + s *
output.  Training minimises the mean squared error of the output against
(clean - noisy) / s over samples and values with Adam.

Parameter vector layout (shared with the library's host interface): for
every layer l, W_l[out][in] then b_l[out].
"""

from __future__ import annotations

import numpy as np

HIDDEN = 128
SAT = 16.0  # saturation of the input compression g
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def in_dim(C: int) -> int:
    """C * 64 mean-patch values + sigma, padded to a multiple of 16."""
    return (C * 64 + 1 + 15) // 16 * 16


def layer_shapes(C: int):
    """[(out, in)] of the three layers."""
    return [(HIDDEN, in_dim(C)), (HIDDEN, HIDDEN), (C * 64, HIDDEN)]


def num_params(C: int) -> int:
    return sum(o * i + o for o, i in layer_shapes(C))


def unpack(theta: np.ndarray, C: int):
    out, o = [], 0
    for n_out, n_in in layer_shapes(C):
        w = np.asarray(theta[o:o + n_out * n_in], dtype=np.float64).reshape(n_out, n_in)
        o += n_out * n_in
        b = np.asarray(theta[o:o + n_out], dtype=np.float64)
        o += n_out
        out.append((w, b))
    return out


def noise_unit(sigma, K: int, n: int) -> np.ndarray:
    """s = sigma / sqrt(K) per sample (n,)."""
    return np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n,)) / np.sqrt(K)


def features(coefs: np.ndarray, sigma, C: int, K: int) -> np.ndarray:
    """Network input (n, in_dim): g(coefs / s), then sigma / 255 (one value or one per sample), zeros."""
    m = np.asarray(coefs, dtype=np.float64)
    s = noise_unit(sigma, K, m.shape[0])[:, None]
    x = m / s
    X = np.zeros((m.shape[0], in_dim(C)))
    X[:, :C * 64] = x / (1.0 + np.abs(x) / SAT)
    X[:, C * 64] = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (m.shape[0],)) / 255.0
    return X


def forward(theta: np.ndarray, X: np.ndarray, C: int):
    """Output (n, C * 64) and the cache for backward."""
    layers = unpack(theta, C)
    a = np.asarray(X, dtype=np.float64)
    cache = [a]
    for li, (w, b) in enumerate(layers):
        z = a @ w.T + b
        a = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        cache.append(a)
    return a, cache


def refine(theta: np.ndarray, coefs: np.ndarray, sigma, C: int, K: int) -> np.ndarray:
    """Eq. 25: the refined mean patches (transform coordinates), c + s * network output."""
    c = np.asarray(coefs, dtype=np.float64)
    out, _ = forward(theta, features(c, sigma, C, K), C)
    return c + noise_unit(sigma, K, c.shape[0])[:, None] * out


def loss_and_dout(out: np.ndarray, noisy: np.ndarray, clean: np.ndarray, sigma, K: int):
    """Mean squared error of the output against (clean - noisy) / s, and d loss / d out."""
    n = np.asarray(noisy, dtype=np.float64)
    target = (np.asarray(clean, dtype=np.float64) - n) / noise_unit(sigma, K, n.shape[0])[:, None]
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(theta: np.ndarray, cache, dout: np.ndarray, C: int) -> np.ndarray:
    """Gradient of sum(dout * out) with respect to the parameter vector."""
    layers = unpack(theta, C)
    d = np.asarray(dout, dtype=np.float64)
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        if li < len(layers) - 1:
            d = d * (cache[li + 1] > 0)
        grads.append((d.T @ cache[li], d.sum(axis=0)))
        d = d @ w
    out = []
    for dw, db in reversed(grads):
        out.append(dw.reshape(-1))
        out.append(db)
    return np.concatenate(out)


def adam_step(theta, m, v, g, t: int, lr: float):
    """One Adam update (bias-corrected), returns (theta, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mh = m / (1 - ADAM_B1 ** t)
    vh = v / (1 - ADAM_B2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v
