"""Seeded synthetic test images for the Haar-tSVD denoiser.

This module only draws inputs: clean piecewise-constant images with gratings
and the noise models used for evaluation.  It holds none of the denoiser's
arithmetic, so both the CUDA path and the FP64 oracle may consume what it
produces without sharing any method code.

Recipe (one ``numpy.random.Generator(PCG64(seed))`` per image):

* background: a constant drawn from U[0, 255];
* 20 axis-aligned rectangles, corners uniform over the image, intensity U[0, 255];
* 10 disks, centre uniform, radius U[4, min(H, W)/6], intensity U[0, 255];
* 2 sinusoidal gratings, each confined to a random rectangle: period U[6, 20] px,
  orientation U[0, pi), amplitude A ~ U[20, 60], mean U[A, 255 - A];
* shapes are painted in that order, each overwriting what lies below it; the
  result is clipped to [0, 255];
* colour images share the geometry; every shape (and the background) gets
  per-channel gains U[0.8, 1.2] applied before clipping.

Layout is planar CHW float32 (C = 1 or 3), row-major.  Noisy images are never
clipped.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "clean_image",
    "awgn",
    "poisson_gaussian",
    "correlate_noise",
    "make_config_image",
    "psnr",
    "make_pg_correlated_image",
    "add_varying_noise",
    "make_varying_noise_image",
    "ref_log_sigma",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def clean_image(H: int, W: int, C: int, seed: int) -> np.ndarray:
    """Seeded clean image, float32 CHW in [0, 255]."""
    if C not in (1, 3):
        raise ValueError("C must be 1 or 3")
    rng = _rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)

    def gains() -> np.ndarray:
        if C == 1:
            return np.ones(1)
        return rng.uniform(0.8, 1.2, size=C)

    img = np.empty((C, H, W), dtype=np.float64)
    bg = rng.uniform(0.0, 255.0)
    g = gains()
    for c in range(C):
        img[c] = bg * g[c]

    # 20 rectangles
    for _ in range(20):
        y0, y1 = np.sort(rng.uniform(0, H, size=2))
        x0, x1 = np.sort(rng.uniform(0, W, size=2))
        val = rng.uniform(0.0, 255.0)
        g = gains()
        m = (yy >= y0) & (yy <= y1) & (xx >= x0) & (xx <= x1)
        for c in range(C):
            img[c][m] = val * g[c]

    # 10 disks
    rmax = max(4.0, min(H, W) / 6.0)
    for _ in range(10):
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        r = rng.uniform(4.0, rmax)
        val = rng.uniform(0.0, 255.0)
        g = gains()
        m = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        for c in range(C):
            img[c][m] = val * g[c]

    # 2 gratings inside random rectangles
    for _ in range(2):
        y0, y1 = np.sort(rng.uniform(0, H, size=2))
        x0, x1 = np.sort(rng.uniform(0, W, size=2))
        period = rng.uniform(6.0, 20.0)
        theta = rng.uniform(0.0, np.pi)
        amp = rng.uniform(20.0, 60.0)
        mean = rng.uniform(amp, 255.0 - amp)
        g = gains()
        m = (yy >= y0) & (yy <= y1) & (xx >= x0) & (xx <= x1)
        phase = 2.0 * np.pi * (xx * np.cos(theta) + yy * np.sin(theta)) / period
        wave = mean + amp * np.sin(phase)
        for c in range(C):
            img[c][m] = (wave * g[c])[m]

    np.clip(img, 0.0, 255.0, out=img)
    return img.astype(np.float32)


def awgn(clean: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """clean + N(0, sigma^2), float32, not clipped."""
    rng = _rng(seed)
    n = rng.standard_normal(clean.shape) * float(sigma)
    return (clean.astype(np.float64) + n).astype(np.float32)


def poisson_gaussian(clean: np.ndarray, a: float, sigma_b: float, seed: int) -> np.ndarray:
    """a * Poisson(clean / a) + N(0, sigma_b^2) on the [0, 255] scale (float32).

    ``a`` may be a scalar or an array broadcastable to ``clean`` (spatially
    varying gain); ``a == 0`` means no shot noise.
    """
    rng = _rng(seed)
    x = clean.astype(np.float64)
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), x.shape)
    shot = np.where(a > 0, a * rng.poisson(np.where(a > 0, x / np.maximum(a, 1e-300), 0.0)), x)
    sb = np.broadcast_to(np.asarray(sigma_b, dtype=np.float64), x.shape)
    y = shot + rng.standard_normal(x.shape) * sb
    return y.astype(np.float32)


def correlate_noise(clean: np.ndarray, noisy: np.ndarray, std: float = 0.7) -> np.ndarray:
    """Convolve the noise (noisy - clean) with a normalised 3x3 Gaussian (reflect border)."""
    r = np.arange(-1, 2, dtype=np.float64)
    k1 = np.exp(-0.5 * (r / std) ** 2)
    k = np.outer(k1, k1)
    k /= k.sum()
    n = noisy.astype(np.float64) - clean.astype(np.float64)
    out = np.zeros_like(n)
    pad = np.pad(n, ((0, 0), (1, 1), (1, 1)), mode="reflect")
    H, W = n.shape[1:]
    for dy in range(3):
        for dx in range(3):
            out += k[dy, dx] * pad[:, dy:dy + H, dx:dx + W]
    return (clean.astype(np.float64) + out).astype(np.float32)


def make_config_image(H: int, W: int, C: int, sigma: float, seed: int):
    """(clean, noisy) pair with AWGN of std ``sigma``; noise seed = seed + 1."""
    clean = clean_image(H, W, C, seed)
    noisy = awgn(clean, sigma, seed + 1)
    return clean, noisy


def psnr(x: np.ndarray, ref: np.ndarray) -> float:
    """10 log10(255^2 / MSE) over all pixels and channels."""
    d = x.astype(np.float64) - ref.astype(np.float64)
    mse = float(np.mean(d * d))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(255.0 * 255.0 / mse)


def make_pg_correlated_image(H: int, W: int, C: int, seed: int, a: float = 0.01, sigma_b: float = 5.0,
                             std: float = 0.7):
    """(clean, noisy): Poisson-Gaussian noise (gain a, read noise sigma_b), then spatially correlated
    by a normalised 3x3 Gaussian of std ``std``; noise seed = seed + 1."""
    clean = clean_image(H, W, C, seed)
    noisy = correlate_noise(clean, poisson_gaussian(clean, a, sigma_b, seed + 1), std)
    return clean, noisy


def add_varying_noise(clean: np.ndarray, seed: int, a_max: float = 0.02, sb_max: float = 30.0,
                      sb_min: float = 0.0, gain: float | None = None, levels: tuple | None = None):
    """(noisy, sigma_px): Poisson-Gaussian noise on `clean` whose read-noise level varies across it.

    Gain a ~ U[0, a_max]; sigma_b ramps linearly between two levels drawn from
    U[sb_min, sb_max] along a direction drawn from U[0, 2 pi) (all from seed's
    generator); the noise itself uses seed + 1.  `gain` and `levels` (the
    ramp's two ends), when given, replace the drawn a and levels (the
    generator still draws them, so the direction is the same).  sigma_px (H, W)
    is the true per-pixel standard deviation, the root mean over channels of
    a * clean + sigma_b^2.
    """
    C, H, W = clean.shape
    rng = _rng(seed)
    a = float(rng.uniform(0.0, a_max))
    s0, s1 = rng.uniform(sb_min, sb_max, size=2)
    if gain is not None:
        a = float(gain)
    if levels is not None:
        s0, s1 = float(levels[0]), float(levels[1])
    th = rng.uniform(0.0, 2.0 * np.pi)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    proj = np.cos(th) * yy + np.sin(th) * xx
    t = (proj - proj.min()) / max(proj.max() - proj.min(), 1e-12)
    sb = s0 + (s1 - s0) * t
    noisy = poisson_gaussian(clean, a, sb[None], seed + 1)
    var = a * clean.astype(np.float64) + sb[None] ** 2
    return noisy, np.sqrt(var.mean(axis=0))


def make_varying_noise_image(H: int, W: int, C: int, seed: int, a_max: float = 0.02, sb_max: float = 30.0,
                             sb_min: float = 0.0, gain: float | None = None, levels: tuple | None = None):
    """(clean, noisy, sigma_px): clean_image(seed) with add_varying_noise(clean, seed + 1, ...)."""
    clean = clean_image(H, W, C, seed)
    noisy, sigma_px = add_varying_noise(clean, seed + 1, a_max, sb_max, sb_min, gain, levels)
    return clean, noisy, sigma_px


def ref_log_sigma(sigma_px: np.ndarray, ps: int = 8, step: int = 4) -> np.ndarray:
    """log of the RMS noise level over every reference patch (row-major over the reference grid:
    0, step, 2 step, ... plus the last position n - ps), float32."""
    H, W = sigma_px.shape

    def grid(n):
        g = list(range(0, n - ps + 1, step))
        if g[-1] != n - ps:
            g.append(n - ps)
        return g

    v = sigma_px.astype(np.float64) ** 2
    S = np.zeros((H + 1, W + 1))
    S[1:, 1:] = v.cumsum(0).cumsum(1)
    ys, xs = np.asarray(grid(H)), np.asarray(grid(W))
    box = (S[np.ix_(ys + ps, xs + ps)] - S[np.ix_(ys, xs + ps)] - S[np.ix_(ys + ps, xs)] + S[np.ix_(ys, xs)])
    return np.log(np.sqrt(np.maximum(box, 0.0) / (ps * ps))).reshape(-1).astype(np.float32)
