"""FP64 CPU oracle of the learned noise-level map -- TEST INFRASTRUCTURE ONLY.

Only the test-suite and the benchmark may import this module; the CUDA
library never calls it and shares no code with it.

The network (the learned sigma estimate that replaces Eq. 12-23 in the
paper's adaptive variant, Sec. III-C) maps the noisy image, scaled by 1/255,
through five 3x3 convolutions with zero padding (widths C -> 32 -> 32 -> 32
-> 32 -> 1, ReLU after the first four) to a map of log(sigma) on the [0, 255]
scale.  Training reads the map at the centre (y + 4, x + 4) of the reference
patch with top-left corner (y, x); denoising averages it over a window around
that centre (window_sigma).  Weights are held in FP16 for the forward pass (the values
here are the FP16-rounded ones, computed in FP64); training minimises the
mean squared error of log(sigma) over the reference patches with Adam.

Parameter vector layout (shared with the library's host interface): for
every layer l, W_l[co][ci][ky][kx] then b_l[co].
"""

from __future__ import annotations

import numpy as np

WIDTH = 32
DEPTH = 5
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def layer_shapes(C: int):
    """[(cout, cin)] of the five layers."""
    widths = [C] + [WIDTH] * (DEPTH - 1) + [1]
    return [(widths[i + 1], widths[i]) for i in range(DEPTH)]


def num_params(C: int) -> int:
    return sum(co * ci * 9 + co for co, ci in layer_shapes(C))


def unpack(theta: np.ndarray, C: int):
    """Parameter vector -> [(W (co, ci, 3, 3), b (co,))]."""
    out, o = [], 0
    for co, ci in layer_shapes(C):
        w = theta[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    return out


def fp16(theta: np.ndarray) -> np.ndarray:
    return np.asarray(theta, dtype=np.float64).astype(np.float16).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[co, y, x] = b[co] + sum_ci sum_ky,kx w[co, ci, ky, kx] * xpad[ci, y + ky, x + kx]."""
    ci, H, W = x.shape
    xp = np.zeros((ci, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.empty((w.shape[0], H, W))
    for co in range(w.shape[0]):
        acc = np.full((H, W), float(b[co]))
        for c in range(ci):
            for ky in range(3):
                for kx in range(3):
                    acc += w[co, c, ky, kx] * xp[c, ky:ky + H, kx:kx + W]
        out[co] = acc
    return out


def forward(theta: np.ndarray, img: np.ndarray):
    """Returns (log-sigma map (H, W), cache for backward).  theta: FP16-rounded values."""
    C = img.shape[0]
    layers = unpack(theta, C)
    a = np.asarray(img, dtype=np.float64) / 255.0
    cache = [a]
    for li, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        a = np.maximum(z, 0.0) if li < DEPTH - 1 else z
        cache.append(a)
    return a[0], cache


def forward_act16(theta: np.ndarray, img: np.ndarray) -> np.ndarray:
    """The forward pass used for denoising: as forward(), with the network input x / 255 and every
    hidden activation (after ReLU) rounded to FP16 (round to nearest even).  Returns the map (H, W)."""
    C = img.shape[0]
    layers = unpack(theta, C)
    a = fp16(np.asarray(img, dtype=np.float64) / 255.0)
    for li, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        a = fp16(np.maximum(z, 0.0)) if li < DEPTH - 1 else z
    return a[0]


def backward(theta: np.ndarray, cache, dout: np.ndarray) -> np.ndarray:
    """Gradient of sum(dout * out) with respect to the parameter vector."""
    C = cache[0].shape[0]
    layers = unpack(theta, C)
    grads = []
    d = dout[None, :, :].astype(np.float64)
    for li in range(DEPTH - 1, -1, -1):
        w, b = layers[li]
        x = cache[li]
        if li < DEPTH - 1:
            d = d * (cache[li + 1] > 0)  # ReLU of this layer's output
        ci, H, W = x.shape
        xp = np.zeros((ci, H + 2, W + 2))
        xp[:, 1:-1, 1:-1] = x
        dw = np.empty_like(w)
        for co in range(w.shape[0]):
            for c in range(ci):
                for ky in range(3):
                    for kx in range(3):
                        dw[co, c, ky, kx] = np.sum(d[co] * xp[c, ky:ky + H, kx:kx + W])
        db = d.sum(axis=(1, 2))
        grads.append((dw, db))
        if li > 0:  # gradient of the layer input: correlation with the flipped kernels
            dp = np.zeros((w.shape[0], H + 2, W + 2))
            dp[:, 1:-1, 1:-1] = d
            dx = np.zeros((ci, H, W))
            for c in range(ci):
                for co in range(w.shape[0]):
                    for ky in range(3):
                        for kx in range(3):
                            dx[c] += w[co, c, ky, kx] * dp[co, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W]
            d = dx
    out = []
    for dw, db in reversed(grads):
        out.append(dw.reshape(-1))
        out.append(db)
    return np.concatenate(out)


def loss_scale(nref: int) -> float:
    """The loss scale of the tensor-core training step: 2^(floor(log2 N_ref) + 2), so that the scaled loss
    gradient 2 (out - target) / N_ref * scale lies within (4, 8] times the error."""
    return float(2 ** (int(np.floor(np.log2(nref))) + 2))


def grad_act16(theta: np.ndarray, img: np.ndarray, centres: np.ndarray, target_log_sigma: np.ndarray,
               scale: float | None = None, rnd=fp16):
    """Loss and gradient as the tensor-core training step forms them: the forward of forward_act16 (network
    input and hidden activations rounded by `rnd`), the loss gradient map times `scale` (loss_scale by
    default) rounded, and going back through each layer the gradient of its input (correlation with the
    flipped kernels, times the ReLU mask of the stored activation) rounded; the weight and bias gradients are
    exact sums of those rounded values, divided by `scale`.  With rnd = identity this is the FP64 gradient of
    backward()."""
    if scale is None:
        scale = loss_scale(len(centres))
    C = img.shape[0]
    layers = unpack(theta, C)
    a = rnd(np.asarray(img, dtype=np.float64) / 255.0)
    acts = [a]
    for li, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        a = rnd(np.maximum(z, 0.0)) if li < DEPTH - 1 else z
        acts.append(a)
    loss, dout = loss_and_dout(acts[-1][0], centres, target_log_sigma)
    d = rnd(dout * scale)[None, :, :]
    grads = []
    for li in range(DEPTH - 1, -1, -1):
        w, _ = layers[li]
        x = acts[li]
        ci, H, W = x.shape
        xp = np.zeros((ci, H + 2, W + 2))
        xp[:, 1:-1, 1:-1] = x
        dw = np.empty_like(w)
        for co in range(w.shape[0]):
            for c in range(ci):
                for ky in range(3):
                    for kx in range(3):
                        dw[co, c, ky, kx] = np.sum(d[co] * xp[c, ky:ky + H, kx:kx + W])
        grads.append((dw / scale, d.sum(axis=(1, 2)) / scale))
        if li > 0:
            dp = np.zeros((w.shape[0], H + 2, W + 2))
            dp[:, 1:-1, 1:-1] = d
            dx = np.zeros((ci, H, W))
            for c in range(ci):
                for co in range(w.shape[0]):
                    for ky in range(3):
                        for kx in range(3):
                            dx[c] += w[co, c, ky, kx] * dp[co, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W]
            d = rnd(dx * (acts[li] > 0))  # the ReLU of layer li - 1's output
    out = []
    for dw, db in reversed(grads):
        out.append(dw.reshape(-1))
        out.append(db)
    return loss, np.concatenate(out)


def ref_centres(H: int, W: int, ps: int = 8, step: int = 4):
    """(y + 4, x + 4) of every reference patch, raster order (Alg. 1 grid)."""
    def grid(n):
        g = list(range(0, n - ps + 1, step))
        if g[-1] != n - ps:
            g.append(n - ps)
        return g
    ys, xs = grid(H), grid(W)
    return np.array([(y + ps // 2, x + ps // 2) for y in ys for x in xs], dtype=np.int64)


def window_sigma(out: np.ndarray, centres: np.ndarray, S: int) -> np.ndarray:
    """Noise level of every reference patch for denoising: exp of the mean of the log-sigma map over
    rows [cy - S // 2, cy - S // 2 + S) x columns [cx - S // 2, cx - S // 2 + S) cut to the image
    (the paper's one level per sub-image, the sub-image moved with the patch; S = 1 reads the centre)."""
    H, W = out.shape
    res = np.empty(len(centres))
    for i, (cy, cx) in enumerate(centres):
        y0, x0 = max(0, cy - S // 2), max(0, cx - S // 2)
        y1, x1 = min(H, cy - S // 2 + S), min(W, cx - S // 2 + S)
        res[i] = np.exp(np.mean(out[y0:y1, x0:x1]))
    return res


def loss_and_dout(out: np.ndarray, centres: np.ndarray, target_log_sigma: np.ndarray):
    """Mean squared error over the reference patches and its gradient map."""
    pred = out[centres[:, 0], centres[:, 1]]
    diff = pred - np.asarray(target_log_sigma, dtype=np.float64)
    n = len(diff)
    dout = np.zeros_like(out)
    np.add.at(dout, (centres[:, 0], centres[:, 1]), 2.0 * diff / n)
    return float(np.mean(diff * diff)), dout


def adam_step(theta, m, v, g, t: int, lr: float):
    """One Adam update (bias-corrected), returns (theta, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mh = m / (1 - ADAM_B1 ** t)
    vh = v / (1 - ADAM_B2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v
