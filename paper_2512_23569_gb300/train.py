"""Training of the learned noise-level map on pairs the method itself generates.

Host-side orchestration only: every forward, backward and optimiser step runs
in the library's kernels (hts_cnn_accumulate_grad, hts_cnn_adam_step), every
denoising in hts_denoise_sigma_map.

Targets.  For a training image whose clean content and per-pixel noise level
are known (synth.make_varying_noise_image), the target of reference patch r is
log(m* sigma_r): sigma_r is the generator's RMS noise level over the patch and
m* the factor on the whole image's sigma map that gives the highest PSNR when
the method denoises the image with per-patch thresholds -- the threshold level
the method itself prefers, found by running it over a grid of factors.
"""

from __future__ import annotations

import numpy as np

from . import hts, synth

MULTS = tuple(round(0.5 + 0.1 * i, 1) for i in range(11))  # 0.5, 0.6, ..., 1.5


def best_multiplier(x, clean, sigma_ref, p, mults=MULTS, out=None) -> float:
    """Factor m of `mults` for which denoising x with thresholds from m * sigma_ref gives the lowest
    mean squared error against `clean` (CUDA tensors of the same shape; sigma_ref: CUDA, N_ref)."""
    import torch

    if out is None:
        out = torch.empty_like(x)
    mse = []
    for m in mults:
        hts.denoise_sigma_map(x, (sigma_ref * m).contiguous(), p=p, out=out)
        mse.append(torch.mean((out - clean) ** 2))
    return float(mults[int(torch.argmin(torch.stack(mse)).item())])


def targets(noisy, clean, sigma_px, p, mults=MULTS):
    """(x, target, m*) of one training image: x the noisy CUDA tensor, target log(m* sigma_r) (CUDA, N_ref)."""
    import torch

    x = torch.from_numpy(np.ascontiguousarray(noisy, dtype=np.float32)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(clean, dtype=np.float32)).cuda()
    ls = synth.ref_log_sigma(sigma_px, p.ps, p.step)
    sref = torch.from_numpy(np.exp(ls.astype(np.float64)).astype(np.float32)).cuda()
    m = best_multiplier(x, c, sref, p, mults)
    return x, torch.from_numpy((ls + np.float32(np.log(m))).astype(np.float32)).cuda(), m


def fit(net, xs, ts, p, steps: int, batch: int = 8, lr0: float = 2e-3, seed: int = 0, every: int = 64):
    """Mini-batch Adam over (xs[i], ts[i]): each step sums the gradients of `batch` images drawn without
    replacement (epochs of a seeded permutation); the step size decays exponentially from lr0 to lr0 / 10.
    Returns the mean loss per image over each block of `every` steps."""
    rng = np.random.default_rng(seed)
    n = len(xs)
    order = np.concatenate([rng.permutation(n) for _ in range(steps * batch // n + 1)])
    hist = []
    for it in range(steps):
        net.zero_grad()
        for j in order[it * batch:(it + 1) * batch]:
            net.accumulate_grad(xs[j], ts[j], p)
        net.adam_step(lr0 * (0.1 ** (it / steps)))
        if it % every == every - 1:
            hist.append(net.take_loss() / (every * batch))
    return hist
