"""hts_denoise_noalloc against hts_denoise (GPU).

hts_denoise_noalloc serves callers that may not allocate device memory while
they run (a plugin whose host application owns the device memory budget, a
loop that cannot take cudaMalloc's implicit synchronisation); it keeps all
intermediates in the library's static device scratch.  These tests call it
through the C ABI and compare it with the allocating entry point, on two calls
in a row of different shapes, so a call that left stale data in the shared
scratch would show.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 1e-3


@pytest.fixture(scope="module")
def hts():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2512_23569_gb300 import build, hts as h

    build.build()
    h.load()
    return h


def _noalloc(hts, x, sigma, p, basis=None):
    lib = hts.load()
    out = torch.empty_like(x)
    C, H, W = x.shape
    s = -1.0 if sigma is None else float(sigma)
    r = lib.hts_denoise_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C,
                                ctypes.c_float(s), basis.handle if basis else None, ctypes.byref(p),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == 0, lib.hts_last_error()
    return out


def _check_cases(hts, cases):
    for (H, W, C), sig, known, kw, own_basis in cases:
        clean, noisy = synth.make_config_image(H, W, C, sig, 500 + C)
        x = torch.from_numpy(noisy).cuda()
        p = hts.params(**kw)
        basis = hts.estimate_basis(x, p) if own_basis else None
        want = hts.denoise(x, sigma=known, p=p, basis=basis).cpu().numpy()
        got = _noalloc(hts, x, known, p, basis).cpu().numpy()
        err = float(np.max(np.abs(got.astype(np.float64) - want)))
        assert err <= MAX_ABS, (H, W, C, kw, own_basis, err)


def test_noalloc_matches_denoise_on_two_calls_in_a_row(hts):
    _check_cases(hts, [
        ((96, 112, 3), 40.0, None, dict(win=21), False),   # colour, sigma and basis estimated
        ((128, 128, 1), 25.0, 25.0, dict(win=21), False),  # gray, known sigma
    ])


def test_noalloc_tensor_core_forms_and_caller_basis(hts):
    # the tensor-core grouping (Eq. 9 flags, rescue list) and filter inside the shared array, and a basis
    # (with eigenvalues) passed by the caller
    _check_cases(hts, [
        ((96, 112, 3), 40.0, None, dict(win=31, precision=1), False),
        ((128, 128, 1), 25.0, None, dict(win=21, precision=1), False),
        ((96, 112, 3), 40.0, 40.0, dict(win=31, precision=2), False),
        ((128, 128, 1), 25.0, None, dict(win=21, precision=2), False),
        ((96, 112, 3), 40.0, None, dict(win=21), True),
        ((128, 128, 1), 25.0, None, dict(win=21, precision=1), True),
    ])


def test_noalloc_rejects_images_beyond_its_scratch(hts):
    lib = hts.load()
    x = torch.zeros((1, 600, 600), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    p = hts.params()
    r = lib.hts_denoise_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), 600, 600, 1,
                                ctypes.c_float(10.0), None, ctypes.byref(p), None)
    assert r == 1
    assert b"static scratch" in lib.hts_last_error()
