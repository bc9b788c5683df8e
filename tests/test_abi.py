"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, and rejects bad arguments before any device work."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23569_gb300 import build, hts

    build.build()
    return hts.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "hts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hts_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_four_method_calls():
    names = _declared()
    for n in ("hts_estimate_basis", "hts_estimate_sigma", "hts_denoise", "hts_denoise_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2512_23569_gb300 import hts

    names = _declared()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hts.EXPORTS)


def test_params_default(lib):
    from paper_2512_23569_gb300 import hts

    p = hts.params()
    assert (p.ps, p.K, p.win, p.step) == (8, 16, 21, 4)
    assert p.gamma_gcp == 1.2 and p.beta == 1.2 and p.tau_mult == 1.0


def test_num_refs_matches_oracle_grid(lib):
    from oracle import hts_oracle as o
    from paper_2512_23569_gb300 import hts

    for H, W, step in [(128, 128, 4), (77, 93, 4), (8, 8, 4), (33, 20, 3), (512, 384, 8)]:
        p = hts.params(step=step, K=2, win=3)
        want = len(o.grid(H, 8, step)) * len(o.grid(W, 8, step))
        assert hts.num_refs(H, W, p) == want


@pytest.mark.parametrize("kw,status", [
    (dict(ps=7), 5), (dict(K=3), 1), (dict(K=64), 1), (dict(win=20), 1), (dict(win=1), 1), (dict(win=65), 5),
    (dict(step=0), 1), (dict(step=9), 1), (dict(beta=0.0), 1), (dict(gamma_gcp=-1.0), 1), (dict(tau_mult=-1.0), 1),
])
def test_bad_params_rejected_before_device_work(lib, kw, status):
    from paper_2512_23569_gb300 import hts

    p = hts.params(**kw)
    fake = ctypes.c_void_p(0x1000)
    r = lib.hts_denoise(fake, ctypes.c_void_p(0x2000), 64, 64, 3, ctypes.c_float(10.0), None, ctypes.byref(p), None)
    assert r == status
    assert lib.hts_last_error()


def test_bad_geometry_rejected(lib):
    from paper_2512_23569_gb300 import hts

    p = hts.params()
    f = ctypes.c_void_p(0x1000)
    o = ctypes.c_void_p(0x2000)
    assert lib.hts_denoise(f, o, 7, 64, 1, ctypes.c_float(1.0), None, ctypes.byref(p), None) == 1  # H < ps
    assert lib.hts_denoise(f, o, 64, 64, 2, ctypes.c_float(1.0), None, ctypes.byref(p), None) == 1  # C
    assert lib.hts_denoise(f, f, 64, 64, 1, ctypes.c_float(1.0), None, ctypes.byref(p), None) == 1  # alias
    assert lib.hts_denoise(f, o, 64, 64, 1, ctypes.c_float(float("nan")), None, ctypes.byref(p), None) == 1
    # a 10x10 image with K = 16 has 3 x 3 candidate positions at most
    assert lib.hts_denoise(f, o, 10, 10, 1, ctypes.c_float(1.0), None, ctypes.byref(p), None) == 1
    assert b"fewer than K" in lib.hts_last_error()
    assert lib.hts_denoise(None, o, 64, 64, 1, ctypes.c_float(1.0), None, ctypes.byref(p), None) == 1
    assert lib.hts_denoise_batch(None, 3, ctypes.byref(p), None) == 1
    assert lib.hts_denoise_batch(None, 0, ctypes.byref(p), None) == 0


def test_basis_create_validates_on_host(lib):
    import numpy as np

    from paper_2512_23569_gb300 import hts

    h = ctypes.c_void_p()
    bad = np.zeros((1, 2, 8, 8, 2))
    assert lib.hts_basis_create(ctypes.c_void_p(bad.ctypes.data), None, 1, ctypes.byref(h)) == 1
    assert b"unitary" in lib.hts_last_error()
    eye = np.zeros((1, 2, 8, 8, 2))
    eye[0, :, :, :, 0] = np.eye(8)
    eye[0, 0, 0, 0, 1] = 0.5  # imaginary part in slice 0
    assert lib.hts_basis_create(ctypes.c_void_p(eye.ctypes.data), None, 1, ctypes.byref(h)) == 1


def test_product_path_has_no_oracle_and_no_fallback():
    pkg = os.path.join(ROOT, "paper_2512_23569_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("the oracle", "").lower() or f == "synth.py", f


def test_fault_spec_parsing(lib):
    # host-side fault injection: well-formed specs arm (and "" disarms); malformed ones are refused
    for spec in (b"alloc:1", b"launch:3,wait:2", b"alloc:2|launch:1", b"", None):
        assert lib.hts_fault_inject(spec) == 0, spec
    for spec in (b"alloc", b"alloc:0", b"alloc:-1", b"boom:1", b"launch:x", b"wait:1,", b"wait:99999999999999"):
        st = lib.hts_fault_inject(spec)
        if spec == b"wait:1,":  # a trailing separator is allowed
            assert st == 0
        else:
            assert st == 1, spec  # HTS_EINVAL
    assert lib.hts_fault_inject(None) == 0
