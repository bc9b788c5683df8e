"""The check build (libhts_check.so, every kernel compiled with -DHTS_CHECK): its device-side bounds checks
stay silent on the library's forms, image shapes and group sizes, and the results equal the normal build's.

Run in a child process (the binding loads one library per process, chosen by HTS_LIBRARY)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
from paper_2512_23569_gb300 import build, hts, synth
build.build(check=True)
lib = hts.load()
assert "libhts_check" in lib._name, lib._name
cases = [((96, 112, 3), dict(win=21)), ((128, 128, 1), dict(win=21)), ((96, 112, 3), dict(win=31, precision=1)),
         ((130, 150, 1), dict(win=21, precision=1, K=8)), ((96, 112, 3), dict(win=31, precision=2, K=32)),
         ((200, 260, 3), dict(win=31, precision=1))]
out = {}
for i, ((H, W, C), kw) in enumerate(cases):
    clean, noisy = synth.make_config_image(H, W, C, 30.0, 900 + i)
    x = torch.from_numpy(noisy).cuda()
    y = hts.denoise(x, p=hts.params(**kw)).cpu().numpy()
    st = hts.last_stats()
    assert st["device_error"] == 0, (i, st)
    out["c%d" % i] = y
net = hts.Cnn(3, seed=2)
clean, noisy = synth.make_config_image(96, 112, 3, 30.0, 950)
x = torch.from_numpy(noisy).cuda()
y = hts.denoise_learned(x, net, hts.params(win=31, precision=1), fallback_factor=50.0).cpu().numpy()
assert hts.last_stats()["device_error"] == 0
assert np.all(np.isfinite(net.log_sigma_map(x).cpu().numpy()))
out["learned"] = y
np.savez(OUTFILE, **out)
print("check build clean")
"""


def test_check_build_is_silent_and_equal(tmp_path):
    import numpy as np

    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    res = {}
    for variant in ("check", "normal"):
        outfile = str(tmp_path / (variant + ".npz"))
        env = dict(os.environ, HTS_LIBRARY=variant)
        code = CHILD.replace("OUTFILE", repr(outfile))
        if variant == "normal":
            code = code.replace("build.build(check=True)", "build.build()").replace(
                'assert "libhts_check" in lib._name, lib._name', "")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=900)
        assert r.returncode == 0, r.stdout + r.stderr
        res[variant] = np.load(outfile)
    for k in res["check"].files:
        np.testing.assert_array_equal(res["check"][k], res["normal"][k])
