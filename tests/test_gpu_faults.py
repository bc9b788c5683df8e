"""Failure paths on the GPU, made on the host (hts_fault_inject): nothing faults, traps or hangs.

* an allocation that fails returns HTS_ENOMEM and the next call works;
* a launch reported as failed returns HTS_ECUDA and the next call works;
* a bounded mbarrier wait of the tensor-core matcher that runs out (it waits, a few thousand polls, on a
  barrier nothing arrives on, before any MMA is issued) is reported as HTS_ETIMEOUT by the calls that read
  the device state back, every reference keeps a valid group (its own position), and the next call gives
  the same result as a call that never failed.
"""

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HTS_ENOMEM, HTS_ECUDA, HTS_ETIMEOUT = 2, 3, 4


@pytest.fixture(scope="module")
def hts():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2512_23569_gb300 import build, hts as h

    build.build()
    h.load()
    yield h
    h.fault_inject(None)


@pytest.fixture(autouse=True)
def disarm(hts):
    hts.fault_inject(None)
    yield
    hts.fault_inject(None)


def _image(C=3, H=96, W=112, sigma=30.0, seed=71):
    _, noisy = synth.make_config_image(H, W, C, sigma, seed)
    return noisy, torch.from_numpy(noisy).cuda()


def test_injected_allocation_failure(hts):
    _, x = _image()
    p = hts.params(win=15)
    want = hts.denoise(x, sigma=None, p=p)
    s = torch.cuda.Stream()  # a new stream: its workspace is allocated by the next call
    hts.fault_inject("alloc:1")
    with pytest.raises(hts.HtsError) as e:
        hts.denoise(x, sigma=None, p=p, stream=s)
    assert e.value.status == HTS_ENOMEM
    got = hts.denoise(x, sigma=None, p=p, stream=s)
    s.synchronize()
    assert torch.equal(got, want)


@pytest.mark.parametrize("nth", [1, 3])
def test_injected_launch_failure(hts, nth):
    _, x = _image()
    p = hts.params(win=15)
    want = hts.denoise(x, sigma=None, p=p)
    hts.fault_inject("launch:%d" % nth)
    with pytest.raises(hts.HtsError) as e:
        hts.denoise(x, sigma=None, p=p)
    assert e.value.status == HTS_ECUDA
    got = hts.denoise(x, sigma=None, p=p)
    assert torch.equal(got, want)


@pytest.mark.parametrize("C", [1, 3])
def test_matcher_wait_runs_out(hts, C):
    noisy, x = _image(C=C)
    p = hts.params(win=21 if C == 1 else 31, precision=1)
    want = hts.denoise(x, sigma=None, p=p)
    hts.last_stats()
    # grouping alone: the wait gives up, every reference keeps only itself
    hts.fault_inject("wait:1")
    idx, _ = hts.match(x, p)
    with pytest.raises(hts.HtsError) as e:
        hts.last_stats()
    assert e.value.status == HTS_ETIMEOUT
    idx = idx.cpu().numpy()
    H, W = noisy.shape[1:]
    ys = list(range(0, H - 8 + 1, 4)) + ([H - 8] if (H - 8) % 4 else [])
    xs = list(range(0, W - 8 + 1, 4)) + ([W - 8] if (W - 8) % 4 else [])
    refs = np.array([y * W + xx for y in ys for xx in xs])
    np.testing.assert_array_equal(idx, np.repeat(refs[:, None], p.K, axis=1))
    # the whole method: the call itself is asynchronous, the state read back reports the failure
    hts.fault_inject("wait:1")
    out = hts.denoise(x, sigma=None, p=p)
    with pytest.raises(hts.HtsError) as e:
        hts.last_stats()
    assert e.value.status == HTS_ETIMEOUT
    assert out.shape == x.shape  # the output is invalid, but every read stayed inside the image
    # synchronising calls report it themselves
    hts.fault_inject("wait:1")
    with pytest.raises(hts.HtsError) as e:
        hts.denoise_host(noisy, sigma=None, p=p)
    assert e.value.status == HTS_ETIMEOUT
    hts.fault_inject("wait:1")
    with pytest.raises(hts.HtsError) as e:
        hts.estimate_sigma(x, p)
    assert e.value.status == HTS_ETIMEOUT
    # and the library carries on
    got = hts.denoise(x, sigma=None, p=p)
    st = hts.last_stats()
    assert st["device_error"] == 0
    assert torch.equal(got, want)
