"""Python binding of the GB300 Haar-tSVD library (``libhts.so``, C ABI of include/hts.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  There is no CPU
fallback -- if ``libhts.so`` is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HTS_LIBRARY=check selects the check build (libhts_check.so: device-side bounds checks)
LIB_PATH = os.path.join(_HERE, "libhts_check.so" if os.environ.get("HTS_LIBRARY") == "check" else "libhts.so")
_LOCK = threading.Lock()
_LIB = None

HTS_OK = 0
_STATUS = {0: "HTS_OK", 1: "HTS_EINVAL", 2: "HTS_ENOMEM", 3: "HTS_ECUDA", 4: "HTS_ETIMEOUT",
           5: "HTS_EUNSUPPORTED", 6: "HTS_EINTERNAL"}

# every symbol include/hts.h declares
EXPORTS = [
    "hts_params_default", "hts_estimate_basis", "hts_basis_create", "hts_basis_read", "hts_basis_free",
    "hts_basis_save", "hts_basis_load", "hts_estimate_sigma", "hts_denoise", "hts_denoise_host",
    "hts_denoise_batch", "hts_match", "hts_num_refs", "hts_last_stats", "hts_last_error",
    "hts_launch_count", "hts_version", "hts_shutdown", "hts_profile_begin", "hts_profile_end",
    "hts_denoise_noalloc", "hts_last_batch_stats", "hts_tuned_tile",
    "hts_denoise_sigma_map", "hts_denoise_learned", "hts_cnn_num_params", "hts_cnn_channels", "hts_cnn_create",
    "hts_cnn_free", "hts_cnn_get_params", "hts_cnn_set_params", "hts_cnn_log_sigma_map", "hts_cnn_sigma_refs",
    "hts_cnn_zero_grad", "hts_cnn_accumulate_grad", "hts_cnn_take_loss", "hts_cnn_get_grad", "hts_cnn_adam_step",
    "hts_cnn_save", "hts_cnn_load", "hts_cnn_set_window", "hts_cnn_window", "hts_cnn_set_train_fp16",
    "hts_cnn_train_fp16",
    "hts_fcn_num_params", "hts_fcn_channels", "hts_fcn_create", "hts_fcn_free", "hts_fcn_get_params",
    "hts_fcn_set_params", "hts_group_means", "hts_fcn_refine", "hts_fcn_zero_grad", "hts_fcn_accumulate_grad",
    "hts_fcn_take_loss", "hts_fcn_get_grad", "hts_fcn_adam_step", "hts_denoise_ra", "hts_mean_coefs",
    "hts_fcn_group_size", "hts_fault_inject", "hts_denoise_batch_learned",
    "hts_denoise_learned_host",
]


class HtsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("ps", ctypes.c_int), ("K", ctypes.c_int), ("win", ctypes.c_int), ("step", ctypes.c_int),
        ("gamma_gcp", ctypes.c_double), ("beta", ctypes.c_double), ("gamma_rank", ctypes.c_double),
        ("tau_mult", ctypes.c_double), ("adjust_rank", ctypes.c_int), ("mp_correct", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


class SigmaInfo(ctypes.Structure):
    _fields_ = [("sigma_hat", ctypes.c_double), ("sigma_est", ctypes.c_double), ("votes", ctypes.c_int),
                ("nref", ctypes.c_int), ("adjusted", ctypes.c_int), ("uncertain", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("nref", ctypes.c_int), ("match_reranked", ctypes.c_int), ("match_fallback", ctypes.c_int),
                ("filter_redo", ctypes.c_int), ("filter_exact", ctypes.c_int), ("vote_uncertain", ctypes.c_int),
                ("sigma", ctypes.c_double), ("tau", ctypes.c_double), ("filter_fixed", ctypes.c_int),
                ("learned", ctypes.c_int), ("learned_ratio", ctypes.c_double), ("device_error", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("images", ctypes.c_int), ("lanes", ctypes.c_int), ("kernels", ctypes.c_int),
                ("captures", ctypes.c_int), ("updates", ctypes.c_int), ("phased", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("total_ms", ctypes.c_double), ("launches", ctypes.c_int)]


class Image(ctypes.Structure):
    _fields_ = [("noisy", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("C", ctypes.c_int), ("sigma", ctypes.c_float), ("params", ctypes.c_void_p),
                ("sigma_map", ctypes.c_void_p)]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhts.so (raises if it is missing: there is no fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(path):
            raise RuntimeError("libhts.so not built (%s); run paper_2512_23569_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        P, I, F, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
        PP = ctypes.POINTER(Params)
        lib.hts_params_default.argtypes = [PP]
        lib.hts_estimate_basis.argtypes = [P, I, I, I, PP, ctypes.POINTER(P), P]
        lib.hts_basis_create.argtypes = [P, P, I, ctypes.POINTER(P)]
        lib.hts_basis_read.argtypes = [P, P, P, ctypes.POINTER(I)]
        lib.hts_basis_free.argtypes = [P]
        lib.hts_basis_save.argtypes = [P, ctypes.c_char_p]
        lib.hts_basis_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(P)]
        lib.hts_estimate_sigma.argtypes = [P, I, I, I, P, PP, ctypes.POINTER(D), ctypes.POINTER(SigmaInfo), P]
        lib.hts_denoise.argtypes = [P, P, I, I, I, F, P, PP, P]
        lib.hts_denoise_host.argtypes = [P, P, I, I, I, F, P, PP, P]
        lib.hts_denoise_noalloc.argtypes = [P, P, I, I, I, F, P, PP, P]
        lib.hts_denoise_batch.argtypes = [ctypes.POINTER(Image), I, PP, P]
        lib.hts_denoise_batch_learned.argtypes = [ctypes.POINTER(Image), I, P, D, PP, P]
        lib.hts_last_batch_stats.argtypes = [ctypes.POINTER(Stats), I, ctypes.POINTER(BatchInfo), P]
        lib.hts_tuned_tile.argtypes = [I, I, I, PP, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.hts_match.argtypes = [P, I, I, I, PP, P, P, P]
        lib.hts_num_refs.argtypes = [I, I, PP]
        lib.hts_num_refs.restype = I
        lib.hts_last_stats.argtypes = [ctypes.POINTER(Stats), P]
        lib.hts_last_error.restype = ctypes.c_char_p
        lib.hts_launch_count.restype = ctypes.c_uint64
        lib.hts_version.restype = ctypes.c_char_p
        lib.hts_profile_end.argtypes = [ctypes.POINTER(KernelTime), I, ctypes.POINTER(I)]
        lib.hts_denoise_sigma_map.argtypes = [P, P, I, I, I, P, P, PP, P]
        lib.hts_denoise_learned.argtypes = [P, P, I, I, I, P, P, PP, D, P]
        lib.hts_denoise_learned_host.argtypes = [P, P, I, I, I, P, P, PP, D, P]
        lib.hts_cnn_num_params.argtypes = [I]
        lib.hts_cnn_num_params.restype = I
        lib.hts_cnn_channels.argtypes = [P]
        lib.hts_cnn_channels.restype = I
        lib.hts_cnn_create.argtypes = [I, ctypes.c_uint64, ctypes.POINTER(P)]
        lib.hts_cnn_free.argtypes = [P]
        lib.hts_cnn_get_params.argtypes = [P, P]
        lib.hts_cnn_set_params.argtypes = [P, P]
        lib.hts_cnn_log_sigma_map.argtypes = [P, P, I, I, P, P]
        lib.hts_cnn_sigma_refs.argtypes = [P, P, I, I, PP, P, P]
        lib.hts_cnn_zero_grad.argtypes = [P, P]
        lib.hts_cnn_accumulate_grad.argtypes = [P, P, I, I, PP, P, P]
        lib.hts_cnn_take_loss.argtypes = [P, ctypes.POINTER(D), P]
        lib.hts_cnn_get_grad.argtypes = [P, P, P]
        lib.hts_cnn_adam_step.argtypes = [P, F, P]
        lib.hts_cnn_save.argtypes = [P, ctypes.c_char_p]
        lib.hts_cnn_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(P)]
        lib.hts_cnn_set_window.argtypes = [P, I]
        lib.hts_cnn_window.argtypes = [P]
        lib.hts_cnn_window.restype = I
        lib.hts_cnn_set_train_fp16.argtypes = [P, I]
        lib.hts_cnn_train_fp16.argtypes = [P]
        lib.hts_cnn_train_fp16.restype = I
        lib.hts_fcn_num_params.argtypes = [I]
        lib.hts_fcn_num_params.restype = I
        lib.hts_fcn_channels.argtypes = [P]
        lib.hts_fcn_channels.restype = I
        lib.hts_fcn_create.argtypes = [I, I, ctypes.c_uint64, ctypes.POINTER(P)]
        lib.hts_fcn_group_size.argtypes = [P]
        lib.hts_fcn_group_size.restype = I
        lib.hts_fcn_free.argtypes = [P]
        lib.hts_fcn_get_params.argtypes = [P, P]
        lib.hts_fcn_set_params.argtypes = [P, P]
        lib.hts_group_means.argtypes = [P, I, I, I, PP, P, P, P]
        lib.hts_fcn_refine.argtypes = [P, P, P, I, P, P]
        lib.hts_fcn_zero_grad.argtypes = [P, P]
        lib.hts_fcn_accumulate_grad.argtypes = [P, P, P, P, I, P]
        lib.hts_fcn_take_loss.argtypes = [P, ctypes.POINTER(D), P]
        lib.hts_fcn_get_grad.argtypes = [P, P, P]
        lib.hts_fcn_adam_step.argtypes = [P, F, P]
        lib.hts_denoise_ra.argtypes = [P, P, I, I, I, F, P, P, PP, P]
        lib.hts_mean_coefs.argtypes = [P, I, I, P, I, P, P]
        lib.hts_fault_inject.argtypes = [ctypes.c_char_p]
        for name in EXPORTS:  # fail loudly on a library that lacks a declared entry point
            getattr(lib, name)
        _LIB = lib
        return lib


def _check(status: int) -> None:
    if status != HTS_OK:
        msg = load().hts_last_error()
        raise HtsError(status, msg.decode() if msg else "")


def params(**kw) -> Params:
    """Defaults of hts_params_default with keyword overrides."""
    p = Params()
    _check(load().hts_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "gamma_rank" and v is None:
            v = 0.0
        setattr(p, k, v)
    return p


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _chw(t):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError("expected a CUDA float32 tensor")
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3 or not t.is_contiguous():
        raise ValueError("expected a contiguous CHW tensor")
    return t


def num_refs(H: int, W: int, p: Params | None = None) -> int:
    p = p or params()
    return int(load().hts_num_refs(H, W, ctypes.byref(p)))


class Basis:
    """Owns an hts_basis* (global t-SVD basis, Eq. 11)."""

    def __init__(self, handle: ctypes.c_void_p, C: int):
        self._h = handle
        self.C = C

    @property
    def handle(self):
        return self._h

    def read(self):
        """-> (basis complex128 (ns, 2, 8, 8), eigvals (ns, 2, 8) or None)."""
        ns = self.C // 2 + 1
        b = np.zeros((ns, 2, 8, 8, 2))
        e = np.zeros((ns, 2, 8))
        lib = load()
        _check(lib.hts_basis_read(self._h, ctypes.c_void_p(b.ctypes.data), None, None))
        try:
            _check(lib.hts_basis_read(self._h, None, ctypes.c_void_p(e.ctypes.data), None))
        except HtsError:
            e = None
        return b[..., 0] + 1j * b[..., 1], e

    def save(self, path: str) -> None:
        _check(load().hts_basis_save(self._h, path.encode()))

    @staticmethod
    def load_file(path: str) -> "Basis":
        h = ctypes.c_void_p()
        _check(load().hts_basis_load(path.encode(), ctypes.byref(h)))
        C = ctypes.c_int()
        _check(load().hts_basis_read(h, None, None, ctypes.byref(C)))
        return Basis(h, C.value)

    @staticmethod
    def from_array(basis: np.ndarray, eigvals: np.ndarray | None = None) -> "Basis":
        """Basis from complex (ns, 2, 8, 8) (+ optional eigenvalues (ns, 2, 8))."""
        b = np.asarray(basis, dtype=np.complex128)
        ns = b.shape[0]
        C = 1 if ns == 1 else 3
        flat = np.ascontiguousarray(np.stack([b.real, b.imag], axis=-1))
        ev = None if eigvals is None else np.ascontiguousarray(eigvals, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(load().hts_basis_create(ctypes.c_void_p(flat.ctypes.data),
                                       None if ev is None else ctypes.c_void_p(ev.ctypes.data), C, ctypes.byref(h)))
        return Basis(h, C)

    def __del__(self):
        try:
            if self._h and _LIB is not None:
                _LIB.hts_basis_free(self._h)
                self._h = None
        except Exception:
            pass


def estimate_basis(img, p: Params | None = None, stream=None) -> Basis:
    img = _chw(img)
    p = p or params()
    C, H, W = img.shape
    h = ctypes.c_void_p()
    _check(load().hts_estimate_basis(ctypes.c_void_p(img.data_ptr()), H, W, C, ctypes.byref(p), ctypes.byref(h),
                                     _stream(stream)))
    return Basis(h, C)


def estimate_sigma(img, p: Params | None = None, basis: Basis | None = None, stream=None):
    img = _chw(img)
    p = p or params()
    C, H, W = img.shape
    s = ctypes.c_double()
    info = SigmaInfo()
    _check(load().hts_estimate_sigma(ctypes.c_void_p(img.data_ptr()), H, W, C, basis.handle if basis else None,
                                     ctypes.byref(p), ctypes.byref(s), ctypes.byref(info), _stream(stream)))
    return s.value, {f: getattr(info, f) for f, _ in SigmaInfo._fields_}


def match(img, p: Params | None = None, stream=None):
    """Grouping step: -> (idx int32 (N_ref, K) CUDA tensor, green uint8 (N_ref,))."""
    import torch

    img = _chw(img)
    p = p or params()
    C, H, W = img.shape
    n = num_refs(H, W, p)
    idx = torch.empty((n, p.K), dtype=torch.int32, device=img.device)
    green = torch.empty((n,), dtype=torch.uint8, device=img.device)
    _check(load().hts_match(ctypes.c_void_p(img.data_ptr()), H, W, C, ctypes.byref(p),
                            ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(green.data_ptr()), _stream(stream)))
    return idx, green


def denoise(noisy, sigma: float | None = None, basis: Basis | None = None, p: Params | None = None, out=None,
            stream=None):
    """Haar-tSVD of a CUDA CHW float32 tensor; sigma None -> estimated on the device."""
    import torch

    noisy = _chw(noisy)
    p = p or params()
    C, H, W = noisy.shape
    if out is None:
        out = torch.empty_like(noisy)
    s = -1.0 if sigma is None else float(sigma)
    _check(load().hts_denoise(ctypes.c_void_p(noisy.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C, s,
                              basis.handle if basis else None, ctypes.byref(p), _stream(stream)))
    return out


def denoise_noalloc(noisy, sigma: float | None = None, basis: Basis | None = None, p: Params | None = None,
                    out=None, stream=None):
    """hts_denoise_noalloc: like denoise(), with the library's static scratch instead of allocations."""
    import torch

    noisy = _chw(noisy)
    p = p or params()
    C, H, W = noisy.shape
    if out is None:
        out = torch.empty_like(noisy)
    s = -1.0 if sigma is None else float(sigma)
    _check(load().hts_denoise_noalloc(ctypes.c_void_p(noisy.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C,
                                      s, basis.handle if basis else None, ctypes.byref(p), _stream(stream)))
    return out


def denoise_sigma_map(noisy, sigma_ref, basis: Basis | None = None, p: Params | None = None, out=None,
                      stream=None):
    """hts_denoise_sigma_map: one noise level per reference patch (CUDA float32 tensor of N_ref)."""
    import torch

    noisy = _chw(noisy)
    p = p or params()
    C, H, W = noisy.shape
    if not isinstance(sigma_ref, torch.Tensor) or not sigma_ref.is_cuda or sigma_ref.dtype != torch.float32:
        raise TypeError("sigma_ref: expected a CUDA float32 tensor")
    if sigma_ref.numel() != num_refs(H, W, p) or not sigma_ref.is_contiguous():
        raise ValueError("sigma_ref: expected a contiguous tensor of N_ref values")
    if out is None:
        out = torch.empty_like(noisy)
    _check(load().hts_denoise_sigma_map(ctypes.c_void_p(noisy.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C,
                                        ctypes.c_void_p(sigma_ref.data_ptr()), basis.handle if basis else None,
                                        ctypes.byref(p), _stream(stream)))
    return out


class Cnn:
    """Owns an hts_cnn* (learned noise-level map: five 3x3 convolutions, output log sigma)."""

    def __init__(self, C: int = 1, seed: int = 1, handle: ctypes.c_void_p | None = None):
        lib = load()
        if handle is None:
            handle = ctypes.c_void_p()
            _check(lib.hts_cnn_create(C, seed, ctypes.byref(handle)))
        self._h = handle
        self.C = int(lib.hts_cnn_channels(self._h))
        self.nparams = int(lib.hts_cnn_num_params(self.C))

    @property
    def handle(self):
        return self._h

    @property
    def window(self) -> int:
        """Readout window S: a patch's sigma is exp(mean of the map over S x S pixels around its centre)."""
        return int(load().hts_cnn_window(self._h))

    @window.setter
    def window(self, S: int) -> None:
        _check(load().hts_cnn_set_window(self._h, int(S)))

    @property
    def train_fp16(self) -> bool:
        """True: training steps run on the tensor cores (FP16 activations and gradients); False: FP32 kernels."""
        return bool(load().hts_cnn_train_fp16(self._h))

    @train_fp16.setter
    def train_fp16(self, on: bool) -> None:
        _check(load().hts_cnn_set_train_fp16(self._h, 1 if on else 0))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().hts_cnn_get_params(self._h, ctypes.c_void_p(a.ctypes.data)))
        return a

    def set_params(self, theta) -> None:
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.nparams:
            raise ValueError("expected %d parameters" % self.nparams)
        _check(load().hts_cnn_set_params(self._h, ctypes.c_void_p(a.ctypes.data)))

    def log_sigma_map(self, img, stream=None):
        """Full-resolution log(sigma) map (H, W) of a CUDA CHW image."""
        import torch

        img = _chw(img)
        C, H, W = img.shape
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
        _check(load().hts_cnn_log_sigma_map(self._h, ctypes.c_void_p(img.data_ptr()), H, W,
                                            ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def sigma_refs(self, img, p: Params | None = None, stream=None):
        """sigma of every reference patch through the readout window (N_ref,)."""
        import torch

        img = _chw(img)
        p = p or params()
        C, H, W = img.shape
        out = torch.empty((num_refs(H, W, p),), dtype=torch.float32, device=img.device)
        _check(load().hts_cnn_sigma_refs(self._h, ctypes.c_void_p(img.data_ptr()), H, W, ctypes.byref(p),
                                         ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def zero_grad(self, stream=None) -> None:
        _check(load().hts_cnn_zero_grad(self._h, _stream(stream)))

    def accumulate_grad(self, img, target_log_sigma, p: Params | None = None, stream=None) -> None:
        """Adds the gradient of the mean squared log-sigma error over the reference patches."""
        import torch

        img = _chw(img)
        p = p or params()
        C, H, W = img.shape
        t = target_log_sigma
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("target: expected a contiguous CUDA float32 tensor")
        if t.numel() != num_refs(H, W, p):
            raise ValueError("target: expected N_ref values")
        _check(load().hts_cnn_accumulate_grad(self._h, ctypes.c_void_p(img.data_ptr()), H, W, ctypes.byref(p),
                                              ctypes.c_void_p(t.data_ptr()), _stream(stream)))

    def take_loss(self, stream=None) -> float:
        """Sum of the per-image losses accumulated since the last call (synchronises; resets it)."""
        v = ctypes.c_double()
        _check(load().hts_cnn_take_loss(self._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def get_grad(self, stream=None) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().hts_cnn_get_grad(self._h, ctypes.c_void_p(a.ctypes.data), _stream(stream)))
        return a

    def adam_step(self, lr: float, stream=None) -> None:
        _check(load().hts_cnn_adam_step(self._h, float(lr), _stream(stream)))

    def save(self, path: str) -> None:
        _check(load().hts_cnn_save(self._h, path.encode()))

    @staticmethod
    def load_file(path: str) -> "Cnn":
        h = ctypes.c_void_p()
        _check(load().hts_cnn_load(path.encode(), ctypes.byref(h)))
        return Cnn(handle=h)

    def __del__(self):
        try:
            if self._h and _LIB is not None:
                _LIB.hts_cnn_free(self._h)
                self._h = None
        except Exception:
            pass


def denoise_learned(noisy, net: Cnn, p: Params | None = None, basis: Basis | None = None,
                    fallback_factor: float = 2.0, out=None, stream=None):
    """hts_denoise_learned: noise level of each reference patch from the network, checked against the estimate."""
    import torch

    noisy = _chw(noisy)
    p = p or params()
    C, H, W = noisy.shape
    if out is None:
        out = torch.empty_like(noisy)
    _check(load().hts_denoise_learned(ctypes.c_void_p(noisy.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C,
                                      net.handle, basis.handle if basis else None, ctypes.byref(p),
                                      float(fallback_factor), _stream(stream)))
    return out


def denoise_learned_host(noisy: np.ndarray, net: Cnn, p: Params | None = None, basis: Basis | None = None,
                         fallback_factor: float = 2.0, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    """hts_denoise_learned_host: host (numpy) in, host out; the copies happen inside the call."""
    a = noisy if noisy.ndim == 3 else noisy[None]
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous float32 CHW array")
    C, H, W = a.shape
    if out is None:
        out = np.empty_like(a)
    p = p or params()
    _check(load().hts_denoise_learned_host(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(out.ctypes.data), H, W,
                                           C, net.handle, basis.handle if basis else None, ctypes.byref(p),
                                           float(fallback_factor), _stream(stream)))
    return out


def _cuda_f32(t, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("%s: expected a contiguous CUDA float32 tensor" % name)
    return t


class Fcn:
    """Owns an hts_fcn* (the enhancement strategy's network: mean patch -> refined mean patch)."""

    def __init__(self, C: int = 1, K: int = 16, seed: int = 1):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.hts_fcn_create(C, K, seed, ctypes.byref(h)))
        self._h = h
        self.C = C
        self.K = K
        self.nparams = int(lib.hts_fcn_num_params(C))

    @property
    def handle(self):
        return self._h

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().hts_fcn_get_params(self._h, ctypes.c_void_p(a.ctypes.data)))
        return a

    def set_params(self, theta) -> None:
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.nparams:
            raise ValueError("expected %d parameters" % self.nparams)
        _check(load().hts_fcn_set_params(self._h, ctypes.c_void_p(a.ctypes.data)))

    def refine(self, means, sigma, stream=None):
        """Refined mean-patch coordinates (n, C * 64) of coordinates (n, C * 64), noise level of each (n,)."""
        import torch

        _cuda_f32(means, "means")
        _cuda_f32(sigma, "sigma")
        n = means.shape[0]
        out = torch.empty_like(means)
        _check(load().hts_fcn_refine(self._h, ctypes.c_void_p(means.data_ptr()), ctypes.c_void_p(sigma.data_ptr()),
                                     n, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def zero_grad(self, stream=None) -> None:
        _check(load().hts_fcn_zero_grad(self._h, _stream(stream)))

    def accumulate_grad(self, noisy_means, clean_means, sigma, stream=None) -> None:
        for t, nm in ((noisy_means, "noisy_means"), (clean_means, "clean_means"), (sigma, "sigma")):
            _cuda_f32(t, nm)
        _check(load().hts_fcn_accumulate_grad(self._h, ctypes.c_void_p(noisy_means.data_ptr()),
                                              ctypes.c_void_p(clean_means.data_ptr()),
                                              ctypes.c_void_p(sigma.data_ptr()), noisy_means.shape[0],
                                              _stream(stream)))

    def take_loss(self, stream=None) -> float:
        v = ctypes.c_double()
        _check(load().hts_fcn_take_loss(self._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def get_grad(self, stream=None) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().hts_fcn_get_grad(self._h, ctypes.c_void_p(a.ctypes.data), _stream(stream)))
        return a

    def adam_step(self, lr: float, stream=None) -> None:
        _check(load().hts_fcn_adam_step(self._h, float(lr), _stream(stream)))

    def __del__(self):
        try:
            if self._h and _LIB is not None:
                _LIB.hts_fcn_free(self._h)
                self._h = None
        except Exception:
            pass


def group_means(img, idx, p: Params | None = None, stream=None):
    """Mean patch of every group (N_ref, C * 64) for the groups idx (N_ref, K) of hts_match."""
    import torch

    img = _chw(img)
    p = p or params()
    C, H, W = img.shape
    out = torch.empty((idx.shape[0], C * 64), dtype=torch.float32, device=img.device)
    _check(load().hts_group_means(ctypes.c_void_p(img.data_ptr()), H, W, C, ctypes.byref(p),
                                  ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def mean_coefs(x, basis: Basis, inverse: bool = False, stream=None):
    """Image-transform coordinates of patches (n, C * 64) with the basis (inverse: back to pixels)."""
    import torch

    _cuda_f32(x, "x")
    out = torch.empty_like(x)
    _check(load().hts_mean_coefs(ctypes.c_void_p(x.data_ptr()), x.shape[0], basis.C, basis.handle,
                                 1 if inverse else 0, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def denoise_ra(noisy, fcn: Fcn, sigma: float | None = None, p: Params | None = None, basis: Basis | None = None,
               out=None, stream=None):
    """hts_denoise_ra: RA-Haar-tSVD (the groups' first Haar rows from the network's refined mean patches)."""
    import torch

    noisy = _chw(noisy)
    p = p or params(precision=2)
    C, H, W = noisy.shape
    if out is None:
        out = torch.empty_like(noisy)
    s = -1.0 if sigma is None else float(sigma)
    _check(load().hts_denoise_ra(ctypes.c_void_p(noisy.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W, C, s,
                                 fcn.handle, basis.handle if basis else None, ctypes.byref(p), _stream(stream)))
    return out


def denoise_host(noisy: np.ndarray, sigma: float | None = None, basis: Basis | None = None,
                 p: Params | None = None, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    """hts_denoise_host: host (numpy) in, host out; copies happen inside the call."""
    a = noisy if noisy.ndim == 3 else noisy[None]
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous float32 CHW array")
    C, H, W = a.shape
    if out is None:
        out = np.empty_like(a)
    s = -1.0 if sigma is None else float(sigma)
    p = p or params()
    _check(load().hts_denoise_host(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(out.ctypes.data), H, W, C, s,
                                   basis.handle if basis else None, ctypes.byref(p), _stream(stream)))
    return out


def _batch_images(noisy, sigmas, outs, per_image, sigma_maps):
    import torch

    imgs = (Image * max(1, len(noisy)))()
    outs = outs or [torch.empty_like(_chw(x)) for x in noisy]
    for i, (x, s) in enumerate(zip(noisy, sigmas)):
        x = _chw(x)
        C, H, W = x.shape
        pi = per_image[i] if per_image else None
        m = sigma_maps[i] if sigma_maps else None
        if m is not None:
            _cuda_f32(m, "sigma_map")
            if m.numel() != num_refs(H, W, pi or params()):
                raise ValueError("sigma_map: expected N_ref values")
        imgs[i] = Image(x.data_ptr(), outs[i].data_ptr(), H, W, C, -1.0 if s is None else float(s),
                        ctypes.addressof(pi) if pi is not None else None, m.data_ptr() if m is not None else None)
    return imgs, outs


def denoise_batch(noisy: list, sigmas: list, p: Params | None = None, outs: list | None = None, stream=None,
                  per_image: list | None = None, sigma_maps: list | None = None):
    """One graph launch over CUDA CHW tensors; sigma None -> estimated; per_image: Params or None each;
    sigma_maps: None, or per image None or a CUDA float32 tensor of N_ref noise levels."""
    p = p or params()
    imgs, outs = _batch_images(noisy, sigmas, outs, per_image, sigma_maps)  # per_image structs stay alive here
    _check(load().hts_denoise_batch(imgs, len(noisy), ctypes.byref(p), _stream(stream)))
    return outs


def denoise_batch_learned(noisy: list, net: "Cnn", p: Params | None = None, fallback_factor: float = 2.0,
                          outs: list | None = None, stream=None, per_image: list | None = None):
    """hts_denoise_batch_learned: one graph launch in which the network maps every image's noise level."""
    p = p or params()
    imgs, outs = _batch_images(noisy, [None] * len(noisy), outs, per_image, None)
    _check(load().hts_denoise_batch_learned(imgs, len(noisy), net.handle, float(fallback_factor), ctypes.byref(p),
                                            _stream(stream)))
    return outs


def last_batch_stats(n: int, stream=None):
    """-> (per-image counters as in last_stats, schedule dict) of the last denoise_batch on stream."""
    arr = (Stats * max(1, n))()
    info = BatchInfo()
    _check(load().hts_last_batch_stats(arr, n, ctypes.byref(info), _stream(stream)))
    per = [{f: getattr(arr[i], f) for f, _ in Stats._fields_} for i in range(n)]
    return per, {f: getattr(info, f) for f, _ in BatchInfo._fields_}


def tuned_tile(H: int, W: int, C: int, p: Params | None = None):
    """Filter tile shape the autotuner chose for this geometry, (0, 0) = non-local, None = not tuned."""
    p = p or params()
    ty, tx = ctypes.c_int(), ctypes.c_int()
    _check(load().hts_tuned_tile(H, W, C, ctypes.byref(p), ctypes.byref(ty), ctypes.byref(tx)))
    return None if ty.value < 0 else (ty.value, tx.value)


def last_stats(stream=None) -> dict:
    """Counters of the last call on the stream; raises HtsError (HTS_ETIMEOUT / HTS_EINTERNAL) if a kernel of
    that call recorded a failure."""
    st = Stats()
    _check(load().hts_last_stats(ctypes.byref(st), _stream(stream)))
    return {f: getattr(st, f) for f, _ in Stats._fields_}


def fault_inject(spec: str | None) -> None:
    """hts_fault_inject: arm one-shot host-side failures ("alloc:N", "launch:N", "wait:N"; None disarms)."""
    _check(load().hts_fault_inject(None if spec is None else spec.encode()))


def launch_count() -> int:
    return int(load().hts_launch_count())


def version() -> str:
    return load().hts_version().decode()


def profile_begin() -> None:
    """Start bracketing every library kernel launch with CUDA events."""
    _check(load().hts_profile_begin())


def profile_end() -> dict:
    """Stop profiling; -> {kernel name: (total ms, launches)} (synchronises)."""
    arr = (KernelTime * 64)()
    n = ctypes.c_int()
    _check(load().hts_profile_end(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): (arr[i].total_ms, arr[i].launches) for i in range(n.value)}
