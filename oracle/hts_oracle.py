"""FP64 CPU oracle of Haar-tSVD -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs may import this module.  The CUDA library never
calls it and shares no code with it.

The heavy loops live in ``hts_oracle.c`` (plain double-precision C, one step
of the paper at a time).  This module marshals arrays, performs the small
Hermitian eigendecompositions with ``numpy.linalg.eigh`` (a library primitive)
and applies the scalar rules of the noise-level estimate:

* global bases, Eq. 11 over all reference patches: U^(j), V^(j) are the
  eigenvectors of C_row^(j), C_col^(j) (eigenvalues ascending);
* noise floor, Eq. 12: the noise adds ps * N_ref * sigma^2 to every
  eigenvalue of the covariances, so sigma_est^2 = min eigenvalue /
  (ps * N_ref), optionally divided by the Marchenko-Pastur lower-edge factor
  (1 - 1/sqrt(N_ref))^2;
* Eq. 22-23: every group votes "adjust" when the rank position a of
  lambda_hat is <= gamma_rank; a strict majority divides sigma_est by beta;
* tau = tau_mult * sigma * sqrt(2 ln(c K ps^2)).
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hts_oracle.c")
_SO = os.path.join(_HERE, "libhts_oracle.so")
_LOCK = threading.Lock()
_LIB = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -ffp-contract=off) next to its source."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("ps", ctypes.c_int), ("K", ctypes.c_int), ("win", ctypes.c_int), ("step", ctypes.c_int),
        ("gamma_gcp", ctypes.c_double), ("beta", ctypes.c_double), ("gamma_rank", ctypes.c_double),
        ("tau_mult", ctypes.c_double), ("adjust_rank", ctypes.c_int), ("mp_correct", ctypes.c_int),
    ]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i = ctypes.c_int
            d = ctypes.c_double
            lib.htso_grid.argtypes = [i, i, i, P]
            lib.htso_grid.restype = i
            lib.htso_gcp_use_green.argtypes = [P, i, i, i, i, i, d]
            lib.htso_gcp_use_green.restype = i
            lib.htso_patch_distance.argtypes = [P, i, i, i, i, i, i, i, i, i]
            lib.htso_patch_distance.restype = d
            lib.htso_match.argtypes = [P, i, i, i, P, P, P, P]
            lib.htso_match.restype = i
            lib.htso_covariance.argtypes = [P, i, i, i, P, P, P]
            lib.htso_covariance.restype = i
            lib.htso_haar_matrix.argtypes = [i, P]
            lib.htso_haar_matrix.restype = None
            lib.htso_patch_forward.argtypes = [P, i, i, P, P]
            lib.htso_patch_forward.restype = None
            lib.htso_patch_inverse.argtypes = [P, i, i, P, P]
            lib.htso_patch_inverse.restype = d
            lib.htso_group_forward.argtypes = [P, i, i, i, P, P]
            lib.htso_group_forward.restype = None
            lib.htso_group_inverse.argtypes = [P, i, i, i, P, P]
            lib.htso_group_inverse.restype = d
            lib.htso_threshold.argtypes = [P, ctypes.c_long, d]
            lib.htso_threshold.restype = ctypes.c_long
            lib.htso_denoise_groups.argtypes = [P, i, i, i, P, P, d, P, P, P]
            lib.htso_denoise_groups.restype = i
            lib.htso_denoise_groups_taus.argtypes = [P, i, i, i, P, P, P, P, P, P]
            lib.htso_denoise_groups_taus.restype = i
            lib.htso_denoise_groups_ra.argtypes = [P, i, i, i, P, P, d, P, P, P, P, P]
            lib.htso_denoise_groups_ra.restype = i
            lib.htso_group_lambdas.argtypes = [P, i, i, P]
            lib.htso_group_lambdas.restype = None
            lib.htso_rank_of_hat.argtypes = [P, i]
            lib.htso_rank_of_hat.restype = i
            lib.htso_rank_votes.argtypes = [P, i, i, i, P, P, P]
            lib.htso_rank_votes.restype = i
            lib.htso_num_threads.argtypes = []
            lib.htso_num_threads.restype = i
            lib.htso_set_num_threads.argtypes = [i]
            lib.htso_set_num_threads.restype = None
            lib.htso_num_slices.argtypes = [i]
            lib.htso_num_slices.restype = i
            _LIB = lib
    return _LIB


@dataclass
class Params:
    """Method parameters (Sec. IV-A defaults, K/window per workload)."""

    ps: int = 8
    K: int = 16
    win: int = 21
    step: int = 4
    gamma_gcp: float = 1.2      # Eq. 9
    beta: float = 1.2           # Eq. 23
    gamma_rank: float | None = None  # Eq. 23; None -> 13 K / 32
    tau_mult: float = 1.0
    adjust_rank: int = 1
    mp_correct: int = 1

    def gamma_rank_value(self) -> float:
        return 13.0 * self.K / 32.0 if self.gamma_rank is None else float(self.gamma_rank)

    def c_struct(self) -> _Params:
        return _Params(self.ps, self.K, self.win, self.step, self.gamma_gcp, self.beta,
                       self.gamma_rank_value(), self.tau_mult, self.adjust_rank, self.mp_correct)


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _img(img: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(img, dtype=np.float32)
    if a.ndim == 2:
        a = a[None]
    if a.ndim != 3 or a.shape[0] not in (1, 3):
        raise ValueError("image must be CHW with C in {1, 3}")
    return a


def num_threads() -> int:
    return int(_lib().htso_num_threads())


def set_num_threads(n: int) -> None:
    _lib().htso_set_num_threads(int(n))


def num_slices(C: int) -> int:
    return C // 2 + 1


def grid(n: int, ps: int, step: int) -> np.ndarray:
    lib = _lib()
    cnt = lib.htso_grid(n, ps, step, None)
    out = np.zeros(max(cnt, 1), dtype=np.int32)
    lib.htso_grid(n, ps, step, _ptr(out))
    return out[:cnt]


def num_refs(H: int, W: int, p: Params) -> int:
    return len(grid(H, p.ps, p.step)) * len(grid(W, p.ps, p.step))


def gcp_use_green(img: np.ndarray, y: int, x: int, p: Params) -> int:
    a = _img(img)
    return int(_lib().htso_gcp_use_green(_ptr(a), a.shape[1], a.shape[2], y, x, p.ps, p.gamma_gcp))


def patch_distance(img, use_green, yr, xr, yc, xc, p: Params) -> float:
    a = _img(img)
    C, H, W = a.shape
    return float(_lib().htso_patch_distance(_ptr(a), H, W, C, int(use_green), p.ps, yr, xr, yc, xc))


def match(img: np.ndarray, p: Params):
    """Alg. 1 grouping.  Returns (idx[nref, K] int32, green[nref] uint8, dist[nref, K])."""
    a = _img(img)
    C, H, W = a.shape
    nref = num_refs(H, W, p)
    idx = np.zeros((nref, p.K), dtype=np.int32)
    green = np.zeros(nref, dtype=np.uint8)
    dist = np.zeros((nref, p.K), dtype=np.float64)
    ps = p.c_struct()
    r = _lib().htso_match(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(idx), _ptr(green), _ptr(dist))
    if r < 0:
        raise ValueError("search window holds fewer than K positions")
    return idx, green, dist


def covariance(img: np.ndarray, p: Params):
    """Eq. 11 global covariances: (C_row, C_col) as complex (ns, ps, ps), and N_ref."""
    a = _img(img)
    C, H, W = a.shape
    ns = num_slices(C)
    crow = np.zeros((ns, p.ps, p.ps, 2))
    ccol = np.zeros((ns, p.ps, p.ps, 2))
    ps = p.c_struct()
    nref = _lib().htso_covariance(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(crow), _ptr(ccol))
    if nref < 0:
        raise ValueError("image smaller than a patch")
    return crow[..., 0] + 1j * crow[..., 1], ccol[..., 0] + 1j * ccol[..., 1], nref


def basis_from_covariance(crow: np.ndarray, ccol: np.ndarray):
    """Eigenvectors of the covariances (numpy eigh, ascending eigenvalues).

    Returns basis (ns, 2, ps, ps) complex128 with basis[j, 0] = U^(j),
    basis[j, 1] = V^(j) (columns are eigenvectors) and eigvals (ns, 2, ps).
    Slice 0 is real and is decomposed as a real symmetric matrix.
    """
    ns, ps, _ = crow.shape
    basis = np.zeros((ns, 2, ps, ps), dtype=np.complex128)
    ev = np.zeros((ns, 2, ps))
    for j in range(ns):
        for m, Cm in enumerate((crow[j], ccol[j])):
            if j == 0:
                w, v = np.linalg.eigh(Cm.real)
            else:
                w, v = np.linalg.eigh(Cm)
            basis[j, m] = v
            ev[j, m] = w
    return basis, ev


def estimate_basis(img: np.ndarray, p: Params):
    """Globally-learned bases (Eq. 11 over all reference patches)."""
    crow, ccol, nref = covariance(img, p)
    basis, ev = basis_from_covariance(crow, ccol)
    return basis, ev, nref


def basis_to_flat(basis: np.ndarray) -> np.ndarray:
    """complex (ns, 2, ps, ps) -> float64 (ns, 2, ps, ps, 2) [re, im] (C layout)."""
    b = np.asarray(basis, dtype=np.complex128)
    return np.ascontiguousarray(np.stack([b.real, b.imag], axis=-1))


def sigma_floor(eigvals: np.ndarray, nref: int, p: Params) -> float:
    """Eq. 12 noise floor: sigma_est^2 = lambda_min / (ps * N_ref) [/ MP edge]."""
    lam = float(np.min(eigvals))
    s2 = max(lam, 0.0) / (p.ps * nref)
    if p.mp_correct:
        s2 = s2 / (1.0 - 1.0 / math.sqrt(nref)) ** 2
    return math.sqrt(s2)


def rank_votes(img: np.ndarray, p: Params, idx: np.ndarray):
    """Eq. 22-23 per-group rank positions; returns (votes, a[nref])."""
    a = _img(img)
    C, H, W = a.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    ranks = np.zeros(idx.shape[0], dtype=np.int32)
    ps = p.c_struct()
    votes = _lib().htso_rank_votes(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(idx), _ptr(ranks))
    return int(votes), ranks


def estimate_sigma(img: np.ndarray, p: Params, eigvals=None, nref=None, idx=None) -> dict:
    """Noise level: covariance floor (Eq. 12) adjusted by the rank vote (Eq. 23)."""
    a = _img(img)
    if eigvals is None:
        _, eigvals, nref = estimate_basis(a, p)
    s_est = sigma_floor(eigvals, nref, p)
    votes = 0
    if p.adjust_rank:
        if idx is None:
            idx, _, _ = match(a, p)
        votes, _ = rank_votes(a, p, idx)
    adjust = bool(p.adjust_rank) and 2 * votes > nref
    s_hat = s_est / p.beta if adjust else s_est
    return {"sigma_hat": s_hat, "sigma_est": s_est, "votes": votes, "nref": nref, "adjust": adjust}


def tau(sigma: float, C: int, p: Params) -> float:
    """Universal threshold of Sec. IV-A: sigma sqrt(2 ln(c K ps^2)) (x tau_mult)."""
    return p.tau_mult * sigma * math.sqrt(2.0 * math.log(C * p.K * p.ps * p.ps))


def haar_matrix(K: int) -> np.ndarray:
    Hm = np.zeros((K, K))
    _lib().htso_haar_matrix(K, _ptr(Hm))
    return Hm


def patch_forward(P: np.ndarray, basis: np.ndarray) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    C, ps, _ = P.shape
    S = np.zeros((C, ps, ps, 2))
    bf = basis_to_flat(basis)
    _lib().htso_patch_forward(_ptr(P), C, ps, _ptr(bf), _ptr(S))
    return S[..., 0] + 1j * S[..., 1]


def patch_inverse(S: np.ndarray, basis: np.ndarray):
    S = np.asarray(S, dtype=np.complex128)
    C, ps, _ = S.shape
    Sf = np.ascontiguousarray(np.stack([S.real, S.imag], axis=-1))
    P = np.zeros((C, ps, ps))
    bf = basis_to_flat(basis)
    im = _lib().htso_patch_inverse(_ptr(Sf), C, ps, _ptr(bf), _ptr(P))
    return P, float(im)


def group_forward(G: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """Eq. 19 for one group G (K, C, ps, ps) -> complex coefficients (K, C, ps, ps)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    K, C, ps, _ = G.shape
    S = np.zeros((K, C, ps, ps, 2))
    bf = basis_to_flat(basis)
    _lib().htso_group_forward(_ptr(G), K, C, ps, _ptr(bf), _ptr(S))
    return S[..., 0] + 1j * S[..., 1]


def group_inverse(S: np.ndarray, basis: np.ndarray):
    """Eq. 21 for one group; returns (G (K, C, ps, ps), max imaginary residue)."""
    S = np.asarray(S, dtype=np.complex128)
    K, C, ps, _ = S.shape
    Sf = np.ascontiguousarray(np.stack([S.real, S.imag], axis=-1))
    G = np.zeros((K, C, ps, ps))
    bf = basis_to_flat(basis)
    im = _lib().htso_group_inverse(_ptr(Sf), K, C, ps, _ptr(bf), _ptr(G))
    return G, float(im)


def threshold(S: np.ndarray, tau_value: float):
    """Eq. 20 on a complex coefficient array (copy); returns (S_thr, kept)."""
    S = np.asarray(S, dtype=np.complex128)
    Sf = np.ascontiguousarray(np.stack([S.real, S.imag], axis=-1))
    kept = _lib().htso_threshold(_ptr(Sf), S.size, float(tau_value))
    return Sf[..., 0] + 1j * Sf[..., 1], int(kept)


def group_lambdas(G: np.ndarray) -> np.ndarray:
    """Eigenvalues lambda_m of circ(G) circ(G)^T for G (K, D)."""
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(G.shape[0], -1)
    lam = np.zeros(G.shape[0])
    _lib().htso_group_lambdas(_ptr(G), G.shape[0], G.shape[1], _ptr(lam))
    return lam


def rank_of_hat(lam: np.ndarray) -> int:
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    return int(_lib().htso_rank_of_hat(_ptr(lam), lam.shape[0]))


def denoise_groups(noisy: np.ndarray, p: Params, basis: np.ndarray, tau_value, idx: np.ndarray):
    """Alg. 1 steps 2-3 for given groups; returns (out CHW float64, stats dict).

    tau_value: one threshold, or an array with one threshold per reference patch."""
    a = _img(noisy)
    C, H, W = a.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros((C, H, W))
    st = np.zeros(3)
    bf = basis_to_flat(basis)
    ps = p.c_struct()
    if np.ndim(tau_value) == 0:
        r = _lib().htso_denoise_groups(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(bf), float(tau_value),
                                       _ptr(idx), _ptr(out), _ptr(st))
    else:
        taus = np.ascontiguousarray(tau_value, dtype=np.float64).reshape(-1)
        if taus.shape[0] != idx.shape[0]:
            raise ValueError("one threshold per reference patch")
        r = _lib().htso_denoise_groups_taus(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(bf), _ptr(taus),
                                            _ptr(idx), _ptr(out), _ptr(st))
    if r < 0:
        raise ValueError("bad input")
    return out, {"kept": int(st[0]), "groups": int(st[1]), "max_imag": float(st[2])}


def denoise(noisy: np.ndarray, p: Params, sigma=None, basis: np.ndarray | None = None):
    """Whole Haar-tSVD: grouping, (basis), (sigma), filtering, aggregation.

    sigma None -> estimated (Eq. 12 floor + Eq. 23 vote); a number -> one
    noise level; an array with one value per reference patch -> a threshold
    per group (spatially varying noise).  basis None -> globally-learned from
    the noisy image (Eq. 11).  Returns (out, info).
    """
    a = _img(noisy)
    C = a.shape[0]
    info: dict = {}
    ev = nref = None
    if basis is None or sigma is None:
        b, ev, nref = estimate_basis(a, p)
        if basis is None:
            basis = b
    idx, green, _ = match(a, p)
    if sigma is None:
        s = estimate_sigma(a, p, eigvals=ev, nref=nref, idx=idx)
        info.update(s)
        sigma = s["sigma_hat"]
    if np.ndim(sigma) == 0:
        t = tau(sigma, C, p)
    else:
        t = np.array([tau(float(sv), C, p) for sv in np.asarray(sigma, dtype=np.float64).reshape(-1)])
    out, st = denoise_groups(a, p, basis, t, idx)
    info.update(st)
    info.update({"sigma": sigma, "tau": t, "idx": idx, "green": green, "basis": basis})
    return out, info


# ------------------------------------------------ enhancement strategy (RA)

def group_means(img: np.ndarray, idx: np.ndarray, ps: int = 8) -> np.ndarray:
    """Mean patch of every group (Eq. 24 up to the sqrt(K) factor): (N_ref, C * ps * ps) FP64, entry
    t * ps^2 + u * ps + v = mean over the group's members of pixel (u, v) of channel t."""
    a = _img(img).astype(np.float64)
    C, H, W = a.shape
    idx = np.asarray(idx)
    out = np.zeros((idx.shape[0], C, ps, ps))
    for k in range(idx.shape[1]):
        y, x = idx[:, k] // W, idx[:, k] % W
        for u in range(ps):
            for v in range(ps):
                out[:, :, u, v] += a[:, y + u, x + v].T
    return (out / idx.shape[1]).reshape(idx.shape[0], -1)


def canonical_basis(basis: np.ndarray) -> np.ndarray:
    """Every eigenvector (column i of U^(j), V^(j)) multiplied by the conjugate phase of its largest-
    magnitude entry (ties to the lower row), which becomes real positive: eigenvectors are defined up to
    that phase (the filter is invariant to it), the network's coordinates need one fixed choice."""
    b = np.array(basis, dtype=np.complex128)
    for j in range(b.shape[0]):
        for m in range(2):
            for i in range(b.shape[3]):
                col = b[j, m, :, i]
                a = int(np.argmax(np.abs(col) ** 2))  # first maximum
                b[j, m, :, i] = col * np.conj(col[a]) / abs(col[a])
    return b


def mean_coefs(means: np.ndarray, basis: np.ndarray, C: int, ps: int = 8) -> np.ndarray:
    """Mean patches (n, C ps^2) in the image's transform (Eq. 19 without the Haar factor, one patch) with
    the canonical basis: the real vector [S^(1), sqrt(2) Re S^(2), sqrt(2) Im S^(2)] (C = 3; slice 3 is the
    conjugate of slice 2, so the vector has the patch's norm) or S^(1) (C = 1), each slice row-major."""
    m = np.ascontiguousarray(means, dtype=np.float64)
    n2 = ps * ps
    bf = basis_to_flat(canonical_basis(basis))
    S = np.zeros(2 * C * n2)
    out = np.zeros((m.shape[0], C * n2))
    for r in range(m.shape[0]):
        _lib().htso_patch_forward(_ptr(np.ascontiguousarray(m[r])), C, ps, _ptr(bf), _ptr(S))
        out[r, :n2] = S[0:2 * n2:2]
        if C == 3:
            out[r, n2:2 * n2] = math.sqrt(2.0) * S[2 * n2:4 * n2:2]
            out[r, 2 * n2:] = math.sqrt(2.0) * S[2 * n2 + 1:4 * n2:2]
    return out


def coefs_to_patch(coefs: np.ndarray, basis: np.ndarray, C: int, ps: int = 8) -> np.ndarray:
    """Inverse of mean_coefs (Eq. 21 without the Haar factor): (n, C ps^2) pixel-domain patches."""
    c = np.asarray(coefs, dtype=np.float64)
    n2 = ps * ps
    bf = basis_to_flat(canonical_basis(basis))
    out = np.zeros((c.shape[0], C * n2))
    P = np.zeros(C * n2)
    for r in range(c.shape[0]):
        S = np.zeros(2 * C * n2)
        S[0:2 * n2:2] = c[r, :n2]
        if C == 3:
            re, im = c[r, n2:2 * n2] / math.sqrt(2.0), c[r, 2 * n2:] / math.sqrt(2.0)
            S[2 * n2:4 * n2:2], S[2 * n2 + 1:4 * n2:2] = re, im
            S[4 * n2::2], S[4 * n2 + 1::2] = re, -im
        _lib().htso_patch_inverse(_ptr(S), C, ps, _ptr(bf), _ptr(P))
        out[r] = P
    return out


def denoise_groups_ra(noisy: np.ndarray, p: Params, basis: np.ndarray, tau_value, idx: np.ndarray,
                      mean_est: np.ndarray):
    """Alg. 1 steps 2-3 with the enhancement strategy: the first Haar row of every group replaced by
    sqrt(K) times the transform of mean_est[r] (N_ref, C * ps * ps) and kept whole (Eq. 24-25)."""
    a = _img(noisy)
    C, H, W = a.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    me = np.ascontiguousarray(mean_est, dtype=np.float64)
    if me.shape != (idx.shape[0], C * p.ps * p.ps):
        raise ValueError("one refined mean patch per reference patch")
    out = np.zeros((C, H, W))
    st = np.zeros(3)
    bf = basis_to_flat(basis)
    ps = p.c_struct()
    taus = None
    if np.ndim(tau_value) != 0:
        taus = np.ascontiguousarray(tau_value, dtype=np.float64).reshape(-1)
    r = _lib().htso_denoise_groups_ra(_ptr(a), H, W, C, ctypes.byref(ps), _ptr(bf),
                                      0.0 if taus is not None else float(tau_value),
                                      None if taus is None else _ptr(taus), _ptr(idx), _ptr(me), _ptr(out), _ptr(st))
    if r < 0:
        raise ValueError("bad input")
    return out, {"kept": int(st[0]), "groups": int(st[1]), "max_imag": float(st[2])}


def denoise_ra(noisy: np.ndarray, p: Params, theta: np.ndarray, sigma=None, basis: np.ndarray | None = None):
    """RA-Haar-tSVD: grouping, basis, noise level as denoise(); the mean patch of every group, in the
    image's transform (mean_coefs), refined by the fully connected network (fcn_oracle.refine, Eq. 25),
    replaces the group's first Haar row."""
    from . import fcn_oracle

    a = _img(noisy)
    C = a.shape[0]
    info: dict = {}
    ev = nref = None
    if basis is None or sigma is None:
        b, ev, nref = estimate_basis(a, p)
        if basis is None:
            basis = b
    idx, green, _ = match(a, p)
    if sigma is None:
        s = estimate_sigma(a, p, eigvals=ev, nref=nref, idx=idx)
        info.update(s)
        sigma = s["sigma_hat"]
    means = group_means(a, idx, p.ps)
    coefs = mean_coefs(means, basis, C, p.ps)
    est = coefs_to_patch(fcn_oracle.refine(theta, coefs, float(sigma), C, p.K), basis, C, p.ps)
    out, st = denoise_groups_ra(a, p, basis, tau(float(sigma), C, p), idx, est)
    info.update(st)
    info.update({"sigma": sigma, "idx": idx, "basis": basis, "means": means, "coefs": coefs, "mean_est": est})
    return out, info
