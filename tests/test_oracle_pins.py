"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route (explicit block-circulant matrices of Eq. 2-3, the
circulant Gram matrix of Eq. 13-15, hand-written Haar matrices of Eq. 7-8,
brute force on integer-valued images, closed forms, statistics of pure noise).
"""

import math
import os

import numpy as np
import pytest

from paper_2512_23569_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_haar_golden():
    r = 1.0 / math.sqrt(2.0)
    vals = {"r": r, "h": 0.5, "0": 0.0}
    mats = {}
    lines = [l.split() for l in open(os.path.join(GOLDEN, "haar_eq7_eq8.txt")) if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        K = int(lines[i][0])
        rows = []
        for j in range(K):
            row = []
            for tok in lines[i + 1 + j]:
                neg = tok.startswith("-")
                v = vals[tok.lstrip("-")]
                row.append(-v if neg else v)
            rows.append(row)
        mats[K] = np.array(rows)
        i += K + 1
    return mats


# ---------------------------------------------------------------- Eq. 7-8


def test_haar_matches_hand_written_eq7_eq8(oracle):
    for K, M in _read_haar_golden().items():
        np.testing.assert_allclose(oracle.haar_matrix(K), M, rtol=0, atol=1e-15)


@pytest.mark.parametrize("K", [2, 4, 8, 16, 32])
def test_haar_orthonormal_first_row_constant(oracle, K):
    Hm = oracle.haar_matrix(K)
    np.testing.assert_allclose(Hm @ Hm.T, np.eye(K), atol=1e-14)
    # Eq. 18: the first Haar row is u_max = 1/sqrt(K) (1, ..., 1)
    np.testing.assert_allclose(Hm[0], np.full(K, 1.0 / math.sqrt(K)), atol=1e-15)
    # rows of Eq. 8 beyond the first sum to zero (detail rows)
    np.testing.assert_allclose(Hm[1:].sum(axis=1), 0.0, atol=1e-14)


# ---------------------------------------------------- Eq. 2-5: t-product


def _bcirc(T):
    """Eq. 2: block circulant matrix of a tensor T (n1 x n2 x n3)."""
    n1, n2, n3 = T.shape
    B = np.zeros((n1 * n3, n2 * n3))
    for i in range(n3):
        for j in range(n3):
            B[i * n1:(i + 1) * n1, j * n2:(j + 1) * n2] = T[:, :, (i - j) % n3]
    return B


def _random_orthogonal_tensor(rng, ps, C):
    """Real ps x ps x C tensor whose FFT slices (mode 3) are unitary."""
    slices = []
    for j in range(C // 2 + 1):
        if j == 0 or (C % 2 == 0 and j == C // 2):
            q, _ = np.linalg.qr(rng.standard_normal((ps, ps)))
            slices.append(q.astype(np.complex128))
        else:
            q, _ = np.linalg.qr(rng.standard_normal((ps, ps)) + 1j * rng.standard_normal((ps, ps)))
            slices.append(q)
    full = [slices[j] if j < len(slices) else np.conj(slices[C - j]) for j in range(C)]
    Fh = np.stack(full, axis=2)
    T = np.fft.ifft(Fh, axis=2)
    assert np.max(np.abs(T.imag)) < 1e-12
    return T.real, slices


@pytest.mark.parametrize("C", [1, 3])
def test_patch_projection_is_t_product(oracle, C):
    """Eq. 3-5 and 19: the oracle's Fourier-domain projection U^H P V equals
    the t-product U^T * P * V computed with explicit bcirc matrices."""
    rng = np.random.default_rng(3 + C)
    ps = 8
    Ut, Us = _random_orthogonal_tensor(rng, ps, C)
    Vt, Vs = _random_orthogonal_tensor(rng, ps, C)
    basis = np.stack([np.stack([Us[j], Vs[j]]) for j in range(len(Us))])
    P = rng.uniform(0, 255, size=(C, ps, ps))
    S_four = oracle.patch_forward(P, basis)  # unitary mode-3 DFT domain
    # unitary -> FFT scaling, back to the real coefficient tensor
    S_real = np.fft.ifft(np.moveaxis(S_four, 0, 2) * math.sqrt(C), axis=2)
    assert np.max(np.abs(S_real.imag)) < 1e-9
    Pt = np.moveaxis(P, 0, 2)
    Bs = _bcirc(Ut).T @ _bcirc(Pt) @ _bcirc(Vt)  # bcirc(U^T) = bcirc(U)^T
    S_ref = np.stack([Bs[0:ps, 0:ps] if False else Bs[i * ps:(i + 1) * ps, 0:ps] for i in range(C)], axis=2)
    np.testing.assert_allclose(S_real.real, S_ref, rtol=0, atol=1e-9 * np.abs(S_ref).max())
    # and the inverse brings the patch back exactly (Eq. 21 without threshold)
    P2, im = oracle.patch_inverse(S_four, basis)
    np.testing.assert_allclose(P2, P, atol=1e-10)
    assert im < 1e-10


# ---------------------------------- Eq. 11 and 2: covariance vs bcirc


@pytest.mark.parametrize("C", [1, 3])
def test_covariance_spectrum_equals_bcirc_gram(oracle, C):
    """Eq. 11 in the Fourier domain is block-circulant PCA: the spectrum of
    sum_i bcirc(P_i) bcirc(P_i)^T equals c times the union of the spectra of
    C_row^(j) over all c slices (slice c-j = conjugate of slice j)."""
    img = synth.clean_image(16, 20, C, seed=11) + np.random.default_rng(5).normal(0, 9, size=(C, 16, 20)).astype(np.float32)
    img = img.astype(np.float32)
    p = oracle.Params(K=2, win=3, step=4)
    crow, ccol, nref = oracle.covariance(img, p)
    ys, xs = oracle.grid(16, 8, 4), oracle.grid(20, 8, 4)
    assert nref == len(ys) * len(xs) == 3 * 4
    G_row = np.zeros((8 * C, 8 * C))
    G_col = np.zeros((8 * C, 8 * C))
    for y in ys:
        for x in xs:
            Pt = np.moveaxis(img[:, y:y + 8, x:x + 8].astype(np.float64), 0, 2)
            B = _bcirc(Pt)
            G_row += B @ B.T
            G_col += B.T @ B
    ns = crow.shape[0]
    full_r = [crow[j] if j < ns else np.conj(crow[C - j]) for j in range(C)]
    full_c = [ccol[j] if j < ns else np.conj(ccol[C - j]) for j in range(C)]
    ev_r = np.sort(np.concatenate([np.linalg.eigvalsh(M) for M in full_r])) * C
    ev_c = np.sort(np.concatenate([np.linalg.eigvalsh(M) for M in full_c])) * C
    np.testing.assert_allclose(ev_r, np.sort(np.linalg.eigvalsh(G_row)), rtol=1e-10, atol=1e-6)
    np.testing.assert_allclose(ev_c, np.sort(np.linalg.eigvalsh(G_col)), rtol=1e-10, atol=1e-6)
    # Hermitian by construction, trace = total energy of the reference patches
    energy = sum(float(np.sum(img[:, y:y + 8, x:x + 8].astype(np.float64) ** 2)) for y in ys for x in xs)
    assert abs(sum(np.trace(M).real for M in full_r) - energy) < 1e-9 * energy


def test_global_basis_diagonalises_and_is_unitary(oracle):
    img = synth.make_config_image(40, 48, 3, 20.0, seed=21)[1]
    p = oracle.Params(K=4, win=7)
    crow, ccol, _ = oracle.covariance(img, p)
    basis, ev = oracle.basis_from_covariance(crow, ccol)
    for j in range(basis.shape[0]):
        for m, Cm in enumerate((crow[j], ccol[j])):
            U = basis[j, m]
            np.testing.assert_allclose(U.conj().T @ U, np.eye(8), atol=1e-12)
            D = U.conj().T @ Cm @ U
            off = D - np.diag(np.diag(D))
            assert np.max(np.abs(off)) < 1e-9 * np.max(np.abs(Cm))
            np.testing.assert_allclose(np.diag(D).real, ev[j, m], rtol=1e-9)
    # slice 0 is real
    assert np.max(np.abs(basis[0].imag)) == 0.0


# ---------------------------------------- Eq. 13-18, 22: circulant group


def _circ_group(G):
    """Eq. 13: circ(G) in R^{K x K*D}, row i is the cyclic shift of patches."""
    K, D = G.shape
    M = np.zeros((K, K * D))
    for i in range(K):
        for j in range(K):
            M[i, j * D:(j + 1) * D] = G[(j - i) % K]  # row i: p_{(j - i) mod K}
    return M


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_lambdas_are_eigenvalues_of_circulant_gram(oracle, K):
    rng = np.random.default_rng(K)
    D = 3 * 4
    G = rng.normal(100, 20, size=(K, D))
    lam = oracle.group_lambdas(G)
    M = _circ_group(G)
    gram = M @ M.T
    # Eq. 15: the Gram matrix is circulant
    for i in range(K):
        np.testing.assert_allclose(gram[i], np.roll(gram[0], i), rtol=1e-12)
    ev = np.linalg.eigvalsh(gram)
    np.testing.assert_allclose(np.sort(lam), ev, rtol=1e-9, atol=1e-6)
    # Eq. 18: lambda_max = ||sum p||^2 with eigenvector 1/sqrt(K)
    rsum = G.sum(axis=0)
    assert abs(lam[0] - rsum @ rsum) < 1e-9 * lam[0]
    u = np.full(K, 1 / math.sqrt(K))
    np.testing.assert_allclose(gram @ u, lam[0] * u, rtol=1e-10)
    assert abs(lam[0] - ev[-1]) < 1e-9 * ev[-1]  # dominant for positive patches
    # Eq. 22: lambda_hat = ||sum (-1)^i p_i||^2 with the alternating eigenvector
    alt = ((-1.0) ** np.arange(1, K + 1))
    s = alt @ G
    assert abs(lam[K // 2] - s @ s) < 1e-9 * max(1.0, lam[0])
    uh = alt / math.sqrt(K)
    np.testing.assert_allclose(gram @ uh, lam[K // 2] * uh, rtol=1e-8, atol=1e-6 * lam[0])


def test_rank_of_lambda_hat(oracle):
    # hand-made spectra (K = 8, hat at m = 4); a = 1 + #{m != 4 : lam_m < lam_4}
    assert oracle.rank_of_hat(np.array([10, 5, 3, 1, 0.5, 1, 3, 5.0])) == 1
    assert oracle.rank_of_hat(np.array([10, 5, 3, 1, 4.0, 1, 3, 5.0])) == 5
    assert oracle.rank_of_hat(np.array([10, 5, 3, 1, 99, 1, 3, 5.0])) == 8
    # ties rank lowest
    assert oracle.rank_of_hat(np.array([10, 2, 2, 2, 2, 2, 2, 2.0])) == 1
    # identical patches: every lambda but lambda_0 vanishes -> a = 1 ("adjust")
    K = 16
    G = np.tile(np.random.default_rng(1).normal(size=24), (K, 1))
    assert oracle.rank_of_hat(oracle.group_lambdas(G)) == 1
    # alternating patches: lambda_hat is the largest non-DC eigenvalue -> a = K
    q = np.random.default_rng(2).normal(size=24)
    G = np.stack([(-1) ** k * q for k in range(K)]) + 0.01 * np.random.default_rng(3).normal(size=(K, 24))
    assert oracle.rank_of_hat(oracle.group_lambdas(G)) == K


# ------------------------------------------------- Eq. 9 and grouping


def _brute_match(img, p, use_green_fn=None):
    C, H, W = img.shape
    ys, xs = np.arange(0, H - 7, p.step), np.arange(0, W - 7, p.step)
    if ys[-1] != H - 8:
        ys = np.append(ys, H - 8)
    if xs[-1] != W - 8:
        xs = np.append(xs, W - 8)
    R = (p.win - 1) // 2
    out = []
    for yr in ys:
        for xr in xs:
            if C == 1:
                plane = img[0].astype(np.float64)
            else:
                ug = use_green_fn(yr, xr)
                plane = img[1].astype(np.float64) if ug else img.astype(np.float64).sum(axis=0)
            ref = plane[yr:yr + 8, xr:xr + 8]
            cands = []
            for y in range(max(0, yr - R), min(H - 8, yr + R) + 1):
                for x in range(max(0, xr - R), min(W - 8, xr + R) + 1):
                    if (y, x) == (yr, xr):
                        continue
                    d = float(np.sum((ref - plane[y:y + 8, x:x + 8]) ** 2))
                    cands.append((d, y * W + x))
            cands.sort()
            out.append([yr * W + xr] + [c[1] for c in cands[:p.K - 1]])
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("H,W,C,win,K", [(16, 16, 1, 5, 4), (19, 23, 1, 7, 8), (17, 21, 3, 5, 4), (24, 20, 3, 9, 16)])
def test_match_equals_brute_force_on_integer_images(oracle, H, W, C, win, K):
    rng = np.random.default_rng(H * W + C)
    img = rng.integers(0, 40, size=(C, H, W)).astype(np.float32)  # exact integer distances
    p = oracle.Params(K=K, win=win, step=4)
    idx, green, _ = oracle.match(img, p)
    ref = _brute_match(img, p, lambda y, x: oracle.gcp_use_green(img, y, x, p))
    np.testing.assert_array_equal(idx, ref)


def test_match_flat_image_ties_go_to_lowest_index(oracle):
    img = np.full((1, 20, 20), 7.0, dtype=np.float32)
    p = oracle.Params(K=8, win=5, step=4)
    idx, _, dist = oracle.match(img, p)
    assert np.all(dist == 0.0)
    ref = _brute_match(img, p)
    np.testing.assert_array_equal(idx, ref)
    # the reference at (4, 4): window rows 2..6, cols 2..6 in raster order
    r = 1 * len(oracle.grid(20, 8, 4)) + 1
    W = 20
    expect = [4 * W + 4] + [y * W + x for y in range(2, 7) for x in range(2, 7) if (y, x) != (4, 4)][:7]
    assert list(idx[r]) == expect


def test_gcp_switch_both_sides_of_boundary(oracle):
    """Eq. 9 with gamma = 1.2: green wins iff ||G|| >= max(||R||, ||B||) / 1.2."""
    p = oracle.Params()
    for ratio, expect in [(1.2 * (1 - 1e-6), 1), (1.2 * (1 + 1e-6), 0), (1.0, 1), (2.0, 0)]:
        img = np.zeros((3, 8, 8), dtype=np.float32)
        img[1] = 50.0
        img[0] = np.float32(50.0 * ratio)
        img[2] = 10.0
        assert oracle.gcp_use_green(img, 0, 0, p) == expect, ratio
        img[0], img[2] = img[2].copy(), img[0].copy()  # B plays R's role
        assert oracle.gcp_use_green(img, 0, 0, p) == expect, ratio


def test_average_plane_orders_like_channel_mean(oracle):
    """The channel sum stands in for Eq. 9's average: 9x the distance, same order."""
    rng = np.random.default_rng(8)
    img = rng.integers(0, 30, size=(3, 12, 12)).astype(np.float32)
    p = oracle.Params()
    d_sum = oracle.patch_distance(img, 0, 0, 0, 3, 4, p)
    avg = img.astype(np.float64).mean(axis=0)
    d_avg = float(np.sum((avg[0:8, 0:8] - avg[3:11, 4:12]) ** 2))
    assert abs(d_sum - 9 * d_avg) < 1e-9 * d_sum


# ------------------------------------------- Eq. 19-21 and Alg. 1


@pytest.mark.parametrize("H,W,C,K,win", [(32, 32, 1, 8, 9), (29, 37, 3, 4, 7), (24, 24, 3, 16, 11)])
def test_perfect_reconstruction_at_zero_threshold(oracle, H, W, C, K, win):
    """tau = 0 keeps every coefficient; orthonormal transforms + averaging
    return the input exactly (Eq. 19-21, Alg. 1 step 3)."""
    img = synth.make_config_image(H, W, C, 25.0, seed=H + W)[1]
    p = oracle.Params(K=K, win=win)
    basis, _, _ = oracle.estimate_basis(img, p)
    idx, _, _ = oracle.match(img, p)
    out, st = oracle.denoise_groups(img, p, basis, 0.0, idx)
    np.testing.assert_allclose(out, img.astype(np.float64), rtol=0, atol=1e-10)
    assert st["kept"] == idx.shape[0] * K * C * 64
    assert st["max_imag"] < 1e-10


def test_group_transform_parseval_and_inverse(oracle):
    rng = np.random.default_rng(4)
    for C in (1, 3):
        img = synth.make_config_image(32, 32, C, 30.0, seed=9)[1]
        p = oracle.Params(K=16, win=11)
        basis, _, _ = oracle.estimate_basis(img, p)
        G = rng.normal(120, 40, size=(16, C, 8, 8))
        S = oracle.group_forward(G, basis)
        assert abs(np.sum(np.abs(S) ** 2) - np.sum(G ** 2)) < 1e-10 * np.sum(G ** 2)
        G2, im = oracle.group_inverse(S, basis)
        np.testing.assert_allclose(G2, G, atol=1e-9)
        # the first Haar row is sqrt(K) x the projected mean patch (Eq. 24)
        Sm = oracle.patch_forward(G.mean(axis=0), basis)
        np.testing.assert_allclose(S[0], 4.0 * Sm, atol=1e-9)


def test_identical_patches_survive_any_small_threshold(oracle):
    """A group of K identical patches has only first-row Haar coefficients
    (Eq. 18, 24); thresholding the rest changes nothing."""
    img = synth.clean_image(24, 24, 3, seed=5)
    p = oracle.Params(K=8, win=5)
    basis, _, _ = oracle.estimate_basis(img + 1.0, p)
    P = img[:, 3:11, 5:13].astype(np.float64)
    G = np.stack([P] * 8)
    S = oracle.group_forward(G, basis)
    assert np.max(np.abs(S[1:])) < 1e-9
    St, kept = oracle.threshold(S, 1e-6)
    G2, _ = oracle.group_inverse(St, basis)
    np.testing.assert_allclose(G2, G, atol=1e-9)


def test_threshold_rule(oracle):
    S = np.array([3.0 + 0j, -3.0, 2.9999, 3.0 + 1e-300j, 2.0 + 2.0j, 2.0 + 2.3j, 0.0])
    St, kept = oracle.threshold(S, 3.0)
    # |s| >= tau kept (Eq. 20); modulus for complex entries
    np.testing.assert_array_equal(St != 0, [True, True, False, True, False, True, False])
    assert kept == 4


def test_tau_constants_match_hand_values(oracle):
    for line in open(os.path.join(GOLDEN, "tau_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        c, K, ratio = line.split()
        p = oracle.Params(K=int(K))
        assert abs(oracle.tau(1.0, int(c), p) - float(ratio)) < 6e-5


# ------------------------------------------------- Eq. 12: noise level


@pytest.mark.parametrize("C,sigma", [(1, 5.0), (1, 25.0), (3, 10.0), (3, 50.0), (3, 75.0)])
def test_sigma_recovered_on_pure_noise(oracle, C, sigma):
    H = W = 256
    flat = np.full((C, H, W), 128.0, dtype=np.float32)
    noisy = synth.awgn(flat, sigma, seed=int(sigma) + C)
    p = oracle.Params(K=16, win=21 if C == 1 else 31)
    s = oracle.estimate_sigma(noisy, p)
    assert abs(s["sigma_est"] / sigma - 1) < 0.02, s
    assert not s["adjust"], s  # pure noise: lambda_hat is not small, no adjustment
    assert 0.3 < s["votes"] / s["nref"] < 0.5


def test_sigma_floor_on_structured_image(oracle):
    clean, noisy = synth.make_config_image(256, 256, 3, 50.0, seed=2001)
    p = oracle.Params(K=16, win=31)
    s = oracle.estimate_sigma(noisy, p)
    assert abs(s["sigma_hat"] / 50.0 - 1) < 0.03, s


def test_denoise_improves_psnr(oracle):
    clean, noisy = synth.make_config_image(128, 128, 1, 25.0, seed=1000)
    p = oracle.Params(K=16, win=21)
    out, info = oracle.denoise(noisy, p, sigma=25.0)
    assert synth.psnr(out, clean) > synth.psnr(noisy, clean) + 7.0


def test_per_reference_thresholds_reduce_to_one(oracle):
    # a threshold per group equal everywhere is the single-threshold filter; a higher threshold on one
    # group only changes the pixels that group covers
    _, noisy = synth.make_config_image(40, 48, 1, 20.0, 91)
    p = oracle.Params(win=11)
    a, _ = oracle.denoise(noisy, p, sigma=20.0)
    n = oracle.num_refs(40, 48, p)
    b, _ = oracle.denoise(noisy, p, sigma=np.full(n, 20.0))
    np.testing.assert_array_equal(a, b)
    sig = np.full(n, 20.0)
    sig[0] = 200.0
    c, info = oracle.denoise(noisy, p, sigma=sig)
    changed = np.argwhere(np.abs(c - a) > 0)
    assert len(changed) > 0


# ------------------------------------------ Eq. 23: the vote's decision


def _vote_image_and_groups(nref_target, voters, K=16):
    """A gray 8 x W image, left half flat 40, right half flat 200, whose reference grid has nref_target
    positions, with hand-made groups (Eq. 22-23 only reads the members the groups name):
    - a "voting" group repeats one flat patch K times: lambda_0 = K^2 |p|^2 and lambda_m = 0 for m != 0,
      so lambda_hat = lambda_{K/2} = 0 has rank position a = 1 (no lambda below it);
    - a "non-voting" group alternates the 40-patch and the 200-patch: lambda_{K/2} = K^2 |d|^2 with
      d = (40 - 200) / 2 per pixel, above every lambda_m (m != 0, K/2) = 0 and below lambda_0 = K^2 |c|^2,
      c = 120 per pixel, so a = K - 1.
    The first `voters` groups vote."""
    W = 8 + 4 * (nref_target - 1)
    img = np.full((1, 8, W), 40.0, dtype=np.float32)
    img[:, :, W // 2:] = 200.0
    left, right = 0, W - 8  # raster indices of two flat patches (row 0)
    idx = np.empty((nref_target, K), dtype=np.int32)
    for r in range(nref_target):
        if r < voters:
            idx[r] = left
        else:
            idx[r] = [left if k % 2 == 0 else right for k in range(K)]
    return img, idx


@pytest.mark.parametrize("nref,voters,adjust", [
    (16, 9, True),    # strict majority of an even count
    (16, 8, False),   # exact tie: no adjustment
    (16, 7, False),   # minority
    (15, 8, True),    # strict majority of an odd count
    (15, 7, False),
    (16, 16, True),   # unanimous
    (16, 0, False),
])
def test_eq23_strict_majority_divides_sigma_by_beta(oracle, nref, voters, adjust):
    K = 16
    img, idx = _vote_image_and_groups(nref, voters, K)
    p = oracle.Params(K=K, win=21, beta=1.5, mp_correct=0)
    assert oracle.num_refs(img.shape[1], img.shape[2], p) == nref
    # rank positions of the two hand-made group kinds (Eq. 22): 1 and K - 1, against gamma_K = 13 K / 32
    votes, ranks = oracle.rank_votes(img, p, idx)
    assert votes == voters
    np.testing.assert_array_equal(ranks, [1] * voters + [K - 1] * (nref - voters))
    # Eq. 12 floor from given eigenvalues (no Marchenko-Pastur edge): sigma_est^2 = lambda_min / (ps N_ref)
    sigma0 = 10.0
    eig = np.array([8.0 * nref * sigma0 ** 2, 5e6, 7e6])
    s = oracle.estimate_sigma(img, p, eigvals=eig, nref=nref, idx=idx)
    assert s["votes"] == voters and s["nref"] == nref
    assert s["sigma_est"] == pytest.approx(sigma0, rel=1e-15)
    assert s["adjust"] is adjust
    # Eq. 23: divided by beta (not multiplied, not the variance divided) on a strict majority only
    want = sigma0 / 1.5 if adjust else sigma0
    assert s["sigma_hat"] == pytest.approx(want, rel=1e-15)


def test_eq23_vote_off_keeps_the_floor(oracle):
    img, idx = _vote_image_and_groups(16, 16)
    p = oracle.Params(K=16, win=21, beta=1.5, mp_correct=0, adjust_rank=0)
    eig = np.array([8.0 * 16 * 9.0])
    s = oracle.estimate_sigma(img, p, eigvals=eig, nref=16, idx=idx)
    assert not s["adjust"] and s["sigma_hat"] == pytest.approx(3.0, rel=1e-15)
