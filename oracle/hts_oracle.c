/*
 * hts_oracle.c -- plain, slow FP64 CPU oracle of Haar-tSVD
 * ("Image Denoising Using Global and Local Circulant Representation",
 *  Kong, Yang, Zhang; arXiv 2512.23569).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference the CUDA
 * path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is computed in double precision from the float32 input, in the
 * order the paper states the method: grouping (Eq. 9, Alg. 1 step 1), the
 * forward transform (Eq. 19, evaluated slice-wise in the Fourier domain of
 * mode 3 as Eq. 4-5 and Eq. 11 prescribe), hard thresholding (Eq. 20), the
 * inverse transform (Eq. 21) and plain averaging (Alg. 1 step 3).  The Haar
 * matrix is built explicitly from Eq. 7-8 and applied as a matrix; there is
 * no fast transform, blocking or fusion here.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   - reference grid: {0, s, 2s, ...} plus the last position n-ps;
 *   - search window: the square of side `win` centred on the reference
 *     top-left corner, clipped (not shifted) at the borders;
 *   - group order: slot 0 is the reference itself, then the K-1 nearest other
 *     candidates in ascending (distance, raster index y*W+x);
 *   - Eq. 9 uses the reference patch's channel norms; "avg" is replaced by the
 *     channel sum R+G+B, which orders candidates identically;
 *   - thresholding acts on the Fourier-domain coefficients: a real
 *     coefficient is kept iff |s| >= tau, a complex one iff its modulus is;
 *   - tau = tau_mult * sigma * sqrt(2 ln(c K ps^2))  (natural log);
 *   - aggregation is a uniform average, the output is not clipped.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps a*b+c as two roundings on every host).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int ps;            /* patch side */
    int K;             /* patches per group (power of two) */
    int win;           /* search window side (odd) */
    int step;          /* reference grid step */
    double gamma_gcp;  /* Eq. 9 weight of the green channel */
    double beta;       /* Eq. 23 divisor */
    double gamma_rank; /* Eq. 23 rank threshold */
    double tau_mult;   /* multiplier on the universal threshold */
    int adjust_rank;   /* apply Eq. 23 */
    int mp_correct;    /* Marchenko-Pastur edge correction of sigma_est */
} htso_params;

typedef struct { double re, im; } cplx;

static cplx c_make(double re, double im) { cplx r; r.re = re; r.im = im; return r; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_mul(cplx a, cplx b) { return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cplx c_conj(cplx a) { return c_make(a.re, -a.im); }
static cplx c_scale(cplx a, double s) { return c_make(a.re * s, a.im * s); }

static const double PI = 3.14159265358979323846;

/* omega^e with omega = exp(-2 pi i / n); the exponent is reduced mod n first.
 * Quarter turns are returned exactly (1, -i, -1, i), so that e.g. the m = K/2
 * root is exactly (-1)^k as in Eq. 22. */
static cplx unit_root(long e, int n)
{
    long r = e % n;
    if (r < 0) r += n;
    if ((4 * r) % n == 0) {
        switch ((4 * r) / n) {
        case 0: return c_make(1.0, 0.0);
        case 1: return c_make(0.0, -1.0);
        case 2: return c_make(-1.0, 0.0);
        default: return c_make(0.0, 1.0);
        }
    }
    double ang = -2.0 * PI * (double)r / (double)n;
    return c_make(cos(ang), sin(ang));
}

/* ------------------------------------------------------------------ grid */

/* Reference positions along one axis: 0, s, 2s, ... <= n-ps, plus n-ps.
 * Returns the count; writes positions to out if non-NULL. */
int htso_grid(int n, int ps, int step, int *out)
{
    if (n < ps || step < 1) return 0;
    int cnt = 0, last = -1;
    for (int p = 0; p <= n - ps; p += step) {
        if (out) out[cnt] = p;
        cnt++;
        last = p;
    }
    if (last != n - ps) {
        if (out) out[cnt] = n - ps;
        cnt++;
    }
    return cnt;
}

/* Number of distinct Fourier slices stored in a basis: slice c-j is the
 * complex conjugate of slice j for real input. */
int htso_num_slices(int C) { return C / 2 + 1; }

/* ------------------------------------------------------- Eq. 9 grouping */

/* Eq. 9: the green channel decides when ||P^G|| >= max(||P^R||/g, ||P^B||/g),
 * evaluated on the reference patch.  Returns 1 for "green", 0 for "average". */
int htso_gcp_use_green(const float *img, int H, int W, int y, int x, int ps, double gamma)
{
    double n2[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; c++)
        for (int u = 0; u < ps; u++)
            for (int v = 0; v < ps; v++) {
                double a = (double)img[(size_t)c * H * W + (size_t)(y + u) * W + (x + v)];
                n2[c] = n2[c] + a * a;
            }
    double nR = sqrt(n2[0]), nG = sqrt(n2[1]), nB = sqrt(n2[2]);
    double lim = fmax(nR / gamma, nB / gamma);
    return nG >= lim ? 1 : 0;
}

/* Value of the matching plane at (y, x): the image for c = 1; for c = 3 the
 * green channel or the channel sum (R+G)+B, per the reference's Eq. 9 flag. */
static double plane_value(const float *img, int H, int W, int C, int use_green, int y, int x)
{
    size_t o = (size_t)y * W + x, hw = (size_t)H * W;
    if (C == 1) return (double)img[o];
    if (use_green) return (double)img[hw + o];
    return ((double)img[o] + (double)img[hw + o]) + (double)img[2 * hw + o];
}

/* Squared Euclidean distance between the patches at (yr,xr) and (yc,xc) on
 * the matching plane (Eq. 9 squared: same order).  Row-major accumulation. */
double htso_patch_distance(const float *img, int H, int W, int C, int use_green, int ps,
                           int yr, int xr, int yc, int xc)
{
    double acc = 0.0;
    for (int u = 0; u < ps; u++)
        for (int v = 0; v < ps; v++) {
            double d = plane_value(img, H, W, C, use_green, yr + u, xr + v) -
                       plane_value(img, H, W, C, use_green, yc + u, xc + v);
            acc = acc + d * d;
        }
    return acc;
}

typedef struct { double d; int32_t idx; } cand_t;

static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* Alg. 1 step 1 for every reference patch.  idx_out: nref x K raster indices
 * y*W+x of patch top-left corners (slot 0 = reference); green_out (optional):
 * the Eq. 9 flag per reference (always 1 for c = 1); dist_out (optional):
 * nref x K distances.  Returns nref, or -1 when some window holds fewer than
 * K positions. */
int htso_match(const float *img, int H, int W, int C, const htso_params *p,
               int32_t *idx_out, uint8_t *green_out, double *dist_out)
{
    int ps = p->ps, K = p->K, R = (p->win - 1) / 2;
    int ny = htso_grid(H, ps, p->step, NULL), nx = htso_grid(W, ps, p->step, NULL);
    if (ny == 0 || nx == 0) return -1;
    int *ys = (int *)malloc(sizeof(int) * ny), *xs = (int *)malloc(sizeof(int) * nx);
    htso_grid(H, ps, p->step, ys);
    htso_grid(W, ps, p->step, xs);
    int nref = ny * nx;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int r = 0; r < nref; r++) {
        int yr = ys[r / nx], xr = xs[r % nx];
        int use_green = (C == 3) ? htso_gcp_use_green(img, H, W, yr, xr, ps, p->gamma_gcp) : 1;
        int y0 = yr - R < 0 ? 0 : yr - R, y1 = yr + R > H - ps ? H - ps : yr + R;
        int x0 = xr - R < 0 ? 0 : xr - R, x1 = xr + R > W - ps ? W - ps : xr + R;
        int n = 0;
        cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * (size_t)(y1 - y0 + 1) * (x1 - x0 + 1));
        for (int y = y0; y <= y1; y++)
            for (int x = x0; x <= x1; x++) {
                if (y == yr && x == xr) continue;
                cand[n].d = htso_patch_distance(img, H, W, C, use_green, ps, yr, xr, y, x);
                cand[n].idx = (int32_t)(y * W + x);
                n++;
            }
        if (n < K - 1) {
            bad = 1;
        } else {
            qsort(cand, (size_t)n, sizeof(cand_t), cand_cmp);
            idx_out[(size_t)r * K] = (int32_t)(yr * W + xr);
            if (dist_out) dist_out[(size_t)r * K] = 0.0;
            for (int s = 1; s < K; s++) {
                idx_out[(size_t)r * K + s] = cand[s - 1].idx;
                if (dist_out) dist_out[(size_t)r * K + s] = cand[s - 1].d;
            }
        }
        if (green_out) green_out[r] = (uint8_t)use_green;
        free(cand);
    }
    free(ys);
    free(xs);
    return bad ? -1 : nref;
}

/* ------------------------------------------- Eq. 4-5: DFT along mode 3 */

/* Unitary DFT of one ps x ps x C patch along mode 3:
 * Phat[j] = (1/sqrt C) sum_t P[t] omega^(j t), omega = exp(-2 pi i / C).
 * P: C x ps x ps real; Phat: C x ps x ps complex. */
static void dft_mode3(const double *P, int C, int ps, cplx *Phat)
{
    int n = ps * ps;
    double s = 1.0 / sqrt((double)C);
    for (int j = 0; j < C; j++)
        for (int e = 0; e < n; e++) {
            cplx acc = c_make(0.0, 0.0);
            for (int t = 0; t < C; t++)
                acc = c_add(acc, c_mul(c_make(P[t * n + e], 0.0), unit_root((long)j * t, C)));
            Phat[j * n + e] = c_scale(acc, s);
        }
}

/* Inverse of dft_mode3; returns the real part and stores the largest
 * imaginary magnitude seen in *max_im. */
static void idft_mode3(const cplx *Phat, int C, int ps, double *P, double *max_im)
{
    int n = ps * ps;
    double s = 1.0 / sqrt((double)C);
    for (int t = 0; t < C; t++)
        for (int e = 0; e < n; e++) {
            cplx acc = c_make(0.0, 0.0);
            for (int j = 0; j < C; j++)
                acc = c_add(acc, c_mul(Phat[j * n + e], unit_root(-(long)j * t, C)));
            acc = c_scale(acc, s);
            P[t * n + e] = acc.re;
            if (max_im && fabs(acc.im) > *max_im) *max_im = fabs(acc.im);
        }
}

/* Basis accessors.  A basis holds, for each stored slice j < C/2+1, the pair
 * (U^(j), V^(j)) as ps x ps complex matrices, element [a][i] = row a of
 * eigenvector i.  Layout: basis[((j*2 + m)*ps*ps + a*ps + i)*2 + {0:re,1:im}],
 * m = 0 for U, 1 for V.  Slices j >= C/2+1 are conjugates of slice C-j. */
static cplx basis_at(const double *basis, int C, int ps, int j, int m, int a, int i)
{
    int ns = htso_num_slices(C);
    int jj = j < ns ? j : C - j;
    size_t o = (((size_t)(jj * 2 + m) * ps * ps) + (size_t)a * ps + i) * 2;
    cplx z = c_make(basis[o], basis[o + 1]);
    return j < ns ? z : c_conj(z);
}

/* ------------------------------------------- Eq. 11: global covariances */

/* Globally-learned bases (Eq. 11 over all reference patches):
 * C_row^(j) = sum_i Phat_i^(j) Phat_i^(j)^H and C_col^(j) = sum_i Phat_i^(j)^H Phat_i^(j)
 * for the stored slices j < C/2+1.  crow/ccol: ns x ps x ps complex (re,im).
 * Accumulated sequentially in reference order.  Returns the number of
 * reference patches, or -1. */
int htso_covariance(const float *img, int H, int W, int C, const htso_params *p,
                    double *crow, double *ccol)
{
    int ps = p->ps, n = ps * ps, ns = htso_num_slices(C);
    int ny = htso_grid(H, ps, p->step, NULL), nx = htso_grid(W, ps, p->step, NULL);
    if (ny == 0 || nx == 0) return -1;
    int *ys = (int *)malloc(sizeof(int) * ny), *xs = (int *)malloc(sizeof(int) * nx);
    htso_grid(H, ps, p->step, ys);
    htso_grid(W, ps, p->step, xs);
    cplx *Cr = (cplx *)calloc((size_t)ns * n, sizeof(cplx));
    cplx *Cc = (cplx *)calloc((size_t)ns * n, sizeof(cplx));
    double *P = (double *)malloc(sizeof(double) * C * n);
    cplx *Ph = (cplx *)malloc(sizeof(cplx) * C * n);
    for (int r = 0; r < ny * nx; r++) {
        int yr = ys[r / nx], xr = xs[r % nx];
        for (int t = 0; t < C; t++)
            for (int u = 0; u < ps; u++)
                for (int v = 0; v < ps; v++)
                    P[t * n + u * ps + v] = (double)img[(size_t)t * H * W + (size_t)(yr + u) * W + (xr + v)];
        dft_mode3(P, C, ps, Ph);
        for (int j = 0; j < ns; j++) {
            const cplx *A = Ph + j * n;
            for (int a = 0; a < ps; a++)
                for (int b = 0; b < ps; b++) {
                    cplx sr = c_make(0.0, 0.0), sc = c_make(0.0, 0.0);
                    for (int k = 0; k < ps; k++) {
                        sr = c_add(sr, c_mul(A[a * ps + k], c_conj(A[b * ps + k])));  /* (A A^H)[a][b] */
                        sc = c_add(sc, c_mul(c_conj(A[k * ps + a]), A[k * ps + b]));  /* (A^H A)[a][b] */
                    }
                    Cr[j * n + a * ps + b] = c_add(Cr[j * n + a * ps + b], sr);
                    Cc[j * n + a * ps + b] = c_add(Cc[j * n + a * ps + b], sc);
                }
        }
    }
    for (int e = 0; e < ns * n; e++) {
        crow[2 * e] = Cr[e].re; crow[2 * e + 1] = Cr[e].im;
        ccol[2 * e] = Cc[e].re; ccol[2 * e + 1] = Cc[e].im;
    }
    free(Cr); free(Cc); free(P); free(Ph); free(ys); free(xs);
    return ny * nx;
}

/* ------------------------------------------------- Eq. 7-8: Haar matrix */

/* H_1 = [1]; H_2N = (1/sqrt 2) [ H_N (x) [1, 1] ; I_N (x) [1, -1] ].
 * Hm: K x K row-major.  K must be a power of two. */
void htso_haar_matrix(int K, double *Hm)
{
    double *cur = (double *)malloc(sizeof(double) * K * K);
    double *nxt = (double *)malloc(sizeof(double) * K * K);
    double h = 1.0 / sqrt(2.0);
    int N = 1;
    cur[0] = 1.0;
    while (N < K) {
        int M = 2 * N;
        for (int e = 0; e < M * M; e++) nxt[e] = 0.0;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                nxt[i * M + 2 * j] = h * cur[i * N + j];
                nxt[i * M + 2 * j + 1] = h * cur[i * N + j];
            }
        for (int i = 0; i < N; i++) {
            nxt[(N + i) * M + 2 * i] = h;
            nxt[(N + i) * M + 2 * i + 1] = -h;
        }
        double *tmp = cur; cur = nxt; nxt = tmp;
        N = M;
    }
    memcpy(Hm, cur, sizeof(double) * K * K);
    free(cur);
    free(nxt);
}

/* ------------------------------------- Eq. 19-21: forward / inverse */

/* Patch-level forward projection of one patch (Eq. 19 without the Haar
 * factor): in the Fourier domain of mode 3, Shat^(j) = U^(j)^H Phat^(j) V^(j).
 * P: C x ps x ps real; S: C x ps x ps complex (re,im pairs). */
void htso_patch_forward(const double *P, int C, int ps, const double *basis, double *S)
{
    int n = ps * ps;
    cplx *Ph = (cplx *)malloc(sizeof(cplx) * C * n);
    cplx *T = (cplx *)malloc(sizeof(cplx) * n);
    dft_mode3(P, C, ps, Ph);
    for (int j = 0; j < C; j++) {
        /* T = Phat V */
        for (int a = 0; a < ps; a++)
            for (int jj = 0; jj < ps; jj++) {
                cplx acc = c_make(0.0, 0.0);
                for (int b = 0; b < ps; b++)
                    acc = c_add(acc, c_mul(Ph[j * n + a * ps + b], basis_at(basis, C, ps, j, 1, b, jj)));
                T[a * ps + jj] = acc;
            }
        /* S = U^H T */
        for (int i = 0; i < ps; i++)
            for (int jj = 0; jj < ps; jj++) {
                cplx acc = c_make(0.0, 0.0);
                for (int a = 0; a < ps; a++)
                    acc = c_add(acc, c_mul(c_conj(basis_at(basis, C, ps, j, 0, a, i)), T[a * ps + jj]));
                S[2 * (j * n + i * ps + jj)] = acc.re;
                S[2 * (j * n + i * ps + jj) + 1] = acc.im;
            }
    }
    free(Ph);
    free(T);
}

/* Inverse of htso_patch_forward: Phat^(j) = U^(j) Shat^(j) V^(j)^H, then the
 * inverse DFT along mode 3.  Returns the largest imaginary residue. */
double htso_patch_inverse(const double *S, int C, int ps, const double *basis, double *P)
{
    int n = ps * ps;
    cplx *Ph = (cplx *)malloc(sizeof(cplx) * C * n);
    cplx *T = (cplx *)malloc(sizeof(cplx) * n);
    for (int j = 0; j < C; j++) {
        /* T = Shat V^H */
        for (int i = 0; i < ps; i++)
            for (int b = 0; b < ps; b++) {
                cplx acc = c_make(0.0, 0.0);
                for (int jj = 0; jj < ps; jj++) {
                    cplx s = c_make(S[2 * (j * n + i * ps + jj)], S[2 * (j * n + i * ps + jj) + 1]);
                    acc = c_add(acc, c_mul(s, c_conj(basis_at(basis, C, ps, j, 1, b, jj))));
                }
                T[i * ps + b] = acc;
            }
        /* Phat = U T */
        for (int a = 0; a < ps; a++)
            for (int b = 0; b < ps; b++) {
                cplx acc = c_make(0.0, 0.0);
                for (int i = 0; i < ps; i++)
                    acc = c_add(acc, c_mul(basis_at(basis, C, ps, j, 0, a, i), T[i * ps + b]));
                Ph[j * n + a * ps + b] = acc;
            }
    }
    double max_im = 0.0;
    idft_mode3(Ph, C, ps, P, &max_im);
    free(Ph);
    free(T);
    return max_im;
}

/* Eq. 19: S = U^T * G * V x_4 U_Haar for a group G of K patches
 * (K x C x ps x ps real).  S: K x C x ps x ps complex; row h of the group
 * axis holds Haar coefficient h (Eq. 8 row order). */
void htso_group_forward(const double *G, int K, int C, int ps, const double *basis, double *S)
{
    int m = C * ps * ps;  /* complex coefficients per patch */
    double *Hm = (double *)malloc(sizeof(double) * K * K);
    double *Sk = (double *)malloc(sizeof(double) * 2 * (size_t)K * m);
    htso_haar_matrix(K, Hm);
    for (int k = 0; k < K; k++) htso_patch_forward(G + (size_t)k * m, C, ps, basis, Sk + 2 * (size_t)k * m);
    for (int h = 0; h < K; h++)
        for (int e = 0; e < 2 * m; e++) {
            double acc = 0.0;
            for (int k = 0; k < K; k++) acc = acc + Hm[h * K + k] * Sk[2 * (size_t)k * m + e];
            S[2 * (size_t)h * m + e] = acc;
        }
    free(Hm);
    free(Sk);
}

/* Eq. 21: G = U * S * V^T x_4 U_Haar^-1 (U_Haar^-1 = U_Haar^T).  Returns the
 * largest imaginary residue of the inverse mode-3 DFT. */
double htso_group_inverse(const double *S, int K, int C, int ps, const double *basis, double *G)
{
    int m = C * ps * ps;
    double *Hm = (double *)malloc(sizeof(double) * K * K);
    double *Sk = (double *)malloc(sizeof(double) * 2 * (size_t)K * m);
    htso_haar_matrix(K, Hm);
    for (int k = 0; k < K; k++)
        for (int e = 0; e < 2 * m; e++) {
            double acc = 0.0;
            for (int h = 0; h < K; h++) acc = acc + Hm[h * K + k] * S[2 * (size_t)h * m + e];
            Sk[2 * (size_t)k * m + e] = acc;
        }
    double max_im = 0.0;
    for (int k = 0; k < K; k++) {
        double r = htso_patch_inverse(Sk + 2 * (size_t)k * m, C, ps, basis, G + (size_t)k * m);
        if (r > max_im) max_im = r;
    }
    free(Hm);
    free(Sk);
    return max_im;
}

/* Eq. 20: hard thresholding.  A coefficient whose imaginary part is exactly
 * zero is real and kept iff |re| >= tau; a complex one is kept iff its
 * modulus is >= tau.  n = number of complex entries.  Returns the count kept. */
long htso_threshold(double *S, long n, double tau)
{
    long kept = 0;
    for (long e = 0; e < n; e++) {
        double re = S[2 * e], im = S[2 * e + 1];
        double mag = (im == 0.0) ? fabs(re) : sqrt(re * re + im * im);
        if (mag < tau) {
            S[2 * e] = 0.0;
            S[2 * e + 1] = 0.0;
        } else {
            kept++;
        }
    }
    return kept;
}

/* -------------------------------------------- Alg. 1: the whole image */

/* Gather group r: K patches (C x ps x ps, double) at the raster indices. */
static void gather_group(const float *img, int H, int W, int C, int ps, int K, const int32_t *idx, double *G)
{
    int n = ps * ps;
    for (int k = 0; k < K; k++) {
        int y = idx[k] / W, x = idx[k] % W;
        for (int t = 0; t < C; t++)
            for (int u = 0; u < ps; u++)
                for (int v = 0; v < ps; v++)
                    G[((size_t)k * C + t) * n + u * ps + v] =
                        (double)img[(size_t)t * H * W + (size_t)(y + u) * W + (x + v)];
    }
}

/* Alg. 1 with given groups (idx: nref x K, from htso_match), basis and tau.
 * out: C x H x W doubles (plain average of all estimates; not clipped).
 * stats (optional, 3 entries): coefficients kept, groups, max imaginary
 * residue x 1e18 (rounded).  Returns 0, or -1 on bad input. */
static int denoise_groups_impl(const float *noisy, int H, int W, int C, const htso_params *p, const double *basis,
                               double tau, const double *taus, const int32_t *idx, const double *mean_est,
                               double *out, double *stats);

int htso_denoise_groups(const float *noisy, int H, int W, int C, const htso_params *p,
                        const double *basis, double tau, const int32_t *idx, double *out, double *stats)
{
    return denoise_groups_impl(noisy, H, W, C, p, basis, tau, NULL, idx, NULL, out, stats);
}

/* The same with a threshold per group (taus[r] for reference r), for a
 * spatially varying noise level. */
int htso_denoise_groups_taus(const float *noisy, int H, int W, int C, const htso_params *p,
                             const double *basis, const double *taus, const int32_t *idx, double *out,
                             double *stats)
{
    return denoise_groups_impl(noisy, H, W, C, p, basis, 0.0, taus, idx, NULL, out, stats);
}

/* RA-Haar-tSVD (the enhancement strategy, Eq. 24-25): as
 * htso_denoise_groups_taus (taus NULL: one tau), with the first Haar row of
 * every group (Eq. 24: sqrt(K) times the group's mean patch in the
 * transform domain) replaced by sqrt(K) times the transform of a refined
 * mean patch mean_est[r] (C x ps x ps doubles per reference, Eq. 25) and
 * kept whole (not thresholded). */
int htso_denoise_groups_ra(const float *noisy, int H, int W, int C, const htso_params *p, const double *basis,
                           double tau, const double *taus, const int32_t *idx, const double *mean_est, double *out,
                           double *stats)
{
    if (!mean_est) return -1;
    return denoise_groups_impl(noisy, H, W, C, p, basis, tau, taus, idx, mean_est, out, stats);
}

static int denoise_groups_impl(const float *noisy, int H, int W, int C, const htso_params *p, const double *basis,
                               double tau, const double *taus, const int32_t *idx, const double *mean_est,
                               double *out, double *stats)
{
    int ps = p->ps, K = p->K, n = ps * ps, m = C * n;
    int ny = htso_grid(H, ps, p->step, NULL), nx = htso_grid(W, ps, p->step, NULL);
    if (ny == 0 || nx == 0) return -1;
    int nref = ny * nx;
    double *num = (double *)calloc((size_t)C * H * W, sizeof(double));
    double *w = (double *)calloc((size_t)H * W, sizeof(double));
    const int CH = 512;
    double *est = (double *)malloc(sizeof(double) * (size_t)CH * K * m);
    long kept_total = 0;
    double max_im = 0.0;
    for (int r0 = 0; r0 < nref; r0 += CH) {
        int r1 = r0 + CH < nref ? r0 + CH : nref;
        long kept_chunk = 0;
        double im_chunk = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : kept_chunk) reduction(max : im_chunk)
        for (int r = r0; r < r1; r++) {
            double *G = (double *)malloc(sizeof(double) * (size_t)K * m);
            double *S = (double *)malloc(sizeof(double) * 2 * (size_t)K * m);
            gather_group(noisy, H, W, C, ps, K, idx + (size_t)r * K, G);
            htso_group_forward(G, K, C, ps, basis, S);            /* Eq. 19 */
            kept_chunk += htso_threshold(S, (long)K * m, taus ? taus[r] : tau); /* Eq. 20 */
            if (mean_est) { /* Eq. 24-25: Haar row 0 := sqrt(K) x transform of the refined mean patch */
                htso_patch_forward(mean_est + (size_t)r * m, C, ps, basis, S);
                for (long e = 0; e < 2 * (long)m; e++) S[e] = S[e] * sqrt((double)K);
            }
            double im = htso_group_inverse(S, K, C, ps, basis, est + (size_t)(r - r0) * K * m); /* Eq. 21 */
            if (im > im_chunk) im_chunk = im;
            free(G);
            free(S);
        }
        kept_total += kept_chunk;
        if (im_chunk > max_im) max_im = im_chunk;
        /* Alg. 1 step 3: write every estimate back to its location, in
         * reference order (sequential, so the sum order is fixed). */
        for (int r = r0; r < r1; r++) {
            const int32_t *g = idx + (size_t)r * K;
            const double *E = est + (size_t)(r - r0) * K * m;
            for (int k = 0; k < K; k++) {
                int y = g[k] / W, x = g[k] % W;
                for (int u = 0; u < ps; u++)
                    for (int v = 0; v < ps; v++) {
                        size_t o = (size_t)(y + u) * W + (x + v);
                        for (int t = 0; t < C; t++)
                            num[(size_t)t * H * W + o] = num[(size_t)t * H * W + o] + E[((size_t)k * C + t) * n + u * ps + v];
                        w[o] = w[o] + 1.0;
                    }
            }
        }
    }
    for (int t = 0; t < C; t++)
        for (size_t o = 0; o < (size_t)H * W; o++)
            out[(size_t)t * H * W + o] = num[(size_t)t * H * W + o] / w[o];
    if (stats) {
        stats[0] = (double)kept_total;
        stats[1] = (double)nref;
        stats[2] = max_im;
    }
    free(num);
    free(w);
    free(est);
    return 0;
}

/* ---------------------------------- Eq. 16-18, 22-23: rank of lambda_hat */

/* Eigenvalues of circ(G) circ(G)^T (Eq. 13-16).  The Gram matrix is
 * circulant, so its eigenvalues are lambda_m = || sum_k e^{-2 pi i m k/K} p_k ||^2,
 * m = 0..K-1 (m = 0 is Eq. 18, m = K/2 is Eq. 22).  G: K x D (patch k = row). */
void htso_group_lambdas(const double *G, int K, int D, double *lam)
{
    for (int m = 0; m < K; m++) {
        double acc = 0.0;
        for (int d = 0; d < D; d++) {
            cplx z = c_make(0.0, 0.0);
            for (int k = 0; k < K; k++)
                z = c_add(z, c_mul(c_make(G[(size_t)k * D + d], 0.0), unit_root((long)m * k, K)));
            acc = acc + (z.re * z.re + z.im * z.im);
        }
        lam[m] = acc;
    }
}

/* Rank position a of lambda_hat = lambda_{K/2} among the K eigenvalues in
 * ascending order (1-based; equal values rank lowest). */
int htso_rank_of_hat(const double *lam, int K)
{
    int a = 1;
    for (int m = 0; m < K; m++)
        if (m != K / 2 && lam[m] < lam[K / 2]) a++;
    return a;
}

/* For every group: a_out[r] = rank position of lambda_hat (optional).
 * Returns the number of groups with a <= gamma_rank (Eq. 23 "adjust" votes). */
int htso_rank_votes(const float *img, int H, int W, int C, const htso_params *p,
                    const int32_t *idx, int32_t *a_out)
{
    int ps = p->ps, K = p->K, D = C * ps * ps;
    int ny = htso_grid(H, ps, p->step, NULL), nx = htso_grid(W, ps, p->step, NULL);
    int nref = ny * nx, votes = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : votes)
    for (int r = 0; r < nref; r++) {
        double *G = (double *)malloc(sizeof(double) * (size_t)K * D);
        double *lam = (double *)malloc(sizeof(double) * K);
        gather_group(img, H, W, C, ps, K, idx + (size_t)r * K, G);
        htso_group_lambdas(G, K, D, lam);
        int a = htso_rank_of_hat(lam, K);
        if (a_out) a_out[r] = a;
        if ((double)a <= p->gamma_rank) votes++;
        free(G);
        free(lam);
    }
    return votes;
}

/* Number of OpenMP threads the oracle's parallel loops use. */
int htso_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void htso_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
