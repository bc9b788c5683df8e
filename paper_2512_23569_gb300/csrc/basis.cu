// Globally-learned t-SVD basis (Sec. III-B2, Eq. 11) on sm_103a, in FP64.
//
// k_cov      : every block takes a run of reference patches, forms their
//              unitary DFT along channels (slice 0 real, slice 1 complex;
//              slice 2 is the conjugate of slice 1) and accumulates the upper
//              triangles of C_row^(j) = sum P P^H and C_col^(j) = sum P^H P,
//              one thread per matrix entry, into per-block partial sums;
// k_cov_sum  : adds the partial sums in block order (deterministic) and
//              fills the Hermitian matrices;
// k_jacobi   : one warp per 8x8 Hermitian matrix, parallel cyclic Jacobi
//              (4 disjoint complex rotations per round, 7 rounds per sweep),
//              eigenvalues sorted ascending, eigenvectors as columns.
#include "hts_internal.h"

namespace hts {
namespace {

constexpr int COV_REFS = 64;   // reference patches per block
constexpr int COV_BATCH = 16;  // staged at once
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void pair_of(int p, int &a, int &b) {
    // p in [0, 36): (a, b) with a <= b, row-major over the upper triangle
    a = 0;
    int rem = p;
    while (rem >= 8 - a) {
        rem -= 8 - a;
        ++a;
    }
    b = a + rem;
}

template <int C>
__global__ void __launch_bounds__(256) k_cov(const float *__restrict__ img, int H, int W, int step, int nx, int nref,
                                              double *__restrict__ partials) {
    constexpr int NS = (C == 3) ? 2 : 1;
    constexpr int NT = NS * 2 * 36;
    constexpr int SW = (C == 3) ? 192 : 64;  // doubles per staged patch
    __shared__ double sp[COV_BATCH][SW];
    const int t = threadIdx.x;
    const size_t HW = (size_t)H * W;
    const double k3 = 0.57735026918962576451;

    int j = 0, m = 0, a = 0, b = 0;
    if (t < NT) {
        j = t / 72;
        m = (t % 72) / 36;
        pair_of(t % 36, a, b);
    }
    double ar = 0.0, ai = 0.0;
    const int r0 = blockIdx.x * COV_REFS;
    const int r1 = min(nref, r0 + COV_REFS);
    for (int rb = r0; rb < r1; rb += COV_BATCH) {
        const int nb = min(COV_BATCH, r1 - rb);
        for (int w = t; w < nb * 64; w += blockDim.x) {
            const int rr = w >> 6, e = w & 63;
            const int r = rb + rr;
            const int y = grid_pos(r / nx, H, step) + (e >> 3), x = grid_pos(r % nx, W, step) + (e & 7);
            const size_t o = (size_t)y * W + x;
            if (C == 1) {
                sp[rr][e] = (double)__ldg(img + o);
            } else {
                const double R = (double)__ldg(img + o), G = (double)__ldg(img + HW + o),
                             B = (double)__ldg(img + 2 * HW + o);
                sp[rr][e] = ((R + G) + B) * k3;
                sp[rr][64 + 2 * e] = (R - 0.5 * (G + B)) * k3;
                sp[rr][64 + 2 * e + 1] = (B - G) * 0.5;
            }
        }
        __syncthreads();
        if (t < NT) {
            for (int rr = 0; rr < nb; ++rr) {
                const double *A = sp[rr];
                if (j == 0) {
                    if (m == 0) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) ar = fma(A[a * 8 + k], A[b * 8 + k], ar);
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) ar = fma(A[k * 8 + a], A[k * 8 + b], ar);
                    }
                } else {
                    const double *Z = A + 64;  // complex, interleaved
                    if (m == 0) {  // sum_k x_ak conj(x_bk)
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const double xr = Z[2 * (a * 8 + k)], xi = Z[2 * (a * 8 + k) + 1];
                            const double yr = Z[2 * (b * 8 + k)], yi = Z[2 * (b * 8 + k) + 1];
                            ar = fma(xr, yr, fma(xi, yi, ar));
                            ai = fma(xi, yr, fma(-xr, yi, ai));
                        }
                    } else {  // sum_k conj(x_ka) x_kb
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const double xr = Z[2 * (k * 8 + a)], xi = Z[2 * (k * 8 + a) + 1];
                            const double yr = Z[2 * (k * 8 + b)], yi = Z[2 * (k * 8 + b) + 1];
                            ar = fma(xr, yr, fma(xi, yi, ar));
                            ai = fma(xr, yi, fma(-xi, yr, ai));
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (t < NT) {
        partials[((size_t)blockIdx.x * NT + t) * 2] = ar;
        partials[((size_t)blockIdx.x * NT + t) * 2 + 1] = ai;
    }
}

// cov: [j][m][a][b][2]
template <int C>
__global__ void k_cov_sum(const double *__restrict__ partials, int nblocks, double *__restrict__ cov) {
    constexpr int NS = (C == 3) ? 2 : 1;
    constexpr int NT = NS * 2 * 36;
    const int t = threadIdx.x;
    if (t >= NT) return;
    double sr = 0.0, si = 0.0;
    for (int bl = 0; bl < nblocks; ++bl) {
        sr += partials[((size_t)bl * NT + t) * 2];
        si += partials[((size_t)bl * NT + t) * 2 + 1];
    }
    const int j = t / 72, m = (t % 72) / 36;
    int a, b;
    pair_of(t % 36, a, b);
    double *M = cov + (size_t)(j * 2 + m) * 128;
    if (a == b) si = 0.0;
    M[(a * 8 + b) * 2] = sr;
    M[(a * 8 + b) * 2 + 1] = si;
    M[(b * 8 + a) * 2] = sr;
    M[(b * 8 + a) * 2 + 1] = -si;
}

__global__ void __launch_bounds__(128) k_jacobi(const double *__restrict__ cov, int nmat, double *__restrict__ b64,
                                                float *__restrict__ b32, double *__restrict__ eig) {
    __shared__ double Ar[4][64], Ai[4][64], Vr[4][64], Vi[4][64];
    __shared__ double pc[4][4], ps_[4][4], per[4][4], pei[4][4];
    __shared__ int pp[4][4], pq[4][4];
    __shared__ int perm[4][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= nmat) return;
    const double *M = cov + (size_t)w * 128;
    for (int e = lane; e < 64; e += 32) {
        Ar[w][e] = M[2 * e];
        Ai[w][e] = M[2 * e + 1];
        Vr[w][e] = ((e >> 3) == (e & 7)) ? 1.0 : 0.0;
        Vi[w][e] = 0.0;
    }
    __syncwarp();
    // Cyclic sweeps until the off-diagonal mass is below 1e-26 of the
    // diagonal's (relative 3e-13 in norm: well under what the parity bars
    // need, and above the FP64 round-off floor so the test terminates);
    // Jacobi converges quadratically, 6-8 sweeps in practice, 16 at most.
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = lane; e < 64; e += 32) {
            const double m2 = Ar[w][e] * Ar[w][e] + Ai[w][e] * Ai[w][e];
            if ((e >> 3) == (e & 7)) dia += m2;
            else off += m2;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(FULL, off, o);
            dia += __shfl_xor_sync(FULL, dia, o);
        }
        if (off <= 1e-26 * dia || off == 0.0) break;
        for (int round = 0; round < 7; ++round) {
            if (lane < 4) {
                const int i = lane;
                const int L0 = (i == 0) ? 0 : 1 + ((i - 1 + round) % 7);
                const int k2 = 7 - i;
                const int L1 = 1 + ((k2 - 1 + round) % 7);
                const int p = min(L0, L1), q = max(L0, L1);
                const double app = Ar[w][p * 8 + p], aqq = Ar[w][q * 8 + q];
                const double zr = Ar[w][p * 8 + q], zi = Ai[w][p * 8 + q];
                const double r = sqrt(zr * zr + zi * zi);
                double c = 1.0, s = 0.0, er = 1.0, ei = 0.0;
                if (r > 1e-300) {
                    er = zr / r;
                    ei = zi / r;
                    const double th = (aqq - app) / (2.0 * r);
                    const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    c = 1.0 / sqrt(tt * tt + 1.0);
                    s = tt * c;
                }
                pc[w][i] = c;
                ps_[w][i] = s;
                per[w][i] = er;
                pei[w][i] = ei;
                pp[w][i] = p;
                pq[w][i] = q;
            }
            __syncwarp();
            const int i = lane >> 3, k = lane & 7;
            const int p = pp[w][i], q = pq[w][i];
            const double c = pc[w][i], s = ps_[w][i], er = per[w][i], ei = pei[w][i];
            {   // columns: A <- A J
                const double xr = Ar[w][k * 8 + p], xi = Ai[w][k * 8 + p];
                const double yr = Ar[w][k * 8 + q], yi = Ai[w][k * 8 + q];
                const double zr = er * yr + ei * yi, zi = er * yi - ei * yr;  // conj(e) * y
                Ar[w][k * 8 + p] = c * xr - s * zr;
                Ai[w][k * 8 + p] = c * xi - s * zi;
                Ar[w][k * 8 + q] = s * xr + c * zr;
                Ai[w][k * 8 + q] = s * xi + c * zi;
            }
            __syncwarp();
            {   // rows: A <- J^H A
                const double xr = Ar[w][p * 8 + k], xi = Ai[w][p * 8 + k];
                const double yr = Ar[w][q * 8 + k], yi = Ai[w][q * 8 + k];
                const double zr = er * yr - ei * yi, zi = er * yi + ei * yr;  // e * y
                Ar[w][p * 8 + k] = c * xr - s * zr;
                Ai[w][p * 8 + k] = c * xi - s * zi;
                Ar[w][q * 8 + k] = s * xr + c * zr;
                Ai[w][q * 8 + k] = s * xi + c * zi;
            }
            __syncwarp();
            {   // eigenvectors: V <- V J
                const double xr = Vr[w][k * 8 + p], xi = Vi[w][k * 8 + p];
                const double yr = Vr[w][k * 8 + q], yi = Vi[w][k * 8 + q];
                const double zr = er * yr + ei * yi, zi = er * yi - ei * yr;
                Vr[w][k * 8 + p] = c * xr - s * zr;
                Vi[w][k * 8 + p] = c * xi - s * zi;
                Vr[w][k * 8 + q] = s * xr + c * zr;
                Vi[w][k * 8 + q] = s * xi + c * zi;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        int idx[8];
        for (int i = 0; i < 8; ++i) idx[i] = i;
        for (int i = 0; i < 8; ++i)
            for (int jj = i + 1; jj < 8; ++jj)
                if (Ar[w][idx[jj] * 9] < Ar[w][idx[i] * 9]) {
                    const int tmp = idx[i];
                    idx[i] = idx[jj];
                    idx[jj] = tmp;
                }
        for (int i = 0; i < 8; ++i) perm[w][i] = idx[i];
    }
    __syncwarp();
    for (int e = lane; e < 64; e += 32) {
        const int a = e >> 3, i = e & 7;
        const int src = a * 8 + perm[w][i];
        const double vr = Vr[w][src], vi = Vi[w][src];
        b64[((size_t)w * 64 + e) * 2] = vr;
        b64[((size_t)w * 64 + e) * 2 + 1] = vi;
        b32[((size_t)w * 64 + e) * 2] = (float)vr;
        b32[((size_t)w * 64 + e) * 2 + 1] = (float)vi;
    }
    if (lane < 8) eig[w * 8 + lane] = Ar[w][perm[w][lane] * 9];
}

}  // namespace

size_t cov_partial_count(const Geom &g) {
    const int nb = (g.nref + COV_REFS - 1) / COV_REFS;
    const int ns = g.C / 2 + 1;
    return (size_t)nb * ns * 2 * 36 * 2 + (size_t)ns * 2 * 64 * 2;
}

hts_status launch_basis(const float *img, const Geom &g, double *partials, double *b64, float *b32, double *eig,
                        cudaStream_t s) {
    const int nb = (g.nref + COV_REFS - 1) / COV_REFS;
    const int ns = g.C / 2 + 1;
    double *cov = partials + (size_t)nb * ns * 2 * 36 * 2;
    if (g.C == 1) {
        {
            KTimer kt("k_cov", s);
            k_cov<1><<<nb, 256, 0, s>>>(img, g.H, g.W, g.step, g.nx, g.nref, partials);
        }
        if (hts_status st = check_launch("k_cov"); st != HTS_OK) return st;
        KTimer kt("k_cov_sum", s);
        k_cov_sum<1><<<1, 160, 0, s>>>(partials, nb, cov);
    } else if (g.C == 3) {
        {
            KTimer kt("k_cov", s);
            k_cov<3><<<nb, 256, 0, s>>>(img, g.H, g.W, g.step, g.nx, g.nref, partials);
        }
        if (hts_status st = check_launch("k_cov"); st != HTS_OK) return st;
        KTimer kt("k_cov_sum", s);
        k_cov_sum<3><<<1, 160, 0, s>>>(partials, nb, cov);
    } else {
        return HTS_EUNSUPPORTED;
    }
    if (hts_status st = check_launch("k_cov_sum"); st != HTS_OK) return st;
    {
        KTimer kt("k_jacobi", s);
        k_jacobi<<<1, 32 * ns * 2, 0, s>>>(cov, ns * 2, b64, b32, eig);
    }
    return check_launch("k_jacobi");
}

}  // namespace hts
