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

// Raw channel products of the reference patches, exactly: every product of
// two floats is split into p + e (p = fl(x y), e = fma(x, y, -p)) and
// accumulated in a double-float (hi, lo) pair; |error| <= n u^2 sum|terms| for
// n terms (u = 2^-24), i.e. FP64-grade without the FP64 pipes.
//   row sums  M_tt'[a][b] = sum_i sum_k P_i^(t)[a][k] P_i^(t')[b][k]
//   col sums  N_tt'[a][b] = sum_i sum_k P_i^(t)[k][a] P_i^(t')[k][b]
// for channel pairs t <= t' (upper triangles when t = t').  k_cov_sum adds
// the blocks' partial sums in FP64 in block order and forms the Fourier-slice
// covariances C_row^(j) = (1/c) sum_{t,t'} w^{j(t-t')} M_tt',
// C_col^(j) = (1/c) sum_{t,t'} w^{j(t'-t)} N_tt', w = exp(-2 pi i / c).
template <int C>
struct CovCfg {
    static constexpr int NSYM = C;                   // channel pairs (t, t)
    static constexpr int NASY = C * (C - 1) / 2;     // channel pairs t < t'
    static constexpr int PER = NSYM * 36 + NASY * 64;  // entries per side
    static constexpr int NT = 2 * PER;               // row + col
    static constexpr int THREADS = (NT + 31) / 32 * 32;
};

__device__ __forceinline__ void task_of(int t, int per, int nsym, int &m, int &t0, int &t1, int &a, int &b) {
    m = t / per;
    int rem = t - m * per;
    if (rem < nsym * 36) {
        t0 = t1 = rem / 36;
        pair_of(rem % 36, a, b);
    } else {
        rem -= nsym * 36;
        const int q = rem / 64;  // (0,1), (0,2), (1,2)
        t0 = (q == 2) ? 1 : 0;
        t1 = (q == 0) ? 1 : 2;
        a = (rem % 64) >> 3;
        b = rem & 7;
    }
}

// Explicit roundings: no contraction may merge these steps.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);                                            // x y = p + e exactly
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));  // hi + p = s + err exactly
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

template <int C>
__global__ void __launch_bounds__(CovCfg<C>::THREADS) k_cov(const float *__restrict__ img, int H, int W, int step,
                                                            int nx, int nref, double *__restrict__ partials) {
    constexpr int NT = CovCfg<C>::NT;
    __shared__ float sp[COV_BATCH][C * 64];
    const int t = threadIdx.x;
    const size_t HW = (size_t)H * W;
    int m = 0, t0 = 0, t1 = 0, a = 0, b = 0;
    if (t < NT) task_of(t, CovCfg<C>::PER, CovCfg<C>::NSYM, m, t0, t1, a, b);
    float hi = 0.f, lo = 0.f;
    const int r0 = blockIdx.x * COV_REFS;
    const int r1 = min(nref, r0 + COV_REFS);
    for (int rb = r0; rb < r1; rb += COV_BATCH) {
        const int nb = min(COV_BATCH, r1 - rb);
        for (int w = t; w < nb * C * 64; w += blockDim.x) {
            const int rr = w / (C * 64), ce = w - rr * (C * 64);
            const int c = ce >> 6, e = ce & 63;
            const int r = rb + rr;
            const int y = grid_pos(r / nx, H, step) + (e >> 3), x = grid_pos(r % nx, W, step) + (e & 7);
            sp[rr][ce] = __ldg(img + (size_t)c * HW + (size_t)y * W + x);
        }
        __syncthreads();
        if (t < NT) {
            for (int rr = 0; rr < nb; ++rr) {
                const float *X = sp[rr] + t0 * 64, *Y = sp[rr] + t1 * 64;
                if (m == 0) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) df_add(hi, lo, X[a * 8 + k], Y[b * 8 + k]);
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) df_add(hi, lo, X[k * 8 + a], Y[k * 8 + b]);
                }
            }
            // renormalise so that lo stays below an ulp of hi
            const float s = __fadd_rn(hi, lo);
            lo = __fsub_rn(lo, __fsub_rn(s, hi));
            hi = s;
        }
        __syncthreads();
    }
    if (t < NT) partials[(size_t)blockIdx.x * NT + t] = (double)hi + (double)lo;
}

// Sum of the blocks' partial sums, one warp per entry, fixed reduction tree.
template <int C>
__global__ void __launch_bounds__(256) k_cov_sum(const double *__restrict__ partials, int nblocks,
                                                 double *__restrict__ totals) {
    constexpr int NT = CovCfg<C>::NT;
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= NT) return;
    double sum = 0.0;
    for (int bl = lane; bl < nblocks; bl += 32) sum += partials[(size_t)bl * NT + t];
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    if (lane == 0) totals[t] = sum;
}

// Entry [a][b] of the Fourier-slice covariance of side m (0 row, 1 col) and
// slice j from the channel-pair sums: (1/c) sum_{t0,t1} w^{j d} X_{t0 t1}[a][b]
// with d = t0 - t1 (row) or t1 - t0 (col), w = exp(-2 pi i / 3).
template <int C>
__device__ void cov_entry(const double *__restrict__ tot, int j, int m, int a, int b, double &sr, double &si) {
    constexpr int PER = CovCfg<C>::PER;
    sr = 0.0;
    si = 0.0;
    for (int t0 = 0; t0 < C; ++t0)
        for (int t1 = 0; t1 < C; ++t1) {
            const int lo_t = min(t0, t1), hi_t = max(t0, t1);
            const int aa = (t0 > t1) ? b : a, bb = (t0 > t1) ? a : b;  // X_{t1 t0} = X_{t0 t1}^T
            int idx;
            if (lo_t == hi_t) {
                const int p = min(aa, bb), r = max(aa, bb);
                idx = lo_t * 36 + (p * 8 - p * (p - 1) / 2) + (r - p);
            } else {
                const int pq = (lo_t == 0 && hi_t == 1) ? 0 : ((lo_t == 0) ? 1 : 2);
                idx = C * 36 + pq * 64 + aa * 8 + bb;
            }
            const double v = tot[m * PER + idx];
            int d = (m == 0) ? (t0 - t1) : (t1 - t0);
            d = ((j * d) % 3 + 3) % 3;
            if (C == 1 || d == 0) {
                sr += v / C;
            } else {
                // exp(-2 pi i d / 3) / 3 = -1/6 -+ i sqrt(3)/6
                const double s6 = 0.28867513459481288225;  // sqrt(3) / 6
                sr += v * (-1.0 / 6.0);
                si += v * (d == 1 ? -s6 : s6);
            }
        }
}

// One 8x8 Hermitian eigenproblem per block (one warp), cyclic parallel Jacobi:
// 4 disjoint rotations per round, 7 rounds per sweep.  The rotation for
// (p, q) makes a_pq real with the phase e^{i phi} = a_pq / |a_pq| and then
// zeroes it with the real Jacobi rotation (t = sgn(th) / (|th| + sqrt(th^2+1)),
// th = (a_qq - a_pp) / (2 |a_pq|)).  The angle is computed in FP32 (a slightly
// inexact angle only slows convergence); the phase and (c, s) are then
// renormalised in FP64 by two Newton steps of 1/sqrt(x) at x ~ 1, so every
// applied rotation is unitary to FP64 precision and the spectrum is exact to
// FP64 rounding.  Updates are in FP64.
template <int C>
__global__ void __launch_bounds__(32) k_jacobi(const double *__restrict__ totals, int nmat, double *__restrict__ b64,
                                               float *__restrict__ b32, double *__restrict__ eig) {
    __shared__ double Ar[64], Ai[64], Vr[64], Vi[64];
    __shared__ double pc[4], ps_[4], per[4], pei[4];
    __shared__ int pp[4], pq[4];
    __shared__ int perm[8];
    const int w = blockIdx.x, lane = threadIdx.x & 31;
    if (w >= nmat) return;
    for (int e = lane; e < 64; e += 32) {
        const int a = e >> 3, b = e & 7;
        double sr, si;
        if (a <= b) {
            cov_entry<C>(totals, w >> 1, w & 1, a, b, sr, si);
            if (a == b) si = 0.0;
        } else {
            cov_entry<C>(totals, w >> 1, w & 1, b, a, sr, si);
            si = -si;  // Hermitian
        }
        Ar[e] = sr;
        Ai[e] = si;
        Vr[e] = (a == b) ? 1.0 : 0.0;
        Vi[e] = 0.0;
    }
    __syncwarp();
    // Sweeps until the off-diagonal mass is below 1e-26 of the diagonal's
    // (relative 3e-13 in norm, above the FP64 round-off floor); 24 at most.
    for (int sweep = 0; sweep < 24; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = lane; e < 64; e += 32) {
            const double m2 = Ar[e] * Ar[e] + Ai[e] * Ai[e];
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
                const int L1 = 1 + ((6 - i + round) % 7);
                const int p = min(L0, L1), q = max(L0, L1);
                const double zr = Ar[p * 8 + q], zi = Ai[p * 8 + q];
                const double r2 = zr * zr + zi * zi;
                double c = 1.0, s = 0.0, er = 1.0, ei = 0.0;
                if (r2 > 1e-300 && r2 > 1e-30 * (Ar[p * 9] * Ar[p * 9] + Ar[q * 9] * Ar[q * 9])) {
                    const float r = sqrtf((float)r2);
                    er = (double)((float)zr / r);
                    ei = (double)((float)zi / r);
                    const float th = (float)((Ar[q * 9] - Ar[p * 9]) / (2.0 * (double)r));
                    const float tt = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                    const float cf = rsqrtf(fmaf(tt, tt, 1.f));
                    c = (double)cf;
                    s = (double)(tt * cf);
#pragma unroll
                    for (int it = 0; it < 2; ++it) {  // x -> x (3 - |x|^2) / 2
                        const double ne = 1.5 - 0.5 * (er * er + ei * ei);
                        er *= ne;
                        ei *= ne;
                        const double nc = 1.5 - 0.5 * (c * c + s * s);
                        c *= nc;
                        s *= nc;
                    }
                }
                pc[i] = c;
                ps_[i] = s;
                per[i] = er;
                pei[i] = ei;
                pp[i] = p;
                pq[i] = q;
            }
            __syncwarp();
            const int i = lane >> 3, k = lane & 7;
            const int p = pp[i], q = pq[i];
            const double c = pc[i], s = ps_[i], er = per[i], ei = pei[i];
            {   // columns: A <- A J
                const double xr = Ar[k * 8 + p], xi = Ai[k * 8 + p];
                const double yr = Ar[k * 8 + q], yi = Ai[k * 8 + q];
                const double zr = er * yr + ei * yi, zi = er * yi - ei * yr;  // conj(e) * y
                Ar[k * 8 + p] = c * xr - s * zr;
                Ai[k * 8 + p] = c * xi - s * zi;
                Ar[k * 8 + q] = s * xr + c * zr;
                Ai[k * 8 + q] = s * xi + c * zi;
            }
            __syncwarp();
            {   // rows: A <- J^H A
                const double xr = Ar[p * 8 + k], xi = Ai[p * 8 + k];
                const double yr = Ar[q * 8 + k], yi = Ai[q * 8 + k];
                const double zr = er * yr - ei * yi, zi = er * yi + ei * yr;  // e * y
                Ar[p * 8 + k] = c * xr - s * zr;
                Ai[p * 8 + k] = c * xi - s * zi;
                Ar[q * 8 + k] = s * xr + c * zr;
                Ai[q * 8 + k] = s * xi + c * zi;
            }
            __syncwarp();
            {   // eigenvectors: V <- V J
                const double xr = Vr[k * 8 + p], xi = Vi[k * 8 + p];
                const double yr = Vr[k * 8 + q], yi = Vi[k * 8 + q];
                const double zr = er * yr + ei * yi, zi = er * yi - ei * yr;
                Vr[k * 8 + p] = c * xr - s * zr;
                Vi[k * 8 + p] = c * xi - s * zi;
                Vr[k * 8 + q] = s * xr + c * zr;
                Vi[k * 8 + q] = s * xi + c * zi;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        int idx[8];
        for (int i = 0; i < 8; ++i) idx[i] = i;
        for (int i = 0; i < 8; ++i)
            for (int jj = i + 1; jj < 8; ++jj)
                if (Ar[idx[jj] * 9] < Ar[idx[i] * 9]) {
                    const int tmp = idx[i];
                    idx[i] = idx[jj];
                    idx[jj] = tmp;
                }
        for (int i = 0; i < 8; ++i) perm[i] = idx[i];
    }
    __syncwarp();
    for (int e = lane; e < 64; e += 32) {
        const int a = e >> 3, i = e & 7;
        const int src = a * 8 + perm[i];
        const double vr = Vr[src], vi = Vi[src];
        b64[((size_t)w * 64 + e) * 2] = vr;
        b64[((size_t)w * 64 + e) * 2 + 1] = vi;
        b32[((size_t)w * 64 + e) * 2] = (float)vr;
        b32[((size_t)w * 64 + e) * 2 + 1] = (float)vi;
    }
    if (lane < 8) eig[w * 8 + lane] = Ar[perm[lane] * 9];
}

}  // namespace

size_t cov_partial_count(const Geom &g) {
    const int nb = (g.nref + COV_REFS - 1) / COV_REFS;
    const int nt = (g.C == 3) ? CovCfg<3>::NT : CovCfg<1>::NT;
    return (size_t)nb * nt + nt;  // per-block partial sums, then the totals
}

template <int C>
hts_status launch_basis_c(const float *img, const Geom &g, double *partials, double *b64, float *b32, double *eig,
                          cudaStream_t s) {
    constexpr int NT = CovCfg<C>::NT;
    const int nb = (g.nref + COV_REFS - 1) / COV_REFS;
    const int ns = C / 2 + 1;
    double *totals = partials + (size_t)nb * NT;
    {
        KTimer kt("k_cov", s);
        k_cov<C><<<nb, CovCfg<C>::THREADS, 0, s>>>(img, g.H, g.W, g.step, g.nx, g.nref, partials);
    }
    if (hts_status st = check_launch("k_cov"); st != HTS_OK) return st;
    {
        KTimer kt("k_cov_sum", s);
        k_cov_sum<C><<<(NT * 32 + 255) / 256, 256, 0, s>>>(partials, nb, totals);
    }
    if (hts_status st = check_launch("k_cov_sum"); st != HTS_OK) return st;
    {
        KTimer kt("k_jacobi", s);
        k_jacobi<C><<<ns * 2, 32, 0, s>>>(totals, ns * 2, b64, b32, eig);
    }
    return check_launch("k_jacobi");
}

hts_status launch_basis(const float *img, const Geom &g, double *partials, double *b64, float *b32, double *eig,
                        cudaStream_t s) {
    if (g.C == 1) return launch_basis_c<1>(img, g, partials, b64, b32, eig, s);
    if (g.C == 3) return launch_basis_c<3>(img, g, partials, b64, b32, eig, s);
    return HTS_EUNSUPPORTED;
}

}  // namespace hts
