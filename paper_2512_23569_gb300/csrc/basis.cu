// Globally-learned t-SVD basis (Sec. III-B2, Eq. 11) on sm_103a, in FP64.
//
// k_cov      : the channel-pair sums behind C_row and C_col as sums along
//              image lines: every row (column) pair of a grid row (column) of
//              patches is summed once over the whole line, each position
//              weighted by the number of reference patches that cover it, in
//              exact products and double-float sums (see below), one thread
//              per matrix entry, per-block partial sums;
// k_cov_sum  : adds the partial sums in block order (deterministic) and
//              fills the Hermitian matrices;
// k_jacobi   : one warp per 8x8 Hermitian matrix, parallel cyclic Jacobi
//              (4 disjoint complex rotations per round, 7 rounds per sweep),
//              first in FP32, then refined in FP64; eigenvalues sorted
//              ascending, eigenvectors as columns.
#include <algorithm>

#include "hts_internal.h"

namespace hts {
namespace {

constexpr int COV_CH = 128;     // line positions staged per step
constexpr int COV_BLOCKS = 608;  // blocks per side at most (a constant: the partial sums' layout and order
                                 // do not depend on the device)
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
// accumulated in a double-float (hi, lo) pair over at most COV_CH terms, then
// added to an FP64 sum; |error| <= n u^2 sum|terms| per pair (u = 2^-24,
// n <= 128), i.e. FP64-grade without the FP64 pipes.
//   row sums  M_tt'[a][b] = sum_i sum_k P_i^(t)[a][k] P_i^(t')[b][k]
//   col sums  N_tt'[a][b] = sum_i sum_k P_i^(t)[k][a] P_i^(t')[k][b]
// for channel pairs t <= t' (upper triangles when t = t').  With the patches
// on the grid Y x X, M_tt'[a][b] = sum_{y in Y} sum_col m_X(col)
// I_t(y + a, col) I_t'(y + b, col), m_X(col) = number of grid positions x
// with x <= col <= x + 7 (1 or 2 at step 4): one weighted dot product of two
// image rows per grid row instead of one 8-term product per patch (and the
// same along columns for N).  Multiplying by m_X (an integer <= 8) is exact.
// k_cov_sum adds the blocks' partial sums in FP64 in block order and forms
// the Fourier-slice covariances C_row^(j) = (1/c) sum_{t,t'} w^{j(t-t')} M_tt',
// C_col^(j) = (1/c) sum_{t,t'} w^{j(t'-t)} N_tt', w = exp(-2 pi i / c).
template <int C>
struct CovCfg {
    static constexpr int NSYM = C;                   // channel pairs (t, t)
    static constexpr int NASY = C * (C - 1) / 2;     // channel pairs t < t'
    static constexpr int PER = NSYM * 36 + NASY * 64;  // entries per side
    static constexpr int NT = 2 * PER;               // row + col
    static constexpr int THREADS = (PER + 31) / 32 * 32 < 64 ? 64 : (PER + 31) / 32 * 32;
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

// Reference patches (grid 0, step, 2 step, ... plus n - 8) that cover index i of an axis of length n.
__device__ __forceinline__ int cover_count(int i, int n, int step) {
    const int last = n - PS;
    const int lo = max(0, i - (PS - 1)), hi = min(i, last);
    if (hi < lo) return 0;
    int c = hi / step - (lo + step - 1) / step + 1;
    if (c < 0) c = 0;
    if (last % step != 0 && last >= lo && last <= hi) c += 1;
    return c;
}

// blockIdx.y = side (0: row sums along image rows, 1: column sums along image columns); block b of a
// side takes grid lines b, b + nb, ... (nb = nb_r or nb_c); thread t < PER takes entry t of its side.
template <int C>
__global__ void __launch_bounds__(CovCfg<C>::THREADS) k_cov(const float *__restrict__ img, int H, int W, int step,
                                                            int ny, int nx, int nb_r, int nb_c,
                                                            double *__restrict__ partials) {
    constexpr int PER = CovCfg<C>::PER;
    constexpr int NL = C * PS;  // staged lines: channel * 8 + offset
    constexpr int LS = COV_CH + 4;
    __shared__ __align__(16) float sl[NL][LS];
    __shared__ __align__(16) float sw[COV_CH];
    const int side = blockIdx.y;
    const int nb = side == 0 ? nb_r : nb_c;
    if ((int)blockIdx.x >= nb) return;  // the whole block
    const int t = threadIdx.x;
    const bool valid = t < PER;
    int m = 0, t0 = 0, t1 = 0, a = 0, b = 0;
    if (valid) task_of(side * PER + t, PER, CovCfg<C>::NSYM, m, t0, t1, a, b);
    const size_t HW = (size_t)H * W;
    const int nlines = side == 0 ? ny : nx;
    const int len = side == 0 ? W : H;
    double acc = 0.0;
    for (int gl = blockIdx.x; gl < nlines; gl += nb) {
        const int base = grid_pos(gl, side == 0 ? H : W, step);  // first image row (column) of the patches
        for (int p0 = 0; p0 < len; p0 += COV_CH) {
            const int np = min(COV_CH, len - p0);
            if (side == 0) {  // rows base .. base + 7 of every channel, columns p0 .. p0 + np - 1
                for (int e = t; e < NL * COV_CH; e += blockDim.x) {
                    const int ln = e / COV_CH, q = e - ln * COV_CH;
                    const int c = ln >> 3, off = ln & 7;
                    sl[ln][q] = q < np ? __ldg(img + c * HW + (size_t)(base + off) * W + p0 + q) : 0.f;
                }
            } else {  // columns base .. base + 7 of every channel, rows p0 .. p0 + np - 1
                for (int e = t; e < NL * COV_CH; e += blockDim.x) {
                    const int q = e / NL, ln = e - q * NL;
                    const int c = ln >> 3, off = ln & 7;
                    sl[ln][q] = q < np ? __ldg(img + c * HW + (size_t)(p0 + q) * W + base + off) : 0.f;
                }
            }
            for (int q = t; q < COV_CH; q += blockDim.x) sw[q] = q < np ? (float)cover_count(p0 + q, len, step) : 0.f;
            __syncthreads();
            if (valid) {
                const float4 *X = reinterpret_cast<const float4 *>(sl[t0 * PS + a]);
                const float4 *Y = reinterpret_cast<const float4 *>(sl[t1 * PS + b]);
                const float4 *Wt = reinterpret_cast<const float4 *>(sw);
                float hi = 0.f, lo = 0.f;
                for (int q4 = 0; q4 < (np + 3) / 4; ++q4) {
                    const float4 x = X[q4], y = Y[q4], w = Wt[q4];
                    df_add(hi, lo, __fmul_rn(x.x, w.x), y.x);
                    df_add(hi, lo, __fmul_rn(x.y, w.y), y.y);
                    df_add(hi, lo, __fmul_rn(x.z, w.z), y.z);
                    df_add(hi, lo, __fmul_rn(x.w, w.w), y.w);
                }
                acc += (double)hi + (double)lo;
            }
            __syncthreads();
        }
    }
    if (valid) partials[((size_t)(side == 0 ? 0 : nb_r) + blockIdx.x) * PER + t] = acc;
}

// Sum of the blocks' partial sums, one warp per entry, fixed reduction tree.
template <int C>
__global__ void __launch_bounds__(256) k_cov_sum(const double *__restrict__ partials, int nb_r, int nb_c,
                                                 double *__restrict__ totals) {
    constexpr int NT = CovCfg<C>::NT, PER = CovCfg<C>::PER;
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= NT) return;
    const int side = t / PER, e = t - side * PER;
    const int nblocks = side == 0 ? nb_r : nb_c;
    const double *part = partials + (size_t)(side == 0 ? 0 : nb_r) * PER + e;
    double sum = 0.0;
    for (int bl = lane; bl < nblocks; bl += 32) sum += part[(size_t)bl * PER];
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

// Rotation pair i (0..3) of round `round` (0..6) of the parallel cyclic
// ordering: the 8 indices sit on a circle of 7 around a fixed index 0.
__device__ __forceinline__ void jac_pair(int i, int round, int &p, int &q) {
    const int L0 = (i == 0) ? 0 : 1 + ((i - 1 + round) % 7);
    const int L1 = 1 + ((6 - i + round) % 7);
    p = min(L0, L1);
    q = max(L0, L1);
}

// Applies the 4 rotations of one round to A (both sides) and V (right side).
// Rotation i acts on columns p, q (old values x, y) as p <- c x - s conj(e) y,
// q <- s x + c conj(e) y, and by its adjoint on rows p, q.
template <typename T>
__device__ __forceinline__ void jac_apply(T *Ar, T *Ai, T *Vr, T *Vi, const T *pc, const T *ps_, const T *per,
                                          const T *pei, const int *pp, const int *pq, int lane) {
    const int i = lane >> 3, k = lane & 7;
    const int p = pp[i], q = pq[i];
    const T c = pc[i], s = ps_[i], er = per[i], ei = pei[i];
    {   // columns: A <- A J
        const T xr = Ar[k * 8 + p], xi = Ai[k * 8 + p];
        const T yr = Ar[k * 8 + q], yi = Ai[k * 8 + q];
        const T zr = er * yr + ei * yi, zi = er * yi - ei * yr;  // conj(e) * y
        Ar[k * 8 + p] = c * xr - s * zr;
        Ai[k * 8 + p] = c * xi - s * zi;
        Ar[k * 8 + q] = s * xr + c * zr;
        Ai[k * 8 + q] = s * xi + c * zi;
    }
    __syncwarp();
    {   // rows: A <- J^H A
        const T xr = Ar[p * 8 + k], xi = Ai[p * 8 + k];
        const T yr = Ar[q * 8 + k], yi = Ai[q * 8 + k];
        const T zr = er * yr - ei * yi, zi = er * yi + ei * yr;  // e * y
        Ar[p * 8 + k] = c * xr - s * zr;
        Ai[p * 8 + k] = c * xi - s * zi;
        Ar[q * 8 + k] = s * xr + c * zr;
        Ai[q * 8 + k] = s * xi + c * zi;
    }
    __syncwarp();
    {   // eigenvectors: V <- V J
        const T xr = Vr[k * 8 + p], xi = Vi[k * 8 + p];
        const T yr = Vr[k * 8 + q], yi = Vi[k * 8 + q];
        const T zr = er * yr + ei * yi, zi = er * yi - ei * yr;
        Vr[k * 8 + p] = c * xr - s * zr;
        Vi[k * 8 + p] = c * xi - s * zi;
        Vr[k * 8 + q] = s * xr + c * zr;
        Vi[k * 8 + q] = s * xi + c * zi;
    }
    __syncwarp();
}

// Rotation (phase e, cosine c, sine s) that zeroes a_pq, in FP32: a_pq is made
// real by e = a_pq / |a_pq|, then the real Jacobi rotation
// t = sgn(th) / (|th| + sqrt(th^2 + 1)), th = (a_qq - a_pp) / (2 |a_pq|).
__device__ __forceinline__ bool jac_angle32(float app, float aqq, float zr, float zi, float &c, float &s, float &er,
                                            float &ei) {
    const float r2 = zr * zr + zi * zi;
    c = 1.f;
    s = 0.f;
    er = 1.f;
    ei = 0.f;
    if (!(r2 > 0.f) || !(r2 > 1e-30f * (app * app + aqq * aqq))) return false;
    const float r = sqrtf(r2);
    er = zr / r;
    ei = zi / r;
    const float th = (aqq - app) / (2.f * r);
    const float tt = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
    c = rsqrtf(fmaf(tt, tt, 1.f));
    s = tt * c;
    return true;
}

// ---- double-float (float pair h + l, |l| <= ulp(h)/2) arithmetic for the
//      refinement phase: error-free transformations (Knuth's TwoSum, TwoProd
//      by fma) with explicit roundings so that no contraction merges steps.
//      About 2^-48 relative per operation, on the FP32 pipes.
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl df_make(float h) { return {h, 0.f}; }
__device__ __forceinline__ dfl df_renorm(float s, float e) {  // |s| >= |e| or s == 0
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bv = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
    return df_renorm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_renorm(p, e);
}
__device__ __forceinline__ dfl df_scale(dfl a, float pow2) { return {a.h * pow2, a.l * pow2}; }  // exact
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.h + (double)a.l; }

// (X^H Y)[a][b] (HX) or (X Y)[a][b] of 8x8 complex double-float matrices.
template <bool HX>
__device__ __forceinline__ void cmm8(const dfl *Xr, const dfl *Xi, const dfl *Yr, const dfl *Yi, int e, dfl &cr,
                                     dfl &ci) {
    const int a = e >> 3, b = e & 7;
    dfl sr = df_make(0.f), si = df_make(0.f);
#pragma unroll 2
    for (int k = 0; k < 8; ++k) {
        const dfl xr = HX ? Xr[k * 8 + a] : Xr[a * 8 + k];
        const dfl xi = HX ? -Xi[k * 8 + a] : Xi[a * 8 + k];
        const dfl yr = Yr[k * 8 + b], yi = Yi[k * 8 + b];
        sr = sr + (xr * yr - xi * yi);
        si = si + (xr * yi + xi * yr);
    }
    cr = sr;
    ci = si;
}

// The 4 rotations of one round applied to A (both sides) and V (right side)
// in double-float; same rotation as jac_apply.
__device__ __forceinline__ void jac_apply_df(dfl *Ar, dfl *Ai, dfl *Vr, dfl *Vi, const dfl *pc, const dfl *ps_,
                                             const dfl *per, const dfl *pei, const int *pp, const int *pq, int lane) {
    const int i = lane >> 3, k = lane & 7;
    const int p = pp[i], q = pq[i];
    const dfl c = pc[i], s = ps_[i], er = per[i], ei = pei[i];
    {   // columns: A <- A J
        const dfl xr = Ar[k * 8 + p], xi = Ai[k * 8 + p];
        const dfl yr = Ar[k * 8 + q], yi = Ai[k * 8 + q];
        const dfl zr = er * yr + ei * yi, zi = er * yi - ei * yr;  // conj(e) * y
        Ar[k * 8 + p] = c * xr - s * zr;
        Ai[k * 8 + p] = c * xi - s * zi;
        Ar[k * 8 + q] = s * xr + c * zr;
        Ai[k * 8 + q] = s * xi + c * zi;
    }
    __syncwarp();
    {   // rows: A <- J^H A
        const dfl xr = Ar[p * 8 + k], xi = Ai[p * 8 + k];
        const dfl yr = Ar[q * 8 + k], yi = Ai[q * 8 + k];
        const dfl zr = er * yr - ei * yi, zi = er * yi + ei * yr;  // e * y
        Ar[p * 8 + k] = c * xr - s * zr;
        Ai[p * 8 + k] = c * xi - s * zi;
        Ar[q * 8 + k] = s * xr + c * zr;
        Ai[q * 8 + k] = s * xi + c * zi;
    }
    __syncwarp();
    {   // eigenvectors: V <- V J
        const dfl xr = Vr[k * 8 + p], xi = Vi[k * 8 + p];
        const dfl yr = Vr[k * 8 + q], yi = Vi[k * 8 + q];
        const dfl zr = er * yr + ei * yi, zi = er * yi - ei * yr;
        Vr[k * 8 + p] = c * xr - s * zr;
        Vi[k * 8 + p] = c * xi - s * zi;
        Vr[k * 8 + q] = s * xr + c * zr;
        Vi[k * 8 + q] = s * xi + c * zi;
    }
    __syncwarp();
}

// One 8x8 Hermitian eigenproblem per block (one warp), in two phases, on the
// matrix scaled by an exact power of two (eigenvectors are unchanged).
// Phase 1: cyclic parallel Jacobi (4 disjoint rotations per round, 7 rounds
// per sweep) in FP32 until the off-diagonal mass is below 1e-12 of the
// diagonal's.  Phase 2, in double-float (GB300's FP64 rate is too low for a
// latency-bound solver): the FP32 eigenvectors are made unitary by two
// Newton-Schulz steps V <- V (3I - V^H V) / 2, the matrix is rotated into that
// basis (B = V^H A V, Hermitian part), and Jacobi continues on B: each angle is
// computed in FP32 from the entries scaled so that |b_pq| ~ 1, then the phase
// and (c, s) are renormalised by two Newton steps of 1/sqrt(x) at x ~ 1, so
// every applied rotation is unitary to double-float precision.  B starts
// within FP32 round-off of diagonal, so one or two sweeps bring the
// off-diagonal mass below 1e-26 of the diagonal's.
template <int C>
__global__ void __launch_bounds__(32) k_jacobi(const double *__restrict__ totals, int nmat, double *__restrict__ b64,
                                               float *__restrict__ b32, double *__restrict__ eig) {
    __shared__ double Ad_r[64], Ad_i[64];
    __shared__ dfl Ar[64], Ai[64], Vr[64], Vi[64], Tr[64], Ti[64];
    __shared__ float Fr[64], Fi[64], Gr[64], Gi[64];
    __shared__ dfl pc[4], ps_[4], per[4], pei[4];
    __shared__ float fc[4], fs[4], fer[4], fei[4];
    __shared__ int pp[4], pq[4];
    __shared__ int perm[8];
    const int w = blockIdx.x, lane = threadIdx.x & 31;
    if (w >= nmat) return;
    double dmax = 0.0;
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
        Ad_r[e] = sr;
        Ad_i[e] = si;
        if (a == b) dmax = fmax(dmax, fabs(sr));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, o));
    int ex = 0;
    if (dmax > 0.0 && dmax < 1e300) frexp(dmax, &ex);
    __syncwarp();
    for (int e = lane; e < 64; e += 32) {
        const double xr = ldexp(Ad_r[e], -ex), xi = ldexp(Ad_i[e], -ex);  // exact scaling, |diag| < 1
        Fr[e] = (float)xr;
        Fi[e] = (float)xi;
        Ar[e] = {(float)xr, (float)(xr - (double)(float)xr)};
        Ai[e] = {(float)xi, (float)(xi - (double)(float)xi)};
        Gr[e] = ((e >> 3) == (e & 7)) ? 1.f : 0.f;
        Gi[e] = 0.f;
    }
    __syncwarp();
    // ---- phase 1, FP32
    for (int sweep = 0; sweep < 20; ++sweep) {
        float off = 0.f, dia = 0.f;
        for (int e = lane; e < 64; e += 32) {
            const float m2 = Fr[e] * Fr[e] + Fi[e] * Fi[e];
            if ((e >> 3) == (e & 7)) dia += m2;
            else off += m2;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(FULL, off, o);
            dia += __shfl_xor_sync(FULL, dia, o);
        }
        if (off <= 1e-12f * dia || off == 0.f) break;
        for (int round = 0; round < 7; ++round) {
            if (lane < 4) {
                int p, q;
                jac_pair(lane, round, p, q);
                float c, s, er, ei;
                jac_angle32(Fr[p * 9], Fr[q * 9], Fr[p * 8 + q], Fi[p * 8 + q], c, s, er, ei);
                fc[lane] = c;
                fs[lane] = s;
                fer[lane] = er;
                fei[lane] = ei;
                pp[lane] = p;
                pq[lane] = q;
            }
            __syncwarp();
            jac_apply<float>(Fr, Fi, Gr, Gi, fc, fs, fer, fei, pp, pq, lane);
        }
    }
    // ---- phase 2, double-float: unitary V from the FP32 eigenvectors
    for (int e = lane; e < 64; e += 32) {
        Vr[e] = df_make(Gr[e]);
        Vi[e] = df_make(Gi[e]);
    }
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
        dfl tr0, ti0, tr1, ti1;
        cmm8<true>(Vr, Vi, Vr, Vi, lane, tr0, ti0);
        cmm8<true>(Vr, Vi, Vr, Vi, lane + 32, tr1, ti1);
        // M = (3I - V^H V) / 2
        const dfl half = df_make(0.5f), three_half = df_make(1.5f);
        Tr[lane] = (((lane >> 3) == (lane & 7)) ? three_half : df_make(0.f)) - half * tr0;
        Ti[lane] = -(half * ti0);
        Tr[lane + 32] = ((((lane + 32) >> 3) == (lane & 7)) ? three_half : df_make(0.f)) - half * tr1;
        Ti[lane + 32] = -(half * ti1);
        __syncwarp();
        cmm8<false>(Vr, Vi, Tr, Ti, lane, tr0, ti0);
        cmm8<false>(Vr, Vi, Tr, Ti, lane + 32, tr1, ti1);
        __syncwarp();
        Vr[lane] = tr0;
        Vi[lane] = ti0;
        Vr[lane + 32] = tr1;
        Vi[lane + 32] = ti1;
        __syncwarp();
    }
    {   // B = V^H (A V), Hermitian part
        dfl tr0, ti0, tr1, ti1;
        cmm8<false>(Ar, Ai, Vr, Vi, lane, tr0, ti0);
        cmm8<false>(Ar, Ai, Vr, Vi, lane + 32, tr1, ti1);
        Tr[lane] = tr0;
        Ti[lane] = ti0;
        Tr[lane + 32] = tr1;
        Ti[lane + 32] = ti1;
        __syncwarp();
        cmm8<true>(Vr, Vi, Tr, Ti, lane, tr0, ti0);
        cmm8<true>(Vr, Vi, Tr, Ti, lane + 32, tr1, ti1);
        __syncwarp();
        Tr[lane] = tr0;
        Ti[lane] = ti0;
        Tr[lane + 32] = tr1;
        Ti[lane + 32] = ti1;
        __syncwarp();
        for (int e = lane; e < 64; e += 32) {
            const int a = e >> 3, b = e & 7, t = b * 8 + a;
            Ar[e] = df_scale(Tr[e] + Tr[t], 0.5f);
            Ai[e] = (a == b) ? df_make(0.f) : df_scale(Ti[e] - Ti[t], 0.5f);
        }
        __syncwarp();
    }
    // Sweeps until the off-diagonal mass is below 1e-26 of the diagonal's
    // (relative 3e-13 in norm); 24 at most.
    for (int sweep = 0; sweep < 24; ++sweep) {
        float off = 0.f, dia = 0.f;
        for (int e = lane; e < 64; e += 32) {
            const float m2 = Ar[e].h * Ar[e].h + Ai[e].h * Ai[e].h;
            if ((e >> 3) == (e & 7)) dia += m2;
            else off += m2;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(FULL, off, o);
            dia += __shfl_xor_sync(FULL, dia, o);
        }
        if (off <= 1e-26f * dia || off == 0.f) break;
        for (int round = 0; round < 7; ++round) {
            if (lane < 4) {
                int p, q;
                jac_pair(lane, round, p, q);
                const dfl zr = Ar[p * 8 + q], zi = Ai[p * 8 + q];
                dfl c = df_make(1.f), s = df_make(0.f), er = df_make(1.f), ei = df_make(0.f);
                const float zm = fmaxf(fabsf(zr.h), fabsf(zi.h));
                const float app = Ar[p * 9].h, aqq = Ar[q * 9].h;
                if (zm > 0.f && zm > 1e-15f * fmaxf(fabsf(app), fabsf(aqq))) {
                    // FP32 angle from the entries scaled so that |b_pq| ~ 1 (exact
                    // power-of-two scaling; the test above bounds |b_pp|, |b_qq|)
                    int ez = 0;
                    frexpf(zm, &ez);
                    float cf, sf, erf_, eif;
                    jac_angle32(ldexpf(app, -ez), ldexpf(aqq, -ez), ldexpf(zr.h, -ez), ldexpf(zi.h, -ez), cf, sf,
                                erf_, eif);
                    c = df_make(cf);
                    s = df_make(sf);
                    er = df_make(erf_);
                    ei = df_make(eif);
                    const dfl three_half = df_make(1.5f), half = df_make(0.5f);
#pragma unroll
                    for (int it = 0; it < 2; ++it) {  // x -> x (3 - |x|^2) / 2
                        const dfl ne = three_half - half * (er * er + ei * ei);
                        er = er * ne;
                        ei = ei * ne;
                        const dfl nc = three_half - half * (c * c + s * s);
                        c = c * nc;
                        s = s * nc;
                    }
                }
                pc[lane] = c;
                ps_[lane] = s;
                per[lane] = er;
                pei[lane] = ei;
                pp[lane] = p;
                pq[lane] = q;
            }
            __syncwarp();
            jac_apply_df(Ar, Ai, Vr, Vi, pc, ps_, per, pei, pp, pq, lane);
        }
    }
    if (lane == 0) {
        int idx[8];
        for (int i = 0; i < 8; ++i) idx[i] = i;
        for (int i = 0; i < 8; ++i)
            for (int jj = i + 1; jj < 8; ++jj)
                if (df_to_double(Ar[idx[jj] * 9]) < df_to_double(Ar[idx[i] * 9])) {
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
        const double vr = df_to_double(Vr[src]), vi = df_to_double(Vi[src]);
        b64[((size_t)w * 64 + e) * 2] = vr;
        b64[((size_t)w * 64 + e) * 2 + 1] = vi;
        b32[((size_t)w * 64 + e) * 2] = (float)vr;
        b32[((size_t)w * 64 + e) * 2 + 1] = (float)vi;
    }
    if (lane < 8) eig[w * 8 + lane] = ldexp(df_to_double(Ar[perm[lane] * 9]), ex);
}

}  // namespace

size_t cov_partial_count(const Geom &g) {
    const int nb = std::min(g.ny, COV_BLOCKS) + std::min(g.nx, COV_BLOCKS);
    const int per = (g.C == 3) ? CovCfg<3>::PER : CovCfg<1>::PER;
    return (size_t)nb * per + 2 * per;  // per-block partial sums of both sides, then the totals
}

template <int C>
hts_status launch_basis_c(const float *img, const Geom &g, double *partials, double *b64, float *b32, double *eig,
                          cudaStream_t s) {
    constexpr int NT = CovCfg<C>::NT, PER = CovCfg<C>::PER;
    const int nb_r = std::min(g.ny, COV_BLOCKS), nb_c = std::min(g.nx, COV_BLOCKS);
    const int ns = C / 2 + 1;
    double *totals = partials + (size_t)(nb_r + nb_c) * PER;
    {
        KTimer kt("k_cov", s);
        k_cov<C><<<dim3(std::max(nb_r, nb_c), 2), CovCfg<C>::THREADS, 0, s>>>(img, g.H, g.W, g.step, g.ny, g.nx,
                                                                              nb_r, nb_c, partials);
    }
    if (hts_status st = check_launch("k_cov"); st != HTS_OK) return st;
    {
        KTimer kt("k_cov_sum", s);
        k_cov_sum<C><<<(NT * 32 + 255) / 256, 256, 0, s>>>(partials, nb_r, nb_c, totals);
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
