// Collaborative filtering and aggregation of Haar-tSVD (Eq. 19-21, Alg. 1
// steps 2-3) on sm_103a.
//
// Layout of the work: a warp holds G = 32/K groups (one for K = 32); lane
// (g, k) owns patch k of group g during the patch phases.  A group's
// coefficients live in shared memory as [stream e][patch k] with a padded
// row (K+1 floats) so that both the patch-major writes and the stream-major
// reads of the Haar phase are bank-conflict free.
//
//   patch phase   : gather the patch (FP32), unitary DFT along channels
//                   (c = 3), Shat^(j) = U^(j)^H Phat^(j) V^(j) per stored
//                   Fourier slice (Eq. 19, slice 3 = conj of slice 2);
//   stream phase  : fast Haar transform along the group axis in registers
//                   (Eq. 8 row order), hard threshold |s| >= tau (Eq. 20;
//                   modulus for complex coefficients), inverse Haar;
//   patch phase   : U Shat V^H, inverse DFT (Eq. 21), and aggregation as
//                   exact fixed-point integer sums (value * 2^24 rounded to
//                   int64) plus an integer weight per pixel, so the result
//                   does not depend on the order of the additions.
//
// Threshold decisions are taken in FP64 where FP32 cannot certify them: the
// FP32 coefficient of a group G differs from the exact one by at most
// 160 u ||G||_F (gray) / 320 u ||G||_F (colour) (twice the sum of the
// per-stage bounds of the DFT, the two 8x8 products with rounded bases and
// the Haar butterflies; the stages are unitary so errors do not grow).  A
// group with any coefficient inside that band around tau is not aggregated
// by the main pass; a second pass recomputes it, evaluates each in-band
// coefficient in FP64 from the input pixels and the FP64 basis (one warp per
// coefficient), and takes the decision there.
#include "hts_internal.h"

namespace hts {
namespace {

constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24
constexpr unsigned FULL = 0xffffffffu;
constexpr float R2F = 0.70710678118654752f;     // 1/sqrt(2)
constexpr float K3F = 0.57735026918962576f;     // 1/sqrt(3)
constexpr float S3H = 0.86602540378443865f;     // sqrt(3)/2
constexpr int QCAP = 64;                        // in-band queue of the exact pass

// Basis in shared memory, float32: for slice 0 U, V, U^T, V^T (row-major
// 8x8); for slice 1 the same for the real and imaginary parts.
struct SBasis {
    float u0[64], v0[64], u0t[64], v0t[64];
    float u1r[64], u1i[64], v1r[64], v1i[64];
    float u1rt[64], u1it[64], v1rt[64], v1it[64];
};

struct FilterArgs {
    const float *img;
    int H, W, step, nx, nref;
    const int32_t *idx;
    const double *b64;
    const float *b32;
    long long *acc;
    int *wcount;
    int32_t *redo;
    DevState *st;
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// ---------------------------------------------------------------- basis

template <int C>
__device__ void load_basis(SBasis &sb, const float *__restrict__ b32) {
    // b32: [j][m][a][i][2]
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        const int a = t >> 3, i = t & 7;
        const float *s0u = b32 + ((0 * 2 + 0) * 64 + t) * 2;
        const float *s0v = b32 + ((0 * 2 + 1) * 64 + t) * 2;
        sb.u0[t] = s0u[0];
        sb.v0[t] = s0v[0];
        sb.u0t[i * 8 + a] = s0u[0];
        sb.v0t[i * 8 + a] = s0v[0];
        if (C == 3) {
            const float *s1u = b32 + ((1 * 2 + 0) * 64 + t) * 2;
            const float *s1v = b32 + ((1 * 2 + 1) * 64 + t) * 2;
            sb.u1r[t] = s1u[0];
            sb.u1i[t] = s1u[1];
            sb.v1r[t] = s1v[0];
            sb.v1i[t] = s1v[1];
            sb.u1rt[i * 8 + a] = s1u[0];
            sb.u1it[i * 8 + a] = s1u[1];
            sb.v1rt[i * 8 + a] = s1v[0];
            sb.v1it[i * 8 + a] = s1v[1];
        }
    }
}

// ---------------------------------------------------- 8x8 products (FP32)

// In place: P <- U^T P V (real).  P row-major 8x8.
__device__ __forceinline__ void fwd_real(float (&P)[64], const float *U, const float *V) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {  // T row a = P row a * V
        float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float4 v0 = ld4(V + b * 8), v1 = ld4(V + b * 8 + 4);
            const float p = P[a * 8 + b];
            t[0] = fmaf(p, v0.x, t[0]); t[1] = fmaf(p, v0.y, t[1]);
            t[2] = fmaf(p, v0.z, t[2]); t[3] = fmaf(p, v0.w, t[3]);
            t[4] = fmaf(p, v1.x, t[4]); t[5] = fmaf(p, v1.y, t[5]);
            t[6] = fmaf(p, v1.z, t[6]); t[7] = fmaf(p, v1.w, t[7]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) P[a * 8 + j] = t[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // S column j = U^T * T column j
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float4 u0 = ld4(U + a * 8), u1 = ld4(U + a * 8 + 4);
            const float t = P[a * 8 + j];
            s[0] = fmaf(u0.x, t, s[0]); s[1] = fmaf(u0.y, t, s[1]);
            s[2] = fmaf(u0.z, t, s[2]); s[3] = fmaf(u0.w, t, s[3]);
            s[4] = fmaf(u1.x, t, s[4]); s[5] = fmaf(u1.y, t, s[5]);
            s[6] = fmaf(u1.z, t, s[6]); s[7] = fmaf(u1.w, t, s[7]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) P[i * 8 + j] = s[i];
    }
}

// In place: S <- U S V^T (real), i.e. the inverse of fwd_real for unitary U, V.
// Ut = U^T, Vt = V^T row-major.
__device__ __forceinline__ void inv_real(float (&S)[64], const float *Ut, const float *Vt) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // T column j = U * S column j
        float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 c0 = ld4(Ut + i * 8), c1 = ld4(Ut + i * 8 + 4);  // column i of U
            const float s = S[i * 8 + j];
            t[0] = fmaf(c0.x, s, t[0]); t[1] = fmaf(c0.y, s, t[1]);
            t[2] = fmaf(c0.z, s, t[2]); t[3] = fmaf(c0.w, s, t[3]);
            t[4] = fmaf(c1.x, s, t[4]); t[5] = fmaf(c1.y, s, t[5]);
            t[6] = fmaf(c1.z, s, t[6]); t[7] = fmaf(c1.w, s, t[7]);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) S[a * 8 + j] = t[a];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {  // P row a = T row a * V^T
        float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 c0 = ld4(Vt + j * 8), c1 = ld4(Vt + j * 8 + 4);  // column j of V
            const float t = S[a * 8 + j];
            p[0] = fmaf(t, c0.x, p[0]); p[1] = fmaf(t, c0.y, p[1]);
            p[2] = fmaf(t, c0.z, p[2]); p[3] = fmaf(t, c0.w, p[3]);
            p[4] = fmaf(t, c1.x, p[4]); p[5] = fmaf(t, c1.y, p[5]);
            p[6] = fmaf(t, c1.z, p[6]); p[7] = fmaf(t, c1.w, p[7]);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) S[a * 8 + b] = p[b];
    }
}

// In place: (Pr, Pi) <- U^H P V (complex).
__device__ __forceinline__ void fwd_cplx(float (&Pr)[64], float (&Pi)[64], const SBasis &sb) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        float tr[8], ti[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { tr[j] = 0.f; ti[j] = 0.f; }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float pr = Pr[a * 8 + b], pi = Pi[a * 8 + b];
            const float4 r0 = ld4(sb.v1r + b * 8), r1 = ld4(sb.v1r + b * 8 + 4);
            const float4 i0 = ld4(sb.v1i + b * 8), i1 = ld4(sb.v1i + b * 8 + 4);
            const float vr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            const float vi[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                tr[j] = fmaf(pr, vr[j], tr[j]);
                tr[j] = fmaf(-pi, vi[j], tr[j]);
                ti[j] = fmaf(pr, vi[j], ti[j]);
                ti[j] = fmaf(pi, vr[j], ti[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) { Pr[a * 8 + j] = tr[j]; Pi[a * 8 + j] = ti[j]; }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // S col j = U^H T col j
        float sr[8], si[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { sr[i] = 0.f; si[i] = 0.f; }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float tr = Pr[a * 8 + j], ti = Pi[a * 8 + j];
            const float4 r0 = ld4(sb.u1r + a * 8), r1 = ld4(sb.u1r + a * 8 + 4);
            const float4 i0 = ld4(sb.u1i + a * 8), i1 = ld4(sb.u1i + a * 8 + 4);
            const float ur[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            const float ui[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {  // conj(u) * t
                sr[i] = fmaf(ur[i], tr, sr[i]);
                sr[i] = fmaf(ui[i], ti, sr[i]);
                si[i] = fmaf(ur[i], ti, si[i]);
                si[i] = fmaf(-ui[i], tr, si[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) { Pr[i * 8 + j] = sr[i]; Pi[i * 8 + j] = si[i]; }
    }
}

// In place: (Sr, Si) <- U S V^H (complex), inverse of fwd_cplx.
__device__ __forceinline__ void inv_cplx(float (&Sr)[64], float (&Si)[64], const SBasis &sb) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // T col j = U S col j
        float tr[8], ti[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) { tr[a] = 0.f; ti[a] = 0.f; }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float sr = Sr[i * 8 + j], si = Si[i * 8 + j];
            const float4 r0 = ld4(sb.u1rt + i * 8), r1 = ld4(sb.u1rt + i * 8 + 4);
            const float4 i0 = ld4(sb.u1it + i * 8), i1 = ld4(sb.u1it + i * 8 + 4);
            const float ur[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            const float ui[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                tr[a] = fmaf(ur[a], sr, tr[a]);
                tr[a] = fmaf(-ui[a], si, tr[a]);
                ti[a] = fmaf(ur[a], si, ti[a]);
                ti[a] = fmaf(ui[a], sr, ti[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) { Sr[a * 8 + j] = tr[a]; Si[a * 8 + j] = ti[a]; }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {  // P row a = T row a V^H
        float pr[8], pi[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) { pr[b] = 0.f; pi[b] = 0.f; }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float tr = Sr[a * 8 + j], ti = Si[a * 8 + j];
            const float4 r0 = ld4(sb.v1rt + j * 8), r1 = ld4(sb.v1rt + j * 8 + 4);
            const float4 i0 = ld4(sb.v1it + j * 8), i1 = ld4(sb.v1it + j * 8 + 4);
            const float vr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            const float vi[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
            for (int b = 0; b < 8; ++b) {  // t * conj(v)
                pr[b] = fmaf(tr, vr[b], pr[b]);
                pr[b] = fmaf(ti, vi[b], pr[b]);
                pi[b] = fmaf(ti, vr[b], pi[b]);
                pi[b] = fmaf(-tr, vi[b], pi[b]);
            }
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) { Sr[a * 8 + b] = pr[b]; Si[a * 8 + b] = pi[b]; }
    }
}

// --------------------------------------------------------- Haar (Eq. 8)

// Forward: output row order of Eq. 8 (row 0 = sum / sqrt K, then the
// coarse-to-fine difference rows, the finest K/2 differences last).
template <int K>
__device__ __forceinline__ void haar_fwd(float (&x)[K]) {
#pragma unroll
    for (int n = K; n >= 2; n >>= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[i] = (x[2 * i] + x[2 * i + 1]) * R2F;
            t[n / 2 + i] = (x[2 * i] - x[2 * i + 1]) * R2F;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

template <int K>
__device__ __forceinline__ void haar_inv(float (&x)[K]) {
#pragma unroll
    for (int n = 2; n <= K; n <<= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[2 * i] = (x[i] + x[n / 2 + i]) * R2F;
            t[2 * i + 1] = (x[i] - x[n / 2 + i]) * R2F;
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

// Entry (h, k) of the Haar matrix of Eq. 8, in FP64.
__device__ __forceinline__ double haar_entry(int K, int h, int k) {
    if (h == 0) return rsqrt((double)K);
    int l = 31 - __clz(h);  // 2^l <= h < 2^(l+1)
    int L = K >> l;
    int i = h - (1 << l);
    if (k < i * L || k >= (i + 1) * L) return 0.0;
    const double m = rsqrt((double)L);
    return (k < i * L + L / 2) ? m : -m;
}

// --------------------------------------------------- threshold decision

// 0 = drop, 1 = keep, 2 = undecided in FP32 (inside the guard band).
__device__ __forceinline__ int decide(float mag, float tau, float band) {
    if (tau <= 0.f) return 1;
    const float b = band + 3.f * U32 * mag;
    if (mag - b >= tau) return 1;
    if (mag + b < tau) return 0;
    return 2;
}

// ------------------------------------------------------ exact coefficient

// FP64 value of Haar coefficient (h, slice j, element e = i*8+jj) of group
// r, evaluated from the input pixels and the FP64 basis by the whole warp.
template <int C>
__device__ void exact_coef(const FilterArgs &a, const int32_t *grp, int K, int h, int j, int e, int lane,
                           double &re, double &im) {
    const int i = e >> 3, jj = e & 7;
    const size_t HW = (size_t)a.H * a.W;
    int k0 = 0, k1 = K;
    if (h > 0) {
        const int l = 31 - __clz(h), L = K >> l, ii = h - (1 << l);
        k0 = ii * L;
        k1 = k0 + L;
    }
    const double *U = a.b64 + (size_t)((j * 2 + 0) * 64) * 2;
    const double *V = a.b64 + (size_t)((j * 2 + 1) * 64) * 2;
    const double k3 = 0.57735026918962576451;  // 1/sqrt(3)
    const double s3h = 0.86602540378443864676; // sqrt(3)/2
    double sr = 0.0, si = 0.0;
    const int nunits = (k1 - k0) * 8;
    for (int u = lane; u < nunits; u += 32) {
        const int k = k0 + (u >> 3), arow = u & 7;
        const int pos = grp[k];
        const int y = pos / a.W, x = pos - (pos / a.W) * a.W;
        double tr = 0.0, ti = 0.0;  // (Phat row arow) * V column jj
        for (int b = 0; b < 8; ++b) {
            const size_t o = (size_t)(y + arow) * a.W + x + b;
            double pr, pi;
            if (C == 1) {
                pr = (double)__ldg(a.img + o);
                pi = 0.0;
            } else {
                const double R = (double)__ldg(a.img + o), G = (double)__ldg(a.img + HW + o),
                             B = (double)__ldg(a.img + 2 * HW + o);
                if (j == 0) {
                    pr = ((R + G) + B) * k3;
                    pi = 0.0;
                } else {
                    pr = (R - 0.5 * (G + B)) * k3;
                    pi = (B - G) * (s3h * k3);
                }
            }
            const double vr = V[(b * 8 + jj) * 2], vi = V[(b * 8 + jj) * 2 + 1];
            tr += pr * vr - pi * vi;
            ti += pr * vi + pi * vr;
        }
        const double ur = U[(arow * 8 + i) * 2], ui = U[(arow * 8 + i) * 2 + 1];
        const double hv = haar_entry(K, h, k);
        sr += hv * (ur * tr + ui * ti);  // conj(u) * t
        si += hv * (ur * ti - ui * tr);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sr += __shfl_xor_sync(FULL, sr, o);
        si += __shfl_xor_sync(FULL, si, o);
    }
    re = sr;
    im = si;
}

// ---------------------------------------------------------------- kernel

template <int C>
struct Cfg {
    static constexpr int NCOEF = (C == 3) ? 192 : 64;  // real streams per patch
    static constexpr int IPG = (C == 3) ? 128 : 64;    // stream items per group
};

template <int C, int K, bool REDO>
__global__ void __launch_bounds__(64) k_filter(FilterArgs a) {
    constexpr int G = REDO ? 1 : (32 / K > 0 ? 32 / K : 1);
    constexpr int NCOEF = Cfg<C>::NCOEF;
    constexpr int IPG = Cfg<C>::IPG;
    constexpr int ROW = K + 1;
    constexpr int GS0 = NCOEF * ROW;
    constexpr int GS = GS0 + ((K - GS0 % 32) % 32 + 32) % 32;  // group stride = K (mod 32)
    constexpr int NWARPS = 2;
    constexpr int NMASK = (NCOEF * K + 31) / 32;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SBasis &sb = *reinterpret_cast<SBasis *>(smem_raw);
    float *wsm = reinterpret_cast<float *>(smem_raw + sizeof(SBasis));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *coef = wsm + warp * (G * GS + 2 * G + (REDO ? NMASK + QCAP + 2 : 0));
    float *gband = coef + G * GS;            // per-group guard band
    int *gflag = reinterpret_cast<int *>(gband + G);
    unsigned *mask = reinterpret_cast<unsigned *>(gflag + G);  // REDO: decided coefficients
    int *queue = reinterpret_cast<int *>(mask + NMASK);        // REDO: in-band queue
    int *qcount = queue + QCAP;

    load_basis<C>(sb, a.b32);
    __syncthreads();

    const float tau = a.st->tau32;
    const double tau64 = a.st->tau;
    const int gl = (REDO || K >= 32) ? 0 : (lane / K);
    const int k = lane % K;
    const size_t HW = (size_t)a.H * a.W;

    int nunits;
    if (REDO) nunits = *(volatile int *)&a.st->filter_redo;
    else nunits = (a.nref + G - 1) / G;

    for (int wu = blockIdx.x * NWARPS + warp; wu < nunits; wu += gridDim.x * NWARPS) {
        int r;
        if (REDO) r = a.redo[wu];
        else r = wu * G + gl;
        const bool active = REDO ? (lane < K) : (r < a.nref);
        float *cg = coef + gl * GS;
        const int32_t *grp = a.idx + (size_t)((REDO || active) ? r : 0) * K;
        int py = 0, px = 0;
        float ss = 0.f;
        if (active) {
            const int pos = grp[k];
            py = pos / a.W;
            px = pos - py * a.W;
        }
        // ---- patch phase: forward projection per slice
        if (active) {
            const float *base = a.img + (size_t)py * a.W + px;
            float P[64];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const size_t o = (size_t)u * a.W + v;
                    if (C == 1) {
                        const float x = __ldg(base + o);
                        P[u * 8 + v] = x;
                        ss = fmaf(x, x, ss);
                    } else {
                        const float R = __ldg(base + o), Gc = __ldg(base + HW + o), B = __ldg(base + 2 * HW + o);
                        P[u * 8 + v] = ((R + Gc) + B) * K3F;
                        ss = fmaf(R, R, ss);
                        ss = fmaf(Gc, Gc, ss);
                        ss = fmaf(B, B, ss);
                    }
                }
            fwd_real(P, sb.u0, sb.v0);
#pragma unroll
            for (int e = 0; e < 64; ++e) cg[e * ROW + k] = P[e];
            if (C == 3) {
                float Pr[64], Pi[64];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const size_t o = (size_t)u * a.W + v;
                        const float R = __ldg(base + o), Gc = __ldg(base + HW + o), B = __ldg(base + 2 * HW + o);
                        Pr[u * 8 + v] = (R - 0.5f * (Gc + B)) * K3F;
                        Pi[u * 8 + v] = (B - Gc) * 0.5f;
                    }
                fwd_cplx(Pr, Pi, sb);
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    cg[(64 + e) * ROW + k] = Pr[e];
                    cg[(128 + e) * ROW + k] = Pi[e];
                }
            }
        }
        // group norm -> guard band
#pragma unroll
        for (int o = 1; o < K && o < 32; o <<= 1) ss += __shfl_xor_sync(FULL, ss, o);
        if (k == 0 && active) {
            const float gb = (C == 3 ? 320.f : 160.f) * U32 * sqrtf(ss) * 1.01f + 2.f * U32 * tau;
            gband[gl] = gb;
            gflag[gl] = 0;
        }
        if (REDO && lane == 0) {
            *qcount = 0;
            for (int q = 0; q < NMASK; ++q) mask[q] = 0u;
        }
        __syncwarp();

        // ---- stream phase: Haar, threshold, inverse Haar
        if (!REDO) {
#pragma unroll 1
            for (int t = lane; t < G * IPG; t += 32) {
                const int g = t / IPG, it = t - g * IPG;
                const int rg = wu * G + g;
                if (rg >= a.nref) continue;
                float *cgg = coef + g * GS;
                const float band = gband[g];
                int flag = 0;
                if (it < 64) {
                    float x[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) x[q] = cgg[it * ROW + q];
                    haar_fwd<K>(x);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        const int d = decide(fabsf(x[q]), tau, band);
                        flag |= (d == 2);
                        x[q] = (d == 0) ? 0.f : x[q];
                    }
                    haar_inv<K>(x);
#pragma unroll
                    for (int q = 0; q < K; ++q) cgg[it * ROW + q] = x[q];
                } else {
                    const int e = it - 64;
                    float xr[K], xi[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        xr[q] = cgg[(64 + e) * ROW + q];
                        xi[q] = cgg[(128 + e) * ROW + q];
                    }
                    haar_fwd<K>(xr);
                    haar_fwd<K>(xi);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        const float mag = sqrtf(xr[q] * xr[q] + xi[q] * xi[q]);
                        const int d = decide(mag, tau, band);
                        flag |= (d == 2);
                        if (d == 0) { xr[q] = 0.f; xi[q] = 0.f; }
                    }
                    haar_inv<K>(xr);
                    haar_inv<K>(xi);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        cgg[(64 + e) * ROW + q] = xr[q];
                        cgg[(128 + e) * ROW + q] = xi[q];
                    }
                }
                if (flag) gflag[g] = 1;
            }
        } else {
            // pass 1: forward Haar only; coefficients stay unthresholded
#pragma unroll 1
            for (int t = lane; t < IPG; t += 32) {
                float *cgg = coef;
                if (t < 64) {
                    float x[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) x[q] = cgg[t * ROW + q];
                    haar_fwd<K>(x);
#pragma unroll
                    for (int q = 0; q < K; ++q) cgg[t * ROW + q] = x[q];
                } else {
                    const int e = t - 64;
                    float xr[K], xi[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        xr[q] = cgg[(64 + e) * ROW + q];
                        xi[q] = cgg[(128 + e) * ROW + q];
                    }
                    haar_fwd<K>(xr);
                    haar_fwd<K>(xi);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        cgg[(64 + e) * ROW + q] = xr[q];
                        cgg[(128 + e) * ROW + q] = xi[q];
                    }
                }
            }
            __syncwarp();
            const float band = gband[0];
            // rounds: queue undecided in-band coefficients, decide them in FP64
            for (int round = 0; round < NCOEF * K; ++round) {
                if (lane == 0) *qcount = 0;
                __syncwarp();
                for (int t = lane; t < IPG * K; t += 32) {
                    const int it = t / K, q = t - it * K;
                    const int bit = it * K + q;
                    if (mask[bit >> 5] & (1u << (bit & 31))) continue;
                    float mag;
                    if (it < 64) mag = fabsf(coef[it * ROW + q]);
                    else {
                        const float xr = coef[(it) * ROW + q], xi = coef[(it + 64) * ROW + q];
                        mag = sqrtf(xr * xr + xi * xi);
                    }
                    if (decide(mag, tau, band) != 2) continue;
                    const int slot = atomicAdd(qcount, 1);
                    if (slot < QCAP) queue[slot] = t;
                }
                __syncwarp();
                const int nq = min(*qcount, QCAP);
                if (nq == 0) break;
                for (int s = 0; s < nq; ++s) {
                    const int t = queue[s];
                    const int it = t / K, q = t - it * K;
                    const int j = it < 64 ? 0 : 1;
                    const int e = it < 64 ? it : it - 64;
                    double re, im;
                    exact_coef<C>(a, grp, K, q, j, e, lane, re, im);
                    const double mag = (j == 0) ? fabs(re) : sqrt(re * re + im * im);
                    if (lane == 0) {
                        const int bit = it * K + q;
                        mask[bit >> 5] |= (1u << (bit & 31));
                        if (!(mag >= tau64)) {
                            if (it < 64) coef[it * ROW + q] = 0.f;
                            else { coef[it * ROW + q] = 0.f; coef[(it + 64) * ROW + q] = 0.f; }
                        }
                        atomicAdd(&a.st->filter_exact, 1);
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
            // pass 2: certain FP32 decisions for the rest, inverse Haar
#pragma unroll 1
            for (int t = lane; t < IPG; t += 32) {
                if (t < 64) {
                    float x[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        float v = coef[t * ROW + q];
                        const int bit = t * K + q;
                        const bool dec = mask[bit >> 5] & (1u << (bit & 31));
                        if (!dec && decide(fabsf(v), tau, band) == 0) v = 0.f;
                        x[q] = v;
                    }
                    haar_inv<K>(x);
#pragma unroll
                    for (int q = 0; q < K; ++q) coef[t * ROW + q] = x[q];
                } else {
                    const int e = t - 64;
                    float xr[K], xi[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        float vr = coef[(64 + e) * ROW + q], vi = coef[(128 + e) * ROW + q];
                        const int bit = t * K + q;
                        const bool dec = mask[bit >> 5] & (1u << (bit & 31));
                        if (!dec && decide(sqrtf(vr * vr + vi * vi), tau, band) == 0) { vr = 0.f; vi = 0.f; }
                        xr[q] = vr;
                        xi[q] = vi;
                    }
                    haar_inv<K>(xr);
                    haar_inv<K>(xi);
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        coef[(64 + e) * ROW + q] = xr[q];
                        coef[(128 + e) * ROW + q] = xi[q];
                    }
                }
            }
        }
        __syncwarp();

        // ---- flagged groups are finished by the exact pass
        bool agg = active;
        if (!REDO && active) {
            if (gflag[gl]) {
                agg = false;
                if (k == 0) {
                    const int pos = atomicAdd(&a.st->filter_redo, 1);
                    a.redo[pos] = r;
                }
            }
        }
        // ---- patch phase: inverse projection and aggregation
        if (agg) {
            float P[64];
#pragma unroll
            for (int e = 0; e < 64; ++e) P[e] = cg[e * ROW + k];
            inv_real(P, sb.u0t, sb.v0t);
            long long *acc0 = a.acc + (size_t)py * a.W + px;
            int *wc = a.wcount + (size_t)py * a.W + px;
            if (C == 1) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const size_t o = (size_t)u * a.W + v;
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + o),
                                  (unsigned long long)__float2ll_rn(P[u * 8 + v] * FIX_SCALE));
                        atomicAdd(wc + o, 1);
                    }
            } else {
#pragma unroll
                for (int e = 0; e < 64; ++e) cg[e * ROW + k] = P[e];
                float Pr[64], Pi[64];
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    Pr[e] = cg[(64 + e) * ROW + k];
                    Pi[e] = cg[(128 + e) * ROW + k];
                }
                inv_cplx(Pr, Pi, sb);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const int e = u * 8 + v;
                        const float p0 = cg[e * ROW + k];
                        const float R = (p0 + 2.f * Pr[e]) * K3F;
                        const float Gc = (p0 - Pr[e] - 2.f * S3H * Pi[e]) * K3F;
                        const float B = (p0 - Pr[e] + 2.f * S3H * Pi[e]) * K3F;
                        const size_t o = (size_t)u * a.W + v;
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + o),
                                  (unsigned long long)__float2ll_rn(R * FIX_SCALE));
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + HW + o),
                                  (unsigned long long)__float2ll_rn(Gc * FIX_SCALE));
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + 2 * HW + o),
                                  (unsigned long long)__float2ll_rn(B * FIX_SCALE));
                        atomicAdd(wc + o, 1);
                    }
            }
        }
        __syncwarp();
    }
}

// out = sum / (2^24 * weight)
__global__ void k_normalize(const long long *__restrict__ acc, const int *__restrict__ wcount, float *__restrict__ out,
                            size_t HW, int C) {
    const size_t n = HW * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i % HW;
        const int w = wcount[p];
        out[i] = __ll2float_rn(acc[i]) / ((float)w * FIX_SCALE);
    }
}

template <int C, int K, bool REDO>
size_t filter_smem() {
    constexpr int G = REDO ? 1 : (32 / K > 0 ? 32 / K : 1);
    constexpr int NCOEF = Cfg<C>::NCOEF;
    constexpr int ROW = K + 1;
    constexpr int GS0 = NCOEF * ROW;
    constexpr int GS = GS0 + ((K - GS0 % 32) % 32 + 32) % 32;
    constexpr int NMASK = (NCOEF * K + 31) / 32;
    return sizeof(SBasis) + (size_t)2 * (G * GS + 2 * G + (REDO ? NMASK + QCAP + 2 : 0)) * 4;
}

template <int C, int K>
hts_status launch_ck(const FilterArgs &a, int nref, float *out, cudaStream_t s) {
    constexpr int G = (32 / K > 0 ? 32 / K : 1);
    const size_t sm0 = filter_smem<C, K, false>(), sm1 = filter_smem<C, K, true>();
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_filter<C, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_filter<C, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1) !=
                cudaSuccess)
            return check_launch("cudaFuncSetAttribute(k_filter)");
        attr_set = true;
    }
    const int units = (nref + G - 1) / G;
    int blocks = (units + 1) / 2;
    if (blocks < 1) blocks = 1;
    {
        KTimer kt("k_filter", s);
        k_filter<C, K, false><<<blocks, 64, sm0, s>>>(a);
    }
    hts_status st = check_launch("k_filter");
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_filter_exact", s);
        k_filter<C, K, true><<<152, 64, sm1, s>>>(a);
    }
    st = check_launch("k_filter_exact");
    if (st != HTS_OK) return st;
    const size_t HW = (size_t)a.H * a.W;
    int nb = (int)((HW * C + 255) / 256);
    if (nb > 152 * 16) nb = 152 * 16;
    {
        KTimer kt("k_normalize", s);
        k_normalize<<<nb, 256, 0, s>>>(a.acc, a.wcount, out, HW, C);
    }
    return check_launch("k_normalize");
}

}  // namespace

hts_status launch_filter(const float *img, const Geom &g, const int32_t *idx, const double *b64, const float *b32,
                         long long *acc, int *wcount, int32_t *redo_list, DevState *st, float *out, cudaStream_t s) {
    FilterArgs a;
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.step = g.step;
    a.nx = g.nx;
    a.nref = g.nref;
    a.idx = idx;
    a.b64 = b64;
    a.b32 = b32;
    a.acc = acc;
    a.wcount = wcount;
    a.redo = redo_list;
    a.st = st;
#define HTS_FILTER_CASE(CC, KK) \
    if (g.C == CC && g.K == KK) return launch_ck<CC, KK>(a, g.nref, out, s);
    HTS_FILTER_CASE(1, 2) HTS_FILTER_CASE(1, 4) HTS_FILTER_CASE(1, 8) HTS_FILTER_CASE(1, 16) HTS_FILTER_CASE(1, 32)
    HTS_FILTER_CASE(3, 2) HTS_FILTER_CASE(3, 4) HTS_FILTER_CASE(3, 8) HTS_FILTER_CASE(3, 16) HTS_FILTER_CASE(3, 32)
#undef HTS_FILTER_CASE
    return HTS_EUNSUPPORTED;
}

}  // namespace hts
