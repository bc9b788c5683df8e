// Collaborative filtering and aggregation of Haar-tSVD (Eq. 19-21, Alg. 1
// steps 2-3) on sm_103a.
//
// Main pass (k_filter_tile): a 512-thread block owns a tile of reference
// patches and keeps 64 group members in flight, eight threads per patch, one
// thread per patch row.  The separable projection Shat = U^H Phat V (Eq. 19,
// per stored Fourier slice of mode 3; slice 3 = conj of slice 2) is split in
// its two 8x8 factors: each thread forms its row of Phat V, the rows meet in
// shared memory, and each thread forms its row of U^H (Phat V).  The Haar
// transform along the group axis (Eq. 8 row order), hard thresholding
// (Eq. 20; modulus for complex coefficients) and the inverse Haar run one
// coefficient stream per thread from a patch-major buffer; the inverse
// projection (Eq. 21) mirrors the forward one.  Estimates are aggregated
// (Alg. 1 step 3) as exact fixed-point integers (value * 2^16, rounded) into
// shared-memory accumulators that cover the tile's whole search region, and
// flushed to the image-wide int64 sums once per tile.  Integer sums do not
// depend on the order of the additions, so the result is deterministic.
//
// Threshold decisions are taken in FP64 where FP32 cannot certify them: the
// FP32 coefficient of a group G differs from the exact one by at most
// 160 u ||G||_F (gray) / 320 u ||G||_F (colour) (twice the sum of the
// per-stage bounds of the DFT, the two 8x8 products with rounded bases and
// the Haar butterflies; the stages are unitary so errors do not grow).  A
// group with any coefficient inside that band around tau is not aggregated
// by the main pass; k_filter_exact recomputes it, evaluates each in-band
// coefficient in FP64 from the input pixels and the FP64 basis (one warp per
// coefficient), and takes the decision there.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "filter_common.h"
#include "hts_internal.h"

namespace hts {
namespace {

using fc::fix16;
using fc::fix16_split;
using fc::haar_fwd;
using fc::haar_inv;
using fc::K3F;
using fc::R2F;
using fc::S3H;

constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24
constexpr unsigned FULL = 0xffffffffu;
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
    int H, W, step, R, nx, ny, nref;
    const int32_t *idx;
    const double *b64;
    const float *b32;
    long long *acc;
    int *wcount;
    int32_t *redo;
    int4 *xlist;  // in-band coefficients: (group, keep<<16 | row<<8 | stream, re, im)
    int xcap;
    int exact;       // 0: FP32 threshold decisions only (precision form)
    const float *sigma_ref;  // [N_ref] noise level per group (nullptr: the call's one level)
    double tau_scale;        // tau = tau_scale * sigma
    int map_judged;          // sigma_ref only if the learned-map check passed
    uint8_t *xskip;  // [N_ref] 1 = group went to the exact pass
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

// Threshold of group r: tau_scale * sigma_r in FP64 when the noise level is
// given per group, else the call's threshold; the FP32 copy is the FP64 one
// rounded, so every pass decides against the same value.
__device__ __forceinline__ bool use_map(const FilterArgs &a) {
    return a.sigma_ref && (!a.map_judged || a.st->learned);
}
__device__ __forceinline__ double group_tau64(const FilterArgs &a, int r) {
    return use_map(a) ? a.tau_scale * (double)a.sigma_ref[r] : a.st->tau;
}
__device__ __forceinline__ float group_tau32(const FilterArgs &a, int r) {
    return use_map(a) ? (float)(a.tau_scale * (double)a.sigma_ref[r]) : a.st->tau32;
}

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
// A Haar detail row h >= 1 sums to zero over its members (Eq. 8), so its coefficient is unchanged when one
// member's patch (kref, the first of the row's support) is subtracted from every member: the FP32 value
// computed from those differences errs only in proportion to them, which at low noise are far smaller
// than the patches.  One (member k, patch row arow) unit: its FP32 contribution (sr, si) to the
// coefficient (slice j, position (i, jj)) and the sum sa of the absolute values of every product in it,
// sum_b |h_k| |U[arow][i]| |d[arow][b]| |V[b][jj]|, which bounds the evaluation error (diff_bound).
template <int C>
__device__ __forceinline__ void diff_unit32(const FilterArgs &a, const int32_t *grp, int K, int h, int j, int i,
                                            int jj, int kref, int k, int arow, float &sr, float &si, float &sa) {
    const size_t HW = (size_t)a.H * a.W;
    const float *U = a.b32 + (size_t)((j * 2 + 0) * 64) * 2;
    const float *V = a.b32 + (size_t)((j * 2 + 1) * 64) * 2;
    const int pos = grp[k], pref = grp[kref];
    const int y = pos / a.W, x = pos - y * a.W, yr = pref / a.W, xr = pref - yr * a.W;
    float tr = 0.f, ti = 0.f, ta = 0.f;
    for (int b = 0; b < 8; ++b) {
        const size_t o = (size_t)(y + arow) * a.W + x + b, orf = (size_t)(yr + arow) * a.W + xr + b;
        float pr, pi = 0.f, pa;
        if (C == 1) {
            pr = __ldg(a.img + o) - __ldg(a.img + orf);
            pa = fabsf(pr);
        } else {
            const float dR = __ldg(a.img + o) - __ldg(a.img + orf);
            const float dG = __ldg(a.img + HW + o) - __ldg(a.img + HW + orf);
            const float dB = __ldg(a.img + 2 * HW + o) - __ldg(a.img + 2 * HW + orf);
            if (j == 0) {
                pr = ((dR + dG) + dB) * K3F;
                pa = (fabsf(dR) + fabsf(dG) + fabsf(dB)) * K3F;
            } else {
                pr = (dR - 0.5f * (dG + dB)) * K3F;
                pi = (dB - dG) * (S3H * K3F);
                pa = (fabsf(dR) + 0.5f * (fabsf(dG) + fabsf(dB))) * K3F + (fabsf(dB) + fabsf(dG)) * (S3H * K3F);
            }
        }
        const float vr = V[(b * 8 + jj) * 2], vi = V[(b * 8 + jj) * 2 + 1];
        tr = fmaf(pr, vr, fmaf(-pi, vi, tr));
        ti = fmaf(pr, vi, fmaf(pi, vr, ti));
        ta = fmaf(pa, fabsf(vr) + fabsf(vi), ta);
    }
    const float ur = U[(arow * 8 + i) * 2], ui = U[(arow * 8 + i) * 2 + 1];
    const float hv = (float)haar_entry(K, h, k);
    sr = hv * fmaf(ur, tr, ui * ti);  // conj(u) * t
    si = hv * fmaf(ur, ti, -ui * tr);
    sa = fabsf(hv) * (fabsf(ur) + fabsf(ui)) * ta;
}

// The keep / drop decision of a coefficient from its FP32 difference evaluation (re, im, the absolute sum
// A of its products over at most 1024 of them): every product carries at most a few FP32 roundings of the
// differences, the basis and its own, and the summation (a thread's run of units, then a 7-level tree)
// adds at most about 20 u relative to A; 128 u A bounds the total with room to spare, and 4 u |value| the
// modulus.  1 keep, 0 drop, -1 undecided (the FP64 evaluation decides).
__device__ __forceinline__ int diff_decide(int j, float re, float im, float A, double tau64) {
    const float mag = (j == 0) ? fabsf(re) : sqrtf(re * re + im * im);
    const double bnd = 128.0 * (double)U32 * (double)A * 1.01 + 4.0 * (double)U32 * (double)mag + 1e-30;
    if ((double)mag - bnd >= tau64) return 1;
    if ((double)mag + bnd < tau64) return 0;
    return -1;
}

// The decision of coefficient (Haar row h >= 1, slice j, position e) of group grp by one warp from the FP32
// differences (diff_unit32 over the row's support, units spread over the lanes, a shuffle tree); -1 when the
// bound cannot decide it.
template <int C>
__device__ int diff_decide_warp(const FilterArgs &a, const int32_t *grp, int K, int h, int j, int e, int lane,
                                double tau64) {
    const int l = 31 - __clz(h), L = K >> l, k0 = (h - (1 << l)) * L;
    float fr = 0.f, fi = 0.f, fa = 0.f;
    for (int u = lane; u < L * 8; u += 32) {
        float ur, ui, ua;
        diff_unit32<C>(a, grp, K, h, j, e >> 3, e & 7, k0, k0 + (u >> 3), u & 7, ur, ui, ua);
        fr += ur;
        fi += ui;
        fa += ua;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        fr += __shfl_xor_sync(FULL, fr, o);
        fi += __shfl_xor_sync(FULL, fi, o);
        fa += __shfl_xor_sync(FULL, fa, o);
    }
    return diff_decide(j, fr, fi, fa, tau64);
}

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

// ---------------------------------------------------------------- kernels

template <int C>
struct Cfg {
    static constexpr int NCOEF = (C == 3) ? 192 : 64;  // real streams per patch
    static constexpr int IPG = (C == 3) ? 128 : 64;    // stream items per group (complex pairs count once)
};

// ---------------------------------------------------------- exact pass

// One group per warp (lane k < K owns patch k), groups taken from the redo
// list of the main pass.  FP32 forward; every coefficient inside the guard
// band is re-evaluated in FP64 by the whole warp and decided there; FP32
// inverse; global integer aggregation.
template <int C, int K>
__global__ void __launch_bounds__(64) k_filter_exact(FilterArgs a) {
    constexpr int NCOEF = Cfg<C>::NCOEF;
    constexpr int IPG = Cfg<C>::IPG;
    constexpr int ROW = K + 1;
    constexpr int GS = NCOEF * ROW;
    constexpr int NWARPS = 2;
    constexpr int NMASK = (NCOEF * K + 31) / 32;
    constexpr int WS = GS + 1 + NMASK + QCAP + 1;  // words per warp

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SBasis &sb = *reinterpret_cast<SBasis *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *coef = reinterpret_cast<float *>(smem_raw + sizeof(SBasis)) + warp * WS;
    float *gband = coef + GS;
    unsigned *mask = reinterpret_cast<unsigned *>(gband + 1);
    int *queue = reinterpret_cast<int *>(mask + NMASK);
    int *qcount = queue + QCAP;

    load_basis<C>(sb, a.b32);
    __syncthreads();

    const int k = lane;
    const bool active = lane < K;
    const size_t HW = (size_t)a.H * a.W;
    const int nunits = *(volatile int *)&a.st->filter_redo;

    for (int wu = blockIdx.x * NWARPS + warp; wu < nunits; wu += gridDim.x * NWARPS) {
        const int r = a.redo[wu];
        const float tau = group_tau32(a, r);
        const double tau64 = group_tau64(a, r);
        const int32_t *grp = a.idx + (size_t)r * K;
        int py = 0, px = 0;
        float ss = 0.f;
        if (active) {
            const int pos = grp[k];
            py = pos / a.W;
            px = pos - py * a.W;
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
            for (int e = 0; e < 64; ++e) coef[e * ROW + k] = P[e];
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
                    coef[(64 + e) * ROW + k] = Pr[e];
                    coef[(128 + e) * ROW + k] = Pi[e];
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(FULL, ss, o);
        if (lane == 0) {
            *gband = (C == 3 ? 320.f : 160.f) * U32 * sqrtf(ss) * 1.01f + 2.f * U32 * tau;
            *qcount = 0;
            for (int q = 0; q < NMASK; ++q) mask[q] = 0u;
        }
        __syncwarp();

        // pass 1: forward Haar only; coefficients stay unthresholded
#pragma unroll 1
        for (int t = lane; t < IPG; t += 32) {
            if (t < 64) {
                float x[K];
#pragma unroll
                for (int q = 0; q < K; ++q) x[q] = coef[t * ROW + q];
                haar_fwd<K>(x);
#pragma unroll
                for (int q = 0; q < K; ++q) coef[t * ROW + q] = x[q];
            } else {
                const int e = t - 64;
                float xr[K], xi[K];
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    xr[q] = coef[(64 + e) * ROW + q];
                    xi[q] = coef[(128 + e) * ROW + q];
                }
                haar_fwd<K>(xr);
                haar_fwd<K>(xi);
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    coef[(64 + e) * ROW + q] = xr[q];
                    coef[(128 + e) * ROW + q] = xi[q];
                }
            }
        }
        __syncwarp();
        const float band = *gband;
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
                    const float xr = coef[it * ROW + q], xi = coef[(it + 64) * ROW + q];
                    mag = sqrtf(xr * xr + xi * xi);
                }
                if (decide(mag, tau, band) != 2) continue;
                const int slot = atomicAdd(qcount, 1);
                if (slot < QCAP) queue[slot] = t;
            }
            __syncwarp();
            const int nq = min(*qcount, QCAP);
            if (nq == 0) break;
            for (int sl = 0; sl < nq; ++sl) {
                const int t = queue[sl];
                const int it = t / K, q = t - it * K;
                const int j = it < 64 ? 0 : 1;
                const int e = it < 64 ? it : it - 64;
                // Haar detail rows: first the certified FP32 evaluation on the members' differences
                int keep = (q > 0) ? diff_decide_warp<C>(a, grp, K, q, j, e, lane, tau64) : -1;
                if (keep < 0) {
                    double re, im;
                    exact_coef<C>(a, grp, K, q, j, e, lane, re, im);
                    const double mag = (j == 0) ? fabs(re) : sqrt(re * re + im * im);
                    keep = (mag >= tau64) ? 1 : 0;
                    if (lane == 0) atomicAdd(&a.st->filter_exact, 1);
                }
                if (lane == 0) {
                    const int bit = it * K + q;
                    mask[bit >> 5] |= (1u << (bit & 31));
                    if (!keep) {
                        coef[it * ROW + q] = 0.f;
                        if (it >= 64) coef[(it + 64) * ROW + q] = 0.f;
                    }
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
                    if (!dec && decide(sqrtf(vr * vr + vi * vi), tau, band) == 0) {
                        vr = 0.f;
                        vi = 0.f;
                    }
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
        __syncwarp();
        if (active) {
            float P[64];
#pragma unroll
            for (int e = 0; e < 64; ++e) P[e] = coef[e * ROW + k];
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
                                  (unsigned long long)fix16(P[u * 8 + v]));
                        atomicAdd(wc + o, 1);
                    }
            } else {
#pragma unroll
                for (int e = 0; e < 64; ++e) coef[e * ROW + k] = P[e];
                float Pr[64], Pi[64];
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    Pr[e] = coef[(64 + e) * ROW + k];
                    Pi[e] = coef[(128 + e) * ROW + k];
                }
                inv_cplx(Pr, Pi, sb);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const int e = u * 8 + v;
                        const float p0 = coef[e * ROW + k];
                        const float R = (p0 + 2.f * Pr[e]) * K3F;
                        const float Gc = (p0 - Pr[e] - 2.f * S3H * Pi[e]) * K3F;
                        const float B = (p0 - Pr[e] + 2.f * S3H * Pi[e]) * K3F;
                        const size_t o = (size_t)u * a.W + v;
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + o), (unsigned long long)fix16(R));
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + HW + o),
                                  (unsigned long long)fix16(Gc));
                        atomicAdd(reinterpret_cast<unsigned long long *>(acc0 + 2 * HW + o),
                                  (unsigned long long)fix16(B));
                        atomicAdd(wc + o, 1);
                    }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ main pass

constexpr int TPB = 512;       // threads per block
constexpr int PPB = TPB / 8;   // patches in flight per block (8 threads per patch)
// Coefficient e of a patch is stored at cpos(e) = e + 4 (e / 32): the 4-word
// gap after every 32 coefficients puts the eight 8-float rows a thread block
// writes at once into eight disjoint bank quads.  Row stride of the buffer:
constexpr int CROW = 212;      // cpos(191) + 1 = 211, padded to a multiple of 4
__device__ __forceinline__ int cpos(int e) { return e + 4 * (e >> 5); }
// 8x8 basis copies indexed by a thread's own row use a 12-float row stride
// (row r starts at bank 12 r mod 32: eight disjoint quads).
constexpr int BROW = 12;

struct TileArgs {
    int ty, tx;          // reference patches per tile (grid units)
    int nty, ntx, ntiles;
    int rh_max, rw_max;  // bound of a tile's region (pixels)
    int local;           // 1: aggregate in shared memory, 0: straight to the global sums
};

template <int C>
struct TileCfg {
    static constexpr int TW = (C == 3) ? 24 : 8;  // floats per row of the exchange buffer
    static constexpr int RS = TW + 4;              // row stride (bank-shifted)
    static constexpr int PSW = 8 * RS + 4;         // patch stride (bank-shifted)
};

constexpr int NSPARSE = 32;  // groups with at most this many kept coefficients are rebuilt from the list

// Entry (h, k) of the Haar matrix of Eq. 8 in FP32: row 0 is 1/sqrt(K); row
// h >= 1 (2^l <= h < 2^(l+1)) is +-1/sqrt(L) on its support of L = K / 2^l
// patches (first half +, second half -), 0 elsewhere.
__device__ __forceinline__ float inv_sqrt_pow2(int L) {
    switch (L) {
        case 1: return 1.0f;
        case 2: return 0.70710678118654752f;
        case 4: return 0.5f;
        case 8: return 0.35355339059327376f;
        case 16: return 0.25f;
        default: return 0.17677669529663688f;  // 32
    }
}
template <int K>
__device__ __forceinline__ float haar_entry_f32(int h, int k) {
    if (h == 0) return inv_sqrt_pow2(K);
    const int l = 31 - __clz(h), L = K >> l, i = h - (1 << l);
    if (k < i * L || k >= (i + 1) * L) return 0.f;
    const float m = inv_sqrt_pow2(L);
    return (k < i * L + L / 2) ? m : -m;
}

// Row-indexed basis copies (row stride BROW) for the block-parallel factors.
struct RBasis {
    float u0[8 * BROW], u0t[8 * BROW];
    float u1r[8 * BROW], u1i[8 * BROW], u1rt[8 * BROW], u1it[8 * BROW];
};

template <int C>
__device__ void load_rbasis(RBasis &rb, const SBasis &sb) {
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        const int r = t >> 3, c = t & 7;
        rb.u0[r * BROW + c] = sb.u0[t];
        rb.u0t[r * BROW + c] = sb.u0t[t];
        if (C == 3) {
            rb.u1r[r * BROW + c] = sb.u1r[t];
            rb.u1i[r * BROW + c] = sb.u1i[t];
            rb.u1rt[r * BROW + c] = sb.u1rt[t];
            rb.u1it[r * BROW + c] = sb.u1it[t];
        }
    }
}

template <int C, int K>
__global__ void __launch_bounds__(TPB, 1) k_filter_tile(FilterArgs a, TileArgs t) {
    constexpr int IPG = Cfg<C>::IPG;
    constexpr int GPB = PPB / K;  // groups in flight
    constexpr int TPG = 8 * K;    // threads per group
    constexpr int RS = TileCfg<C>::RS;
    constexpr int PSW = TileCfg<C>::PSW;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SBasis &sb = *reinterpret_cast<SBasis *>(smem_raw);
    RBasis &rb = *reinterpret_cast<RBasis *>(smem_raw + sizeof(SBasis));
    float *coef = reinterpret_cast<float *>(smem_raw + sizeof(SBasis) + sizeof(RBasis));  // [PPB][CROW]
    float *tbuf = coef + PPB * CROW;                                                      // [PPB][PSW]
    float *ssq = tbuf + PPB * PSW;                                                        // [TPB / 32]
    float *gband = ssq + TPB / 32;                                        // [GPB]
    int *gflag = reinterpret_cast<int *>(gband + GPB);                    // [GPB]
    int *gkept = gflag + GPB;                                             // kept coefficients per group
    int *grefs = gkept + GPB;                                             // reference index per group
    int *gv = grefs + GPB;                                                // group slot holds a group
    int *glen = gv + GPB;                                                 // [GPB] kept-list lengths
    int *klist = glen + GPB;                                              // [GPB][NSPARSE] kept (row, stream)
    int *accs = klist + GPB * NSPARSE;                                    // hi[C][RA] lo[C][RA] w[RA]
    const int RA = t.rh_max * t.rw_max;
    int *acc_hi = accs, *acc_lo = accs + C * RA, *acc_w = accs + 2 * C * RA;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ps = tid >> 3, row = tid & 7;  // patch slot, row
    const int gb = ps / K, k = ps - gb * K;  // group in flight, patch in group
    const int tg = tid - gb * TPG;           // thread within group

    load_basis<C>(sb, a.b32);
    __syncthreads();
    load_rbasis<C>(rb, sb);
    __syncthreads();
    const size_t HW = (size_t)a.H * a.W;
    const int gpt = t.ty * t.tx;
    const int nbatch = (gpt + GPB - 1) / GPB;

    for (int tile = blockIdx.x; tile < t.ntiles; tile += gridDim.x) {
        const int tyi = tile / t.ntx, txi = tile - tyi * t.ntx;
        const int gy0 = tyi * t.ty, gx0 = txi * t.tx;
        const int gy1 = min(a.ny, gy0 + t.ty) - 1, gx1 = min(a.nx, gx0 + t.tx) - 1;
        const int Y0 = grid_pos(gy0, a.H, a.step), Y1 = grid_pos(gy1, a.H, a.step);
        const int X0 = grid_pos(gx0, a.W, a.step), X1 = grid_pos(gx1, a.W, a.step);
        const int ry0 = max(0, Y0 - a.R), ry1 = min(a.H - 1, Y1 + a.R + PS - 1);
        const int rx0 = max(0, X0 - a.R), rx1 = min(a.W - 1, X1 + a.R + PS - 1);
        const int rh = ry1 - ry0 + 1, rw = rx1 - rx0 + 1;
        if (t.local) {
            for (int e = tid; e < (2 * C + 1) * RA; e += TPB) accs[e] = 0;
            __syncthreads();
        }
        for (int b = 0; b < nbatch; ++b) {
            const int lg = b * GPB + gb;
            const int gy = gy0 + lg / t.tx, gx = gx0 + lg % t.tx;
            const bool valid = (lg < gpt) && gy <= gy1 && gx <= gx1;
            const int r = valid ? gy * a.nx + gx : 0;
            const float tau = group_tau32(a, r);  // this thread's group
            int py = 0, px = 0;
            float ss = 0.f;
            if (tg == 0) {
                gkept[gb] = 0;
                glen[gb] = 0;
                grefs[gb] = r;
                gv[gb] = valid ? 1 : 0;
            }
            // ---- forward, factor 1: row `row` of Phat V
            if (valid) {
                const int pos = a.idx[(size_t)r * K + k];
                py = pos / a.W;
                px = pos - py * a.W;
                const float *src = a.img + (size_t)(py + row) * a.W + px;
                float P0[8], P1r[8], P1i[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    if (C == 1) {
                        const float x = __ldg(src + v);
                        P0[v] = x;
                        ss = fmaf(x, x, ss);
                    } else {
                        const float R = __ldg(src + v), Gc = __ldg(src + HW + v), B = __ldg(src + 2 * HW + v);
                        P0[v] = ((R + Gc) + B) * K3F;
                        P1r[v] = (R - 0.5f * (Gc + B)) * K3F;
                        P1i[v] = (B - Gc) * 0.5f;
                        ss = fmaf(R, R, ss);
                        ss = fmaf(Gc, Gc, ss);
                        ss = fmaf(B, B, ss);
                    }
                }
                float t0[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int bb = 0; bb < 8; ++bb) {
                    const float4 v0 = ld4(sb.v0 + bb * 8), v1 = ld4(sb.v0 + bb * 8 + 4);
                    const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) t0[j] = fmaf(P0[bb], vv[j], t0[j]);
                }
                float *T = tbuf + ps * PSW + row * RS;
                *reinterpret_cast<float4 *>(T) = make_float4(t0[0], t0[1], t0[2], t0[3]);
                *reinterpret_cast<float4 *>(T + 4) = make_float4(t0[4], t0[5], t0[6], t0[7]);
                if (C == 3) {
                    float tr[8], ti[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) { tr[j] = 0.f; ti[j] = 0.f; }
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
                        const float4 r0 = ld4(sb.v1r + bb * 8), r1 = ld4(sb.v1r + bb * 8 + 4);
                        const float4 i0 = ld4(sb.v1i + bb * 8), i1 = ld4(sb.v1i + bb * 8 + 4);
                        const float vr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                        const float vi[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
                        const float pr = P1r[bb], pi = P1i[bb];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            tr[j] = fmaf(pr, vr[j], tr[j]);
                            tr[j] = fmaf(-pi, vi[j], tr[j]);
                            ti[j] = fmaf(pr, vi[j], ti[j]);
                            ti[j] = fmaf(pi, vr[j], ti[j]);
                        }
                    }
                    *reinterpret_cast<float4 *>(T + 8) = make_float4(tr[0], tr[1], tr[2], tr[3]);
                    *reinterpret_cast<float4 *>(T + 12) = make_float4(tr[4], tr[5], tr[6], tr[7]);
                    *reinterpret_cast<float4 *>(T + 16) = make_float4(ti[0], ti[1], ti[2], ti[3]);
                    *reinterpret_cast<float4 *>(T + 20) = make_float4(ti[4], ti[5], ti[6], ti[7]);
                }
            }
            // group norm (deterministic: fixed shuffle tree, then warp partials in order)
#pragma unroll
            for (int o = 1; o < 32 && o < TPG; o <<= 1) ss += __shfl_xor_sync(FULL, ss, o);
            if (TPG <= 32) {
                if (tg == 0) {
                    gband[gb] = (C == 3 ? 320.f : 160.f) * U32 * sqrtf(ss) * 1.01f + 2.f * U32 * tau;
                    gflag[gb] = 0;
                }
            } else if ((tid & 31) == 0) {
                ssq[tid >> 5] = ss;
            }
            __syncthreads();
            if (TPG > 32 && tg == 0) {
                float s = 0.f;
                for (int w = 0; w < TPG / 32; ++w) s += ssq[(tid >> 5) + w];
                gband[gb] = (C == 3 ? 320.f : 160.f) * U32 * sqrtf(s) * 1.01f + 2.f * U32 * tau;
                gflag[gb] = 0;
            }
            // ---- forward, factor 2: row `row` (= i) of U^H (Phat V)
            if (valid) {
                const float *T = tbuf + ps * PSW;
                float s0[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const float4 c0 = ld4(rb.u0t + row * BROW), c1 = ld4(rb.u0t + row * BROW + 4);
                const float uc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int aa = 0; aa < 8; ++aa) {
                    const float4 x0 = ld4(T + aa * RS), x1 = ld4(T + aa * RS + 4);
                    const float tv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) s0[j] = fmaf(uc[aa], tv[j], s0[j]);
                }
                float *S = coef + ps * CROW;
                float *S0 = S + cpos(row * 8), *S1r = S + cpos(64 + row * 8), *S1i = S + cpos(128 + row * 8);
                *reinterpret_cast<float4 *>(S0) = make_float4(s0[0], s0[1], s0[2], s0[3]);
                *reinterpret_cast<float4 *>(S0 + 4) = make_float4(s0[4], s0[5], s0[6], s0[7]);
                if (C == 3) {
                    const float4 r0 = ld4(rb.u1rt + row * BROW), r1 = ld4(rb.u1rt + row * BROW + 4);
                    const float4 i0 = ld4(rb.u1it + row * BROW), i1 = ld4(rb.u1it + row * BROW + 4);
                    const float ur[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                    const float ui[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
                    float sr[8], si[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) { sr[j] = 0.f; si[j] = 0.f; }
#pragma unroll
                    for (int aa = 0; aa < 8; ++aa) {
                        const float4 a0 = ld4(T + aa * RS + 8), a1 = ld4(T + aa * RS + 12);
                        const float4 b0 = ld4(T + aa * RS + 16), b1 = ld4(T + aa * RS + 20);
                        const float trr[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        const float tii[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                        for (int j = 0; j < 8; ++j) {  // conj(u) * t
                            sr[j] = fmaf(ur[aa], trr[j], sr[j]);
                            sr[j] = fmaf(ui[aa], tii[j], sr[j]);
                            si[j] = fmaf(ur[aa], tii[j], si[j]);
                            si[j] = fmaf(-ui[aa], trr[j], si[j]);
                        }
                    }
                    *reinterpret_cast<float4 *>(S1r) = make_float4(sr[0], sr[1], sr[2], sr[3]);
                    *reinterpret_cast<float4 *>(S1r + 4) = make_float4(sr[4], sr[5], sr[6], sr[7]);
                    *reinterpret_cast<float4 *>(S1i) = make_float4(si[0], si[1], si[2], si[3]);
                    *reinterpret_cast<float4 *>(S1i + 4) = make_float4(si[4], si[5], si[6], si[7]);
                }
            }
            __syncthreads();
            // ---- Haar along the group axis and threshold, one coefficient stream per
            //      thread; the thresholded Haar-domain values stay in place.  A value
            //      inside the guard band is decided in FP32 here and recorded; the
            //      correction pass takes its decision in FP64.
            if (valid) {
                float *cg = coef + (gb * K) * CROW;
                const float band = gband[gb];
                int kept = 0;
#pragma unroll 1
                for (int it = tg; it < IPG; it += TPG) {
                    if (it < 64) {
                        const int pe = cpos(it);
                        float x[K];
#pragma unroll
                        for (int q = 0; q < K; ++q) x[q] = cg[q * CROW + pe];
                        haar_fwd<K>(x);
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            int d = decide(fabsf(x[q]), tau, band);
                            if (d == 2) {  // FP32 decides for now; the FP64 decision may correct it
                                const int keep = fabsf(x[q]) >= tau ? 1 : 0;
                                if (a.exact) {
                                    const int slot = atomicAdd(&a.st->xcount, 1);
                                    if (slot < a.xcap) {
                                        a.xlist[slot] =
                                            make_int4(r, (keep << 16) | (q << 8) | it, __float_as_int(x[q]), 0);
                                    } else {
                                        gflag[gb] = 1;
                                    }
                                }
                                d = keep;
                            }
                            if (d == 0) {
                                x[q] = 0.f;
                            } else {
                                ++kept;
                                const int slot = atomicAdd(glen + gb, 1);
                                if (slot < NSPARSE) klist[gb * NSPARSE + slot] = (q << 8) | it;
                            }
                            cg[q * CROW + pe] = x[q];
                        }
                    } else {
                        const int pr = cpos(it), pi = cpos(it + 64);
                        float xr[K], xi[K];
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            xr[q] = cg[q * CROW + pr];
                            xi[q] = cg[q * CROW + pi];
                        }
                        haar_fwd<K>(xr);
                        haar_fwd<K>(xi);
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const float mag = sqrtf(xr[q] * xr[q] + xi[q] * xi[q]);
                            int d = decide(mag, tau, band);
                            if (d == 2) {  // FP32 decides for now; the FP64 decision may correct it
                                const int keep = mag >= tau ? 1 : 0;
                                if (a.exact) {
                                    const int slot = atomicAdd(&a.st->xcount, 1);
                                    if (slot < a.xcap) {
                                        a.xlist[slot] = make_int4(r, (keep << 16) | (q << 8) | it,
                                                                  __float_as_int(xr[q]), __float_as_int(xi[q]));
                                    } else {
                                        gflag[gb] = 1;
                                    }
                                }
                                d = keep;
                            }
                            if (d == 0) {
                                xr[q] = 0.f;
                                xi[q] = 0.f;
                            } else {
                                ++kept;
                                const int slot = atomicAdd(glen + gb, 1);
                                if (slot < NSPARSE) klist[gb * NSPARSE + slot] = (q << 8) | it;
                            }
                            cg[q * CROW + pr] = xr[q];
                            cg[q * CROW + pi] = xi[q];
                        }
                    }
                }
                if (kept) atomicAdd(gkept + gb, kept);
            }
            __syncthreads();
            const bool agg = valid && gflag[gb] == 0;
            const bool sparse = agg && glen[gb] <= NSPARSE;
            if (valid && tg == 0) {
                a.xskip[r] = agg ? 0 : 1;  // a redone group takes no corrections
                if (!agg) {
                    const int pos = atomicAdd(&a.st->filter_redo, 1);
                    a.redo[pos] = r;
                }
            }
            // ---- kept lists of the sparse groups, sorted by (Haar row, stream) so that
            //      the reconstruction adds them in a fixed order
            for (int g2 = warp; g2 < GPB; g2 += TPB / 32) {
                if (!gv[g2] || gflag[g2] != 0 || glen[g2] > NSPARSE) continue;
                const int n = glen[g2];
                const int code = (lane < n) ? klist[g2 * NSPARSE + lane] : 0x7fffffff;
                int rank = 0;
                for (int j = 0; j < n; ++j) rank += (__shfl_sync(FULL, code, j) < code) ? 1 : 0;
                __syncwarp();
                if (lane < n) klist[g2 * NSPARSE + rank] = code;
            }
            // ---- dense groups: inverse Haar along the group axis
            if (agg && !sparse) {
                float *cg = coef + (gb * K) * CROW;
#pragma unroll 1
                for (int it = tg; it < IPG; it += TPG) {
                    if (it < 64) {
                        const int pe = cpos(it);
                        float x[K];
#pragma unroll
                        for (int q = 0; q < K; ++q) x[q] = cg[q * CROW + pe];
                        haar_inv<K>(x);
#pragma unroll
                        for (int q = 0; q < K; ++q) cg[q * CROW + pe] = x[q];
                    } else {
                        const int pr = cpos(it), pi = cpos(it + 64);
                        float xr[K], xi[K];
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            xr[q] = cg[q * CROW + pr];
                            xi[q] = cg[q * CROW + pi];
                        }
                        haar_inv<K>(xr);
                        haar_inv<K>(xi);
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            cg[q * CROW + pr] = xr[q];
                            cg[q * CROW + pi] = xi[q];
                        }
                    }
                }
            }
            __syncthreads();
            // ---- dense groups, inverse factor 1: row `row` (= i) of Shat V^H
            if (agg && !sparse) {
                const float *S = coef + ps * CROW;
                const float *S0 = S + cpos(row * 8), *S1r = S + cpos(64 + row * 8), *S1i = S + cpos(128 + row * 8);
                const float4 x0 = ld4(S0), x1 = ld4(S0 + 4);
                const float sv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                float q0[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 c0 = ld4(sb.v0t + j * 8), c1 = ld4(sb.v0t + j * 8 + 4);  // column j of V
                    const float vc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) q0[bb] = fmaf(sv[j], vc[bb], q0[bb]);
                }
                float *T = tbuf + ps * PSW + row * RS;
                *reinterpret_cast<float4 *>(T) = make_float4(q0[0], q0[1], q0[2], q0[3]);
                *reinterpret_cast<float4 *>(T + 4) = make_float4(q0[4], q0[5], q0[6], q0[7]);
                if (C == 3) {
                    const float4 a0 = ld4(S1r), a1 = ld4(S1r + 4), b0 = ld4(S1i), b1 = ld4(S1i + 4);
                    const float sr[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float si[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                    float qr[8], qi[8];
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) { qr[bb] = 0.f; qi[bb] = 0.f; }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 r0 = ld4(sb.v1rt + j * 8), r1 = ld4(sb.v1rt + j * 8 + 4);
                        const float4 i0 = ld4(sb.v1it + j * 8), i1 = ld4(sb.v1it + j * 8 + 4);
                        const float vr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                        const float vi[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) {  // s * conj(v)
                            qr[bb] = fmaf(sr[j], vr[bb], qr[bb]);
                            qr[bb] = fmaf(si[j], vi[bb], qr[bb]);
                            qi[bb] = fmaf(si[j], vr[bb], qi[bb]);
                            qi[bb] = fmaf(-sr[j], vi[bb], qi[bb]);
                        }
                    }
                    *reinterpret_cast<float4 *>(T + 8) = make_float4(qr[0], qr[1], qr[2], qr[3]);
                    *reinterpret_cast<float4 *>(T + 12) = make_float4(qr[4], qr[5], qr[6], qr[7]);
                    *reinterpret_cast<float4 *>(T + 16) = make_float4(qi[0], qi[1], qi[2], qi[3]);
                    *reinterpret_cast<float4 *>(T + 20) = make_float4(qi[4], qi[5], qi[6], qi[7]);
                }
            }
            __syncthreads();
            // ---- inverse factor 2 (dense) or the kept list (sparse): row `row` (= a)
            //      of P_hat, inverse DFT, aggregation
            if (agg) {
                float out[3][8];
                if (!sparse) {
                    const float *Q = tbuf + ps * PSW;
                    const float4 c0 = ld4(rb.u0 + row * BROW), c1 = ld4(rb.u0 + row * BROW + 4);
                    const float ua[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                    float p0[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 x0 = ld4(Q + i * RS), x1 = ld4(Q + i * RS + 4);
                        const float qv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) p0[bb] = fmaf(ua[i], qv[bb], p0[bb]);
                    }
                    if (C == 1) {
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) out[0][bb] = p0[bb];
                    } else {
                        const float4 r0 = ld4(rb.u1r + row * BROW), r1 = ld4(rb.u1r + row * BROW + 4);
                        const float4 i0 = ld4(rb.u1i + row * BROW), i1 = ld4(rb.u1i + row * BROW + 4);
                        const float ur[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                        const float ui[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
                        float pr[8], pi[8];
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) { pr[bb] = 0.f; pi[bb] = 0.f; }
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float4 a0 = ld4(Q + i * RS + 8), a1 = ld4(Q + i * RS + 12);
                            const float4 b0 = ld4(Q + i * RS + 16), b1 = ld4(Q + i * RS + 20);
                            const float qr[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                            const float qi[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                            for (int bb = 0; bb < 8; ++bb) {  // u * q
                                pr[bb] = fmaf(ur[i], qr[bb], pr[bb]);
                                pr[bb] = fmaf(-ui[i], qi[bb], pr[bb]);
                                pi[bb] = fmaf(ur[i], qi[bb], pi[bb]);
                                pi[bb] = fmaf(ui[i], qr[bb], pi[bb]);
                            }
                        }
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) {
                            out[0][bb] = (p0[bb] + 2.f * pr[bb]) * K3F;
                            out[1][bb] = (p0[bb] - pr[bb] - 2.f * S3H * pi[bb]) * K3F;
                            out[2][bb] = (p0[bb] - pr[bb] + 2.f * S3H * pi[bb]) * K3F;
                        }
                    }

                } else {
                    // P_hat_k[a][b] = sum over kept (h, i, j) of H[h][k] s U[a][i] conj(V[b][j])
                    float p0[8], pr[8], pi[8];
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) { p0[bb] = 0.f; pr[bb] = 0.f; pi[bb] = 0.f; }
                    const int *kl = klist + gb * NSPARSE;
                    const float *cgk = coef + (gb * K) * CROW;
                    const int nl = glen[gb];
                    for (int e = 0; e < nl; ++e) {
                        const int code = kl[e];
                        const int hq = code >> 8, it = code & 0xff;
                        const float hv = haar_entry_f32<K>(hq, k);
                        if (hv == 0.f) continue;
                        // current value: zero if the FP64 decision dropped it
                        const float vr = cgk[hq * CROW + cpos(it)] * hv;
                        const float vi = (it >= 64) ? cgk[hq * CROW + cpos(it + 64)] * hv : 0.f;
                        if (it < 64) {
                            const float w = vr * rb.u0[row * BROW + (it >> 3)];
                            const float4 c0 = ld4(sb.v0t + (it & 7) * 8), c1 = ld4(sb.v0t + (it & 7) * 8 + 4);
                            const float vc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                            for (int bb = 0; bb < 8; ++bb) p0[bb] = fmaf(w, vc[bb], p0[bb]);
                        } else if (C == 3) {
                            const int e1 = it - 64, i = e1 >> 3, j = e1 & 7;
                            const float ur = rb.u1r[row * BROW + i], ui = rb.u1i[row * BROW + i];
                            const float wr = vr * ur - vi * ui, wi = vr * ui + vi * ur;  // s u
                            const float4 r0 = ld4(sb.v1rt + j * 8), r1 = ld4(sb.v1rt + j * 8 + 4);
                            const float4 i0 = ld4(sb.v1it + j * 8), i1 = ld4(sb.v1it + j * 8 + 4);
                            const float cr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                            const float ci[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
                            for (int bb = 0; bb < 8; ++bb) {  // (s u) conj(v)
                                pr[bb] = fmaf(wr, cr[bb], pr[bb]);
                                pr[bb] = fmaf(wi, ci[bb], pr[bb]);
                                pi[bb] = fmaf(wi, cr[bb], pi[bb]);
                                pi[bb] = fmaf(-wr, ci[bb], pi[bb]);
                            }
                        }
                    }
                    if (C == 1) {
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) out[0][bb] = p0[bb];
                    } else {
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) {
                            out[0][bb] = (p0[bb] + 2.f * pr[bb]) * K3F;
                            out[1][bb] = (p0[bb] - pr[bb] - 2.f * S3H * pi[bb]) * K3F;
                            out[2][bb] = (p0[bb] - pr[bb] + 2.f * S3H * pi[bb]) * K3F;
                        }
                    }
                }
                if (t.local) {
                    const int ly = py + row - ry0, lx = px - rx0;
                    if (ly >= 0 && ly < rh && lx >= 0 && lx + 7 < rw) {
                        const int o = ly * rw + lx;
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) {
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                int qh, ql;
                                fix16_split(out[c][bb], qh, ql);
                                atomicAdd(acc_hi + c * RA + o + bb, qh);
                                atomicAdd(acc_lo + c * RA + o + bb, ql);
                            }
                            atomicAdd(acc_w + o + bb, 1);
                        }
                    } else {
                        atomicExch(&a.st->error, 1);
                    }
                } else {
                    const size_t o = (size_t)(py + row) * a.W + px;
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + c * HW + o + bb),
                                      (unsigned long long)fix16(out[c][bb]));
                        atomicAdd(a.wcount + o + bb, 1);
                    }
                }
            }
            __syncthreads();
        }
        if (t.local) {
            // flush the tile's sums to the image-wide int64 sums
            for (int e = tid; e < rh * rw; e += TPB) {
                const int w = acc_w[e];
                if (w == 0) continue;
                const int yy = e / rw, xx = e - yy * rw;
                const size_t g = (size_t)(ry0 + yy) * a.W + (rx0 + xx);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const long long s = (long long)acc_hi[c * RA + e] * 65536ll + (long long)acc_lo[c * RA + e];
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + c * HW + g), (unsigned long long)s);
                }
                atomicAdd(a.wcount + g, w);
            }
            __syncthreads();
        }
    }
}

// FP64 value of one Haar coefficient's unit (patch k of the support, row
// arow): conj(U[:, i])^T-row arow of P_k times V[:, jj], scaled by H[h][k].
template <int C>
__device__ __forceinline__ void exact_unit(const FilterArgs &a, const int32_t *grp, int K, int h, int j, int i, int jj,
                                           int k, int arow, double &sr, double &si) {
    const size_t HW = (size_t)a.H * a.W;
    const double *U = a.b64 + (size_t)((j * 2 + 0) * 64) * 2;
    const double *V = a.b64 + (size_t)((j * 2 + 1) * 64) * 2;
    const double k3 = 0.57735026918962576451;  // 1/sqrt(3)
    const double s3h = 0.86602540378443864676; // sqrt(3)/2
    const int pos = grp[k];
    const int y = pos / a.W, x = pos - (pos / a.W) * a.W;
    double tr = 0.0, ti = 0.0;
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
    sr = hv * (ur * tr + ui * ti);  // conj(u) * t
    si = hv * (ur * ti - ui * tr);
}

// FP64 decisions of the in-band coefficients recorded by k_filter_tile, one
// block of 128 threads each (one thread per (patch, row) unit of the
// coefficient's Haar support).  Where FP64 disagrees with the tentative FP32
// decision, the coefficient's contribution to the group's estimate --
// separable: Haar row h over its patch support, u_i v_j^H within each patch --
// is added (FP64 keeps it) or subtracted (FP64 drops it), in the same
// fixed-point sums.
template <int C, int K>
__global__ void __launch_bounds__(128) k_filter_fix(FilterArgs a) {
    __shared__ double red[2][4];
    __shared__ float red32[3][4];
    __shared__ int dec;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = min(*(volatile int *)&a.st->xcount, a.xcap);
    const size_t HW = (size_t)a.H * a.W;
    for (int f = blockIdx.x; f < n; f += gridDim.x) {
        const int4 e = a.xlist[f];
        const int r = e.x, keep32 = (e.y >> 16) & 1, h = (e.y >> 8) & 0xff, it = e.y & 0xff;
        if (a.xskip[r]) continue;  // the exact pass recomputes this group (uniform over the block)
        const int j = it < 64 ? 0 : 1, ei = it < 64 ? it : it - 64;
        const int i = ei >> 3, jj = ei & 7;
        const int32_t *grp = a.idx + (size_t)r * K;
        int k0 = 0, k1 = K;
        if (h > 0) {
            const int l = 31 - __clz(h), L = K >> l, ii = h - (1 << l);
            k0 = ii * L;
            k1 = k0 + L;
        }
        // Haar detail rows: first the certified FP32 evaluation on the members' differences
        if (h > 0) {
            float fr = 0.f, fi = 0.f, fa = 0.f;
            for (int u = tid; u < (k1 - k0) * 8; u += 128) {
                float ur, ui, ua;
                diff_unit32<C>(a, grp, K, h, j, i, jj, k0, k0 + (u >> 3), u & 7, ur, ui, ua);
                fr += ur;
                fi += ui;
                fa += ua;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                fr += __shfl_xor_sync(FULL, fr, o);
                fi += __shfl_xor_sync(FULL, fi, o);
                fa += __shfl_xor_sync(FULL, fa, o);
            }
            if (lane == 0) {
                red32[0][warp] = fr;
                red32[1][warp] = fi;
                red32[2][warp] = fa;
            }
            __syncthreads();
            if (tid == 0) {
                const float re = (red32[0][0] + red32[0][1]) + (red32[0][2] + red32[0][3]);
                const float im = (red32[1][0] + red32[1][1]) + (red32[1][2] + red32[1][3]);
                const float A = (red32[2][0] + red32[2][1]) + (red32[2][2] + red32[2][3]);
                dec = diff_decide(j, re, im, A, group_tau64(a, r));
            }
            __syncthreads();
        } else if (tid == 0) {
            dec = -1;
        }
        __syncthreads();
        if (dec < 0) {  // FP64 from the pixels and the FP64 basis
            double sr = 0.0, si = 0.0;
            for (int u = tid; u < (k1 - k0) * 8; u += 128) {
                double ur, ui;
                exact_unit<C>(a, grp, K, h, j, i, jj, k0 + (u >> 3), u & 7, ur, ui);
                sr += ur;
                si += ui;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                sr += __shfl_xor_sync(FULL, sr, o);
                si += __shfl_xor_sync(FULL, si, o);
            }
            if (lane == 0) {
                red[0][warp] = sr;
                red[1][warp] = si;
            }
            __syncthreads();
            if (tid == 0) {
                const double re = (red[0][0] + red[0][1]) + (red[0][2] + red[0][3]);
                const double im = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
                dec = (((j == 0) ? fabs(re) : sqrt(re * re + im * im)) >= group_tau64(a, r)) ? 1 : 0;
                atomicAdd(&a.st->filter_exact, 1);
            }
            __syncthreads();
        }
        if (tid == 0 && dec != keep32) atomicAdd(&a.st->filter_fixed, 1);
        __syncthreads();
        const int keep64 = dec;
        __syncthreads();  // dec and red are reused by the next entry
        if (keep64 == keep32) continue;
        const float sgn = keep64 ? 1.f : -1.f;
        const float cr = __int_as_float(e.z) * sgn, ci = __int_as_float(e.w) * sgn;
        const float *U = a.b32 + (size_t)((j * 2 + 0) * 64) * 2;
        const float *V = a.b32 + (size_t)((j * 2 + 1) * 64) * 2;
        for (int u = tid; u < (k1 - k0) * 64; u += 128) {
            const int k = k0 + (u >> 6), pe = u & 63;
            const float hv = haar_entry_f32<K>(h, k);
            const int pos = grp[k];
            const int py = pos / a.W, px = pos - py * a.W;
            const int aa = pe >> 3, bb = pe & 7;
            const float ur = U[(aa * 8 + i) * 2], ui = U[(aa * 8 + i) * 2 + 1];
            const float vr = V[(bb * 8 + jj) * 2], vi = V[(bb * 8 + jj) * 2 + 1];
            // hv c u conj(v)
            const float tr = hv * (cr * ur - ci * ui), ti = hv * (cr * ui + ci * ur);
            const float pr = tr * vr + ti * vi, pim = ti * vr - tr * vi;
            const size_t o = (size_t)(py + aa) * a.W + px + bb;
            if (C == 1) {
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + o), (unsigned long long)fix16(pr));
            } else if (j == 0) {
                const float v = pr * K3F;  // slice 0 is (R+G+B)/sqrt 3: equal share per channel
                for (int c = 0; c < 3; ++c)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + c * HW + o),
                              (unsigned long long)fix16(v));
            } else {
                const float R = 2.f * pr * K3F;
                const float G = (-pr - 2.f * S3H * pim) * K3F;
                const float B = (-pr + 2.f * S3H * pim) * K3F;
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + o), (unsigned long long)fix16(R));
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + HW + o), (unsigned long long)fix16(G));
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + 2 * HW + o), (unsigned long long)fix16(B));
            }
        }
    }
}

// out = sum / (2^16 * weight)
__global__ void k_normalize(const long long *__restrict__ acc, const int *__restrict__ wcount, float *__restrict__ out,
                            size_t HW, int C) {
    const size_t n = HW * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i % HW;
        const int w = wcount[p];
        out[i] = __ll2float_rn(acc[i]) * (1.0f / 65536.0f) / (float)w;
    }
}

// The same, four pixels per thread with 16-byte loads and stores (HW a multiple of 4, 16-byte aligned
// arrays): each pixel's weight is read once for all channels.
template <int C>
__global__ void k_normalize4(const longlong2 *__restrict__ acc, const int4 *__restrict__ wcount, float4 *__restrict__ out,
                             size_t HW4) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < HW4; q += (size_t)gridDim.x * blockDim.x) {
        const int4 w = __ldg(wcount + q);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const longlong2 a0 = __ldg(acc + (c * HW4 + q) * 2), a1 = __ldg(acc + (c * HW4 + q) * 2 + 1);
            float4 o;
            o.x = __ll2float_rn(a0.x) * (1.0f / 65536.0f) / (float)w.x;
            o.y = __ll2float_rn(a0.y) * (1.0f / 65536.0f) / (float)w.y;
            o.z = __ll2float_rn(a1.x) * (1.0f / 65536.0f) / (float)w.z;
            o.w = __ll2float_rn(a1.y) * (1.0f / 65536.0f) / (float)w.w;
            out[c * HW4 + q] = o;
        }
    }
}

// Weights from patch-origin counts (the tensor-core filter's aggregation): the weight of pixel (y, x)
// is the sum of the counts of the origins (y - u, x - v), 0 <= u, v < 8, formed per 32 x 32 block of
// pixels from the counts staged in shared memory (row sums over 8 columns, then 8 rows); then
// out = sum / (2^16 weight) as in k_normalize.  Colour: the tensor-core filter sums the slices of the
// channel DFT (P^(1), sqrt2 Re P^(2), sqrt2 Im P^(2), orthonormal), turned back into R, G, B here.
constexpr int NB_T = 32;
template <int C>
__global__ void __launch_bounds__(256) k_normalize_box(const long long *__restrict__ acc, const int *__restrict__ cnt,
                                                       float *__restrict__ out, int H, int W) {
    __shared__ int sc[NB_T + PS - 1][NB_T + PS - 1];
    __shared__ int sr[NB_T + PS - 1][NB_T];
    const int by = blockIdx.y * NB_T, bx = blockIdx.x * NB_T;
    const size_t HW = (size_t)H * W;
    for (int e = threadIdx.x; e < (NB_T + PS - 1) * (NB_T + PS - 1); e += blockDim.x) {
        const int yy = e / (NB_T + PS - 1), xx = e - yy * (NB_T + PS - 1);
        const int y = by + yy - (PS - 1), x = bx + xx - (PS - 1);
        sc[yy][xx] = (y >= 0 && y < H && x >= 0 && x < W) ? __ldg(cnt + (size_t)y * W + x) : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (NB_T + PS - 1) * NB_T; e += blockDim.x) {
        const int yy = e / NB_T, xx = e - yy * NB_T;
        int t = 0;
#pragma unroll
        for (int v = 0; v < PS; ++v) t += sc[yy][xx + v];
        sr[yy][xx] = t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB_T * NB_T; e += blockDim.x) {
        const int yy = e / NB_T, xx = e - yy * NB_T;
        const int y = by + yy, x = bx + xx;
        if (y >= H || x >= W) continue;
        int w = 0;
#pragma unroll
        for (int u = 0; u < PS; ++u) w += sr[yy + u][xx];
        const size_t p = (size_t)y * W + x;
        if constexpr (C == 1) {
            out[p] = __ll2float_rn(acc[p]) * (1.0f / 65536.0f) / (float)w;
        } else {  // the sums are per slice [P^(1) | sqrt2 Re P^(2) | sqrt2 Im P^(2)]: the inverse channel DFT
            const float sc = (1.0f / 65536.0f) / (float)w;
            const float s0 = __ll2float_rn(acc[p]) * sc, s1 = __ll2float_rn(acc[HW + p]) * sc,
                        s2 = __ll2float_rn(acc[2 * HW + p]) * sc;
            const float t = fc::K3F * s0 - 0.5f * fc::K23F * s1;
            out[p] = fmaf(fc::K23F, s1, fc::K3F * s0);
            out[HW + p] = t - fc::R2F * s2;
            out[2 * HW + p] = t + fc::R2F * s2;
        }
    }
}

template <int C, int K>
size_t exact_smem() {
    constexpr int NCOEF = Cfg<C>::NCOEF;
    constexpr int GS = NCOEF * (K + 1);
    constexpr int NMASK = (NCOEF * K + 31) / 32;
    return sizeof(SBasis) + (size_t)2 * (GS + 1 + NMASK + QCAP + 1) * 4;
}

template <int C, int K>
size_t tile_fixed_smem() {
    constexpr int GPB = PPB / K;
    return sizeof(SBasis) + sizeof(RBasis) +
           ((size_t)PPB * CROW + (size_t)PPB * TileCfg<C>::PSW + TPB / 32 + 6 * GPB + (size_t)GPB * NSPARSE) * 4;
}

constexpr int NSHAPES = 6;
constexpr int SHAPES[NSHAPES][2] = {{4, 8}, {4, 4}, {2, 4}, {2, 2}, {1, 2}, {1, 1}};

size_t tile_fixed_bytes(int C, int K) {
#define HTS_FIXED_CASE(CC, KK) \
    if (C == CC && K == KK) return tile_fixed_smem<CC, KK>();
    HTS_FIXED_CASE(1, 2) HTS_FIXED_CASE(1, 4) HTS_FIXED_CASE(1, 8) HTS_FIXED_CASE(1, 16) HTS_FIXED_CASE(1, 32)
    HTS_FIXED_CASE(3, 2) HTS_FIXED_CASE(3, 4) HTS_FIXED_CASE(3, 8) HTS_FIXED_CASE(3, 16) HTS_FIXED_CASE(3, 32)
#undef HTS_FIXED_CASE
    return ~size_t(0);
}

// Shared memory of a tile of ty x tx references (0 for the non-local mode's tile part).
size_t tile_bytes(const Geom &g, int ty, int tx, int *rh_out = nullptr, int *rw_out = nullptr) {
    const int rh = ty ? std::min(g.H, (ty - 1) * g.step + 2 * g.R + PS) : 0;
    const int rw = tx ? std::min(g.W, (tx - 1) * g.step + 2 * g.R + PS) : 0;
    if (rh_out) *rh_out = rh;
    if (rw_out) *rw_out = rw;
    return tile_fixed_bytes(g.C, g.K) + (size_t)(2 * g.C + 1) * rh * rw * 4;
}

size_t tile_budget() { return std::min((size_t)smem_optin(), (size_t)227 * 1024); }

thread_local const TileChoice *t_forced = nullptr;
thread_local TileChoice t_forced_val;
std::mutex g_tune_mu;
std::map<std::vector<int>, TileChoice> g_tuned;

std::vector<int> tune_key(const Geom &g) {
    int dev = 0;
    cudaGetDevice(&dev);
    return {dev, g.H, g.W, g.C, g.K, g.R, g.step};
}

// Normalisation when wcount holds patch-origin counts (the tensor-core filter).
hts_status normalize_box(const long long *acc, const int *cnt, float *out, int H, int W, int C, cudaStream_t s) {
    const dim3 grid((W + NB_T - 1) / NB_T, (H + NB_T - 1) / NB_T);
    {
        KTimer kt("k_normalize_box", s);
        if (C == 1) k_normalize_box<1><<<grid, 256, 0, s>>>(acc, cnt, out, H, W);
        else k_normalize_box<3><<<grid, 256, 0, s>>>(acc, cnt, out, H, W);
    }
    return check_launch("k_normalize_box");
}

hts_status launch_normalize(const long long *acc, const int *wcount, float *out, size_t HW, int C, int nsm,
                            cudaStream_t s) {
    const bool vec = HW % 4 == 0 && ((reinterpret_cast<uintptr_t>(acc) | reinterpret_cast<uintptr_t>(wcount) |
                                      reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (vec) {
        const size_t HW4 = HW / 4;
        int nb = (int)((HW4 + 255) / 256);
        if (nb > nsm * 8) nb = nsm * 8;
        KTimer kt("k_normalize", s);
        if (C == 1)
            k_normalize4<1><<<nb, 256, 0, s>>>(reinterpret_cast<const longlong2 *>(acc),
                                               reinterpret_cast<const int4 *>(wcount), reinterpret_cast<float4 *>(out), HW4);
        else
            k_normalize4<3><<<nb, 256, 0, s>>>(reinterpret_cast<const longlong2 *>(acc),
                                               reinterpret_cast<const int4 *>(wcount), reinterpret_cast<float4 *>(out), HW4);
    } else {
        int nb = (int)((HW * C + 255) / 256);
        if (nb > nsm * 16) nb = nsm * 16;
        KTimer kt("k_normalize", s);
        k_normalize<<<nb, 256, 0, s>>>(acc, wcount, out, HW, C);
    }
    return check_launch("k_normalize");
}

template <int C, int K>
hts_status launch_ck(const FilterArgs &a, const Geom &g, float *out, cudaStream_t s) {
    const size_t HW = (size_t)a.H * a.W;
    // tile shape: forced (autotuning), tuned, or the largest that fits
    TileChoice ch;
    TileChoice cands[NSHAPES + 1];
    tile_candidates(g, cands, NSHAPES + 1);
    if (t_forced) ch = *t_forced;
    else if (!tuned_tile(g, &ch)) ch = cands[0];
    if (ch.ty > 0 && tile_bytes(g, ch.ty, ch.tx) > tile_budget()) ch = cands[0];
    const size_t fixed = tile_fixed_smem<C, K>();
    TileArgs ta;
    ta.local = ch.ty > 0 ? 1 : 0;
    ta.ty = ch.ty > 0 ? ch.ty : 4;
    ta.tx = ch.ty > 0 ? ch.tx : 8;
    ta.rh_max = 0;
    ta.rw_max = 0;
    if (ta.local) tile_bytes(g, ta.ty, ta.tx, &ta.rh_max, &ta.rw_max);
    ta.nty = (g.ny + ta.ty - 1) / ta.ty;
    ta.ntx = (g.nx + ta.tx - 1) / ta.tx;
    ta.ntiles = ta.nty * ta.ntx;
    const size_t sm_tile = fixed + (size_t)(2 * C + 1) * ta.rh_max * ta.rw_max * 4;
    const size_t sm_exact = exact_smem<C, K>();
    {
        hts_status st0 = allow_smem(reinterpret_cast<const void *>(k_filter_tile<C, K>), sm_tile);
        if (st0 == HTS_OK) st0 = allow_smem(reinterpret_cast<const void *>(k_filter_exact<C, K>), sm_exact);
        if (st0 != HTS_OK) return st0;
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(ta.ntiles, nsm));
    {
        KTimer kt("k_filter", s);
        k_filter_tile<C, K><<<grid, TPB, sm_tile, s>>>(a, ta);
    }
    hts_status st = check_launch("k_filter");
    if (st != HTS_OK) return st;
    if (a.exact) {
        // the FP64 passes' work lists live on the device: as many blocks as fit on the SMs, each taking
        // entries in turn (their integer additions do not depend on the order)
        int per_sm_x = 1, per_sm_f = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, k_filter_exact<C, K>, 64, sm_exact);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_filter_fix<C, K>, 128, 0);
        {
            KTimer kt("k_filter_exact", s);
            k_filter_exact<C, K><<<nsm * std::max(per_sm_x, 1), 64, sm_exact, s>>>(a);
        }
        st = check_launch("k_filter_exact");
        if (st != HTS_OK) return st;
        {
            KTimer kt("k_filter_fix", s);
            k_filter_fix<C, K><<<nsm * std::max(per_sm_f, 1), 128, 0, s>>>(a);
        }
        st = check_launch("k_filter_fix");
        if (st != HTS_OK) return st;
    }
    return launch_normalize(a.acc, a.wcount, out, HW, C, nsm, s);
}

}  // namespace

int tile_candidates(const Geom &g, TileChoice *out, int max) {
    int n = 0;
    for (int i = 0; i < NSHAPES && n < max; ++i)
        if (tile_bytes(g, SHAPES[i][0], SHAPES[i][1]) <= tile_budget()) out[n++] = {SHAPES[i][0], SHAPES[i][1]};
    if (n < max) out[n++] = {0, 0};  // non-local mode: always valid
    return n;
}

void force_tile(const TileChoice *c) {
    if (c) {
        t_forced_val = *c;
        t_forced = &t_forced_val;
    } else {
        t_forced = nullptr;
    }
}

bool tuned_tile(const Geom &g, TileChoice *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(g));
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
}

void set_tuned_tile(const Geom &g, TileChoice c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(g)] = c;
}

hts_status launch_filter(const float *img, const Geom &g, const int32_t *idx, const double *b64, const float *b32,
                         long long *acc, int *wcount, int32_t *redo_list, int4 *xlist, uint8_t *xskip,
                         DevState *st, float *out, int exact, const float *sigma_ref, int map_judged, double tau_scale,
                         cudaStream_t s, const float *mean_est) {
    FilterArgs a;
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nref = g.nref;
    a.idx = idx;
    a.b64 = b64;
    a.b32 = b32;
    a.acc = acc;
    a.wcount = wcount;
    a.redo = redo_list;
    a.xlist = xlist;
    a.xcap = XLIST_PER_REF * g.nref;
    a.exact = exact;
    a.sigma_ref = sigma_ref;
    a.tau_scale = tau_scale;
    a.map_judged = map_judged;
    a.xskip = xskip;
    a.st = st;
    if (mean_est && exact) return report(HTS_EUNSUPPORTED, "the enhancement strategy needs the tensor-core filter");
    if (!exact) {  // precision form: the tensor-core filter where a tile fits
        bool used = false;
        const hts_status st0 =
            launch_filter_tc(img, g, idx, b32, acc, wcount, st, sigma_ref, map_judged, tau_scale, mean_est, s, &used);
        if (st0 != HTS_OK) return st0;
        if (!used && mean_est) return report(HTS_EUNSUPPORTED, "the enhancement strategy needs the tensor-core filter");
        if (used) return normalize_box(acc, wcount, out, g.H, g.W, g.C, s);
    }
#define HTS_FILTER_CASE(CC, KK) \
    if (g.C == CC && g.K == KK) return launch_ck<CC, KK>(a, g, out, s);
    HTS_FILTER_CASE(1, 2) HTS_FILTER_CASE(1, 4) HTS_FILTER_CASE(1, 8) HTS_FILTER_CASE(1, 16) HTS_FILTER_CASE(1, 32)
    HTS_FILTER_CASE(3, 2) HTS_FILTER_CASE(3, 4) HTS_FILTER_CASE(3, 8) HTS_FILTER_CASE(3, 16) HTS_FILTER_CASE(3, 32)
#undef HTS_FILTER_CASE
    return HTS_EUNSUPPORTED;
}

hts_status launch_normalize_box(const long long *acc, const int *cnt, float *out, int H, int W, int C,
                                cudaStream_t s) {
    return normalize_box(acc, cnt, out, H, W, C, s);
}

}  // namespace hts
