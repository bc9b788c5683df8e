// Noise level of Haar-tSVD on sm_103a.
//
// k_sigma_est  : Eq. 12 -- for AWGN every eigenvalue of the global
//                covariances carries ps * N_ref * sigma^2, so sigma_est^2 is
//                the smallest eigenvalue over all slices and both covariances
//                divided by ps * N_ref (optionally by the Marchenko-Pastur
//                lower edge (1 - 1/sqrt(N_ref))^2 of the noise spectrum);
// k_vote       : Eq. 16-18 and 22 -- the eigenvalues of circ(G) circ(G)^T are
//                lambda_m = ||sum_k e^{-2 pi i m k / K} p_k||^2; the rank
//                position a of lambda_hat = lambda_{K/2} among them decides a
//                vote a <= gamma (Eq. 23).  Computed in FP32 on the group with
//                the reference patch subtracted (lambda_m, m != 0, is
//                unchanged by a common offset), with a rigorous error bound;
//                a group whose count the bound cannot settle is recomputed in
//                FP64.  Each block adds its votes once (integer, order-free);
// k_sigma_final: a strict majority divides sigma_est by beta (Eq. 23); then
//                tau = tau_mult sigma sqrt(2 ln(c K ps^2)).
#include <algorithm>
#include <cooperative_groups.h>

#include "hts_internal.h"

namespace hts {
namespace {

constexpr float U32 = 5.9604644775390625e-08f;
constexpr unsigned FULL = 0xffffffffu;

__global__ void k_sigma_est(const double *__restrict__ eig, int nvals, int nref, int mp, DevState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lam = eig[0];
    for (int i = 1; i < nvals; ++i) lam = fmin(lam, eig[i]);
    double s2 = fmax(lam, 0.0) / (double)(PS * nref);
    if (mp && nref > 1) {
        const double f = 1.0 - 1.0 / sqrt((double)nref);
        s2 = s2 / (f * f);
    }
    st->sigma_est = sqrt(s2);  // the vote counters are zeroed with the state and may be live on another stream
}

__device__ __forceinline__ void twiddle64(int j, int K, double &c, double &s) {
    // exp(-2 pi i j / K) = c + i s, exact at quarter turns
    j %= K;
    if ((4 * j) % K == 0) {
        const int q = (4 * j) / K;
        c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
        s = (q == 1) ? -1.0 : (q == 3 ? 1.0 : 0.0);
        return;
    }
    double sn, cs;
    sincospi(2.0 * (double)j / (double)K, &sn, &cs);
    c = cs;
    s = -sn;
}

// exp(-2 pi i j / 32) = c_twc[j] + i c_tws[j], rounded to float (quarter turns
// exact).  Indexed with warp-uniform j, they are read as constant operands.
__constant__ float c_twc[32] = {
    1.0f, 0.9807852506637573f, 0.9238795042037964f, 0.8314695954322815f,
    0.7071067690849304f, 0.5555702447891235f, 0.3826834261417389f, 0.19509032368659973f,
    0.0f, -0.19509032368659973f, -0.3826834261417389f, -0.5555702447891235f,
    -0.7071067690849304f, -0.8314695954322815f, -0.9238795042037964f, -0.9807852506637573f,
    -1.0f, -0.9807852506637573f, -0.9238795042037964f, -0.8314695954322815f,
    -0.7071067690849304f, -0.5555702447891235f, -0.3826834261417389f, -0.19509032368659973f,
    0.0f, 0.19509032368659973f, 0.3826834261417389f, 0.5555702447891235f,
    0.7071067690849304f, 0.8314695954322815f, 0.9238795042037964f, 0.9807852506637573f,
};
__constant__ float c_tws[32] = {
    0.0f, -0.19509032368659973f, -0.3826834261417389f, -0.5555702447891235f,
    -0.7071067690849304f, -0.8314695954322815f, -0.9238795042037964f, -0.9807852506637573f,
    -1.0f, -0.9807852506637573f, -0.9238795042037964f, -0.8314695954322815f,
    -0.7071067690849304f, -0.5555702447891235f, -0.3826834261417389f, -0.19509032368659973f,
    0.0f, 0.19509032368659973f, 0.3826834261417389f, 0.5555702447891235f,
    0.7071067690849304f, 0.8314695954322815f, 0.9238795042037964f, 0.9807852506637573f,
    1.0f, 0.9807852506637573f, 0.9238795042037964f, 0.8314695954322815f,
    0.7071067690849304f, 0.5555702447891235f, 0.3826834261417389f, 0.19509032368659973f,
};

// The same twiddles in FP64 (correctly rounded cos / sin of 2 pi j / 32).
__constant__ double c_twc64[32] = {
    1.0, 0.9807852804032304, 0.9238795325112867, 0.8314696123025452,
    0.7071067811865476, 0.5555702330196023, 0.38268343236508984, 0.19509032201612833,
    0.0, -0.1950903220161282, -0.3826834323650897, -0.555570233019602,
    -0.7071067811865475, -0.8314696123025453, -0.9238795325112867, -0.9807852804032304,
    -1.0, -0.9807852804032304, -0.9238795325112868, -0.8314696123025455,
    -0.7071067811865477, -0.5555702330196022, -0.38268343236509034, -0.19509032201612866,
    0.0, 0.1950903220161283, 0.38268343236509, 0.5555702330196018,
    0.7071067811865474, 0.8314696123025452, 0.9238795325112865, 0.9807852804032303,
};
__constant__ double c_tws64[32] = {
    0.0, -0.19509032201612825, -0.3826834323650898, -0.5555702330196022,
    -0.7071067811865475, -0.8314696123025452, -0.9238795325112867, -0.9807852804032304,
    -1.0, -0.9807852804032304, -0.9238795325112867, -0.8314696123025455,
    -0.7071067811865476, -0.5555702330196022, -0.3826834323650899, -0.1950903220161286,
    0.0, 0.19509032201612836, 0.38268343236508967, 0.555570233019602,
    0.7071067811865475, 0.8314696123025452, 0.9238795325112865, 0.9807852804032303,
    1.0, 0.9807852804032304, 0.9238795325112866, 0.8314696123025455,
    0.7071067811865477, 0.5555702330196022, 0.3826834323650904, 0.19509032201612872,
};

// FP64 lambda_m, m = 0..K/2 (lambda_{K-m} = lambda_m for real patches), of
// the component range [d0, d1) of a group: one component per thread, block
// sum in a fixed order.
template <int C, int K>
__device__ void lambda64_partial(const float *__restrict__ img, int H, int W, const int32_t *__restrict__ grp,
                                 int d0, int d1, double *__restrict__ sm, double *__restrict__ out) {
    constexpr int NM = K / 2 + 1;
    const size_t HW = (size_t)H * W;
    double l[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) l[m] = 0.0;
    const int d = d0 + (int)threadIdx.x;
    if (d < d1) {
        const int c = d / NPIX, e = d - c * NPIX;
        const size_t base = (size_t)c * HW + (size_t)(e >> 3) * W + (e & 7);
        double p[K];
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = (double)__ldg(img + base + grp[k]);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            double xr = 0.0, xi = 0.0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = ((m * k) % K) * (32 / K);
                // quarter turns: the twiddle parts are exactly 0 or +-1, the same sums without the products
                if (j == 0) xr += p[k];
                else if (j == 8) xi -= p[k];
                else if (j == 16) xr -= p[k];
                else if (j == 24) xi += p[k];
                else {
                    xr += p[k] * c_twc64[j];
                    xi += p[k] * c_tws64[j];
                }
            }
            l[m] = xr * xr + xi * xi;
        }
    }
    // block sum, fixed order: warps by shuffle tree, then warp partials in order
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        double v = l[m];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if ((threadIdx.x & 31) == 0) sm[(threadIdx.x >> 5) * NM + m] = v;
    }
    __syncthreads();
    if (threadIdx.x < NM) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sm[w * NM + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// Half spectrum X_m, m = 0..N/2, of N real values x (N a power of two, 2..32), into re[m OS], im[m OS]:
// one radix-2 split per level (a_k = x_k + x_{k+N/2} carries the even outputs, d_k = x_k - x_{k+N/2} the
// odd ones), the odd outputs X_{2j+1} = sum_k d_k w^{(2j+1) k} evaluated directly, pairing d_k with
// d_{N/2-k} (their twiddles are minus each other's conjugates):
//   X_{2j+1} = d_0 + sum_{0<k<N/4} [(d_k - d_{N/2-k}) cos t - i (d_k + d_{N/2-k}) sin t] + (-i)^{2j+1} d_{N/4},
// t = 2 pi (2j+1) k / N.  Every input reaches a real or imaginary output part along one path, whose
// constants are at most 1 in modulus: for an odd output split off after L levels, L sums, the
// difference d, the pair, the twiddle's own rounding and at most N / 2^(L+2) - 1 steps of the chain,
// i.e. at most N/4 + 2 roundings (N >= 4); for X_0, log2 N.  So |Re, Im error| <= gamma_(N/4 + 2)
// sum_k |x_k|.
template <int N, int OS, int NO>
__device__ __forceinline__ void rdft_half(const float *x, float (&re)[NO], float (&im)[NO]) {
    if constexpr (N == 2) {
        re[0] = x[0] + x[1];
        im[0] = 0.f;
        re[OS] = x[0] - x[1];
        im[OS] = 0.f;
    } else {
        constexpr int n = N / 2;
        float a[n], d[n];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            a[k] = x[k] + x[k + n];
            d[k] = x[k] - x[k + n];
        }
        rdft_half<n, 2 * OS, NO>(a, re, im);
        float dd[n / 2 > 0 ? n / 2 : 1], ss[n / 2 > 0 ? n / 2 : 1];
#pragma unroll
        for (int k = 1; k < n / 2; ++k) {
            dd[k] = d[k] - d[n - k];
            ss[k] = d[k] + d[n - k];
        }
#pragma unroll
        for (int j = 0; j < n / 2; ++j) {
            float r = d[0], i = (j & 1) ? d[n / 2] : -d[n / 2];
#pragma unroll
            for (int k = 1; k < n / 2; ++k) {
                const int t = ((2 * j + 1) * k * (32 / N)) & 31;
                // quarter turns: the twiddle parts are exactly 0 or +-1, the same sums without the products
                if (t == 0) r += dd[k];
                else if (t == 8) i -= ss[k];
                else if (t == 16) r -= dd[k];
                else if (t == 24) i += ss[k];
                else {
                    r = fmaf(dd[k], c_twc[t], r);
                    i = fmaf(ss[k], c_tws[t], i);
                }
            }
            re[(2 * j + 1) * OS] = r;
            im[(2 * j + 1) * OS] = i;
        }
    }
}

// The vote of one group (one warp): lambda_m of its members' patches, components read from src at
// c * plane + (e >> 3) * rstride + (e & 7) + off[k] for member k; returns 1 for a vote, 0 otherwise (a group
// the FP32 bound cannot settle is listed for k_vote_exact and counts 0 here).
template <int C, int K>
__device__ __forceinline__ int vote_group(const float *__restrict__ src, size_t plane, int rstride,
                                          const int (&off)[K], double gamma_rank, int r, int32_t *__restrict__ list,
                                          DevState *st) {
    constexpr int D = C * NPIX;
    constexpr int NM = K / 2 + 1;
    const int lane = threadIdx.x & 31;
    float lam[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) lam[m] = 0.f;
    float e0sq = 0.f, esq = 0.f;
#pragma unroll 1
    for (int d = lane; d < D; d += 32) {
        const int c = d / NPIX, e = d - c * NPIX;
        const size_t base = (size_t)c * plane + (size_t)(e >> 3) * rstride + (e & 7);
        float p[K];
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = src[base + off[k]];
        // q_k = p_k - p_0: X_m(q) = X_m(p) for m != 0, and X_0(p) = X_0(q) + K p_0
        float q[K], a1 = 0.f;
        q[0] = 0.f;
#pragma unroll
        for (int k = 1; k < K; ++k) {
            q[k] = p[k] - p[0];
            a1 += fabsf(q[k]);
        }
        float xr[NM], xi[NM];
        rdft_half<K, 1, NM>(q, xr, xi);
        const float x0 = fmaf((float)K, p[0], xr[0]);
        lam[0] = fmaf(x0, x0, lam[0]);
#pragma unroll
        for (int m = 1; m < NM; ++m) lam[m] = fmaf(xr[m], xr[m], fmaf(xi[m], xi[m], lam[m]));
        // error bounds: X_m, m != 0, errs by at most sqrt(2) gamma_(K/4 + 3) sum_k |q_k| (the subtraction's
        // rounding added), X_0(p) by gamma_(log2 K + 2) (sum_k |q_k| + K |p_0|); both inside sqrt(2) (K + 3) u
        // times these sums, the bounds below
        const float a0 = fmaf((float)K, fabsf(p[0]), a1);
        e0sq = fmaf(a0, a0, e0sq);
        esq = fmaf(a1, a1, esq);
    }
    // warp sums of the NM eigenvalues and the two bound sums by a reduce-scatter: at each level a lane keeps
    // the half of its values that its lane bit selects and adds the partner's copy of that half, so that
    // after log2(NV) levels it holds the full sum of one value (index vidx); the addition depth per value
    // is the same as a butterfly's (five levels), inside the bound's 16 u lambda
    constexpr int NV = NM + 2 <= 8 ? 8 : NM + 2 <= 16 ? 16 : 32;
    float val[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) val[m] = m < NM ? lam[m] : m == NM ? e0sq : m == NM + 1 ? esq : 0.f;
    int vidx = 0;
#pragma unroll
    for (int lv = 0, o = 16, nv = NV; lv < 5; ++lv, o >>= 1) {
        if (nv > 1) {
            const int half = nv / 2;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float send = up ? val[i] : val[half + i];
                const float keep = up ? val[half + i] : val[i];
                val[i] = keep + __shfl_xor_sync(FULL, send, o);
            }
            vidx += up ? half : 0;
            nv = half;
        } else {
            val[0] += __shfl_xor_sync(FULL, val[0], o);
        }
    }
    // the bound terms and lambda_hat = lambda_{K/2} from the lanes holding them (value v sits in lane 2 v' where
    // v' has v's bits in lane bits 4..(5 - log2 NV), read from the first such lane)
    auto lane_of = [&](int v) {
        int l = 0;
#pragma unroll
        for (int lv = 0, o = 16, nv = NV; lv < 5 && nv > 1; ++lv, o >>= 1) {
            const int half = nv / 2;
            if (v >= half) {
                l |= o;
                v -= half;
            }
            nv = half;
        }
        return l;
    };
    const float e0s = __shfl_sync(FULL, val[0], lane_of(NM)), es = __shfl_sync(FULL, val[0], lane_of(NM + 1));
    // rigorous bound on |lambda32 - lambda|
    const float dx0 = 1.4143f * (float)(K + 3) * U32 * sqrtf(e0s) * 1.01f;
    const float dx = 1.4143f * (float)(K + 3) * U32 * sqrtf(es) * 1.01f;
    const float lm = val[0];
    const float dd = (vidx == 0) ? dx0 : dx;
    const float sl = sqrtf(fmaxf(lm, 0.f) * 1.02f);
    const float bm = (2.f * sl * dd + dd * dd) * 1.01f + 16.f * U32 * lm + 1e-30f;
    const float lh = __shfl_sync(FULL, lm, lane_of(K / 2)), bh = __shfl_sync(FULL, bm, lane_of(K / 2));
    // classification of lambda_m, m < K/2, one lane each (the first lane holding it), counted by ballots;
    // m and K - m give the same eigenvalue, so m >= 1 counts twice
    const bool mine_m = vidx < K / 2 && lane == lane_of(vidx);
    const bool s_below = mine_m && (lm + bm < lh - bh);
    const bool s_unc = mine_m && !(lm + bm < lh - bh) && !(lm - bm >= lh + bh);
    const unsigned bs = __ballot_sync(FULL, s_below), bu = __ballot_sync(FULL, s_unc);
    const unsigned l0 = 1u << lane_of(0);
    const int sure = 2 * __popc(bs) - ((bs & l0) ? 1 : 0);
    const int unc = 2 * __popc(bu) - ((bu & l0) ? 1 : 0);
    if ((double)(1 + sure + unc) <= gamma_rank) return 1;
    if ((double)(1 + sure) > gamma_rank) return 0;
    if (lane == 0) {  // decided in FP64 by k_vote_exact
        const int pos = atomicAdd(&st->vote_uncertain, 1);
        list[pos] = r;
    }
    return 0;
}

// Row stride (floats) of the vote's staged region: the width rounded up to 8 mod 32, so that a warp's 32
// components (4 rows x 8 pixels of a patch) fall in 32 distinct banks.
__host__ __device__ constexpr int vote_stride(int w) { return w + ((8 - w) & 31); }
constexpr int VT = 8;        // reference tile: VT x VT references
constexpr int VNT = 256;     // threads per block (8 warps)

// The rank vote over tiles of VT x VT references: a block stages the tile's search region (every channel,
// FP32, exactly the image's values) in shared memory and its warps take the tile's groups in turn; the
// arithmetic of a group is vote_group's, on the staged values (a group with a member outside the region,
// which no matcher produces, reads the image instead).  Each block adds its votes once (integer, order-free).
template <int C, int K>
__global__ void __launch_bounds__(VNT) k_vote(const float *__restrict__ img, int H, int W,
                                              const int32_t *__restrict__ idx, int nx, int ny, int step, int R,
                                              double gamma_rank, int32_t *__restrict__ list, DevState *st) {
    extern __shared__ float vreg[];
    __shared__ int s_votes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_votes = 0;
    const size_t HW = (size_t)H * W;
    const int ntx = (nx + VT - 1) / VT, ntiles = ntx * ((ny + VT - 1) / VT);
    int my_votes = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int gy0 = (tile / ntx) * VT, gx0 = (tile % ntx) * VT;
        const int gy1 = min(ny, gy0 + VT) - 1, gx1 = min(nx, gx0 + VT) - 1;
        const int ry0 = max(0, grid_pos(gy0, H, step) - R), ry1 = min(H - 1, grid_pos(gy1, H, step) + R + PS - 1);
        const int rx0 = max(0, grid_pos(gx0, W, step) - R), rx1 = min(W - 1, grid_pos(gx1, W, step) + R + PS - 1);
        const int rh = ry1 - ry0 + 1, rw = rx1 - rx0 + 1, rs = vote_stride(rw);
        const size_t plane = (size_t)rh * rs;
        __syncthreads();  // the previous tile's groups are done with the region
        {
            // element e = tid + i VNT: column x, region row `row` = channel c, row y; advanced by VNT per step
            const int dq = VNT / rw, dr = VNT - dq * rw;
            int row = tid / rw, x = tid - row * rw;
            int c = row / rh, y = row - c * rh;
            for (int e0 = 0; e0 < C * rh * rw; e0 += 8 * VNT) {
                float v[8];
                int dst[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool in = c < C;
                    dst[i] = in ? (c * rh + y) * rs + x : -1;
                    v[i] = in ? __ldg(img + c * HW + (size_t)(ry0 + y) * W + rx0 + x) : 0.f;
                    x += dr;
                    row += dq;
                    y += dq;
                    if (x >= rw) {
                        x -= rw;
                        ++row;
                        ++y;
                    }
                    while (y >= rh) {
                        y -= rh;
                        ++c;
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (dst[i] >= 0) vreg[dst[i]] = v[i];
            }
        }
        __syncthreads();
        const int tw = gx1 - gx0 + 1, ng = (gy1 - gy0 + 1) * tw;
        for (int t = warp; t < ng; t += VNT / 32) {
            const int gy = gy0 + t / tw, gx = gx0 + t % tw, r = gy * nx + gx;
            const int pos = (lane < K) ? idx[(size_t)r * K + lane] : 0;
            const int py = pos / W, px = pos - py * W;
            const bool inside = lane >= K || (py >= ry0 && py + PS - 1 <= ry1 && px >= rx0 && px + PS - 1 <= rx1);
            int off[K];
            if (__all_sync(FULL, inside)) {
                const int mine = (py - ry0) * rs + (px - rx0);
                if (!HTS_IN_BOUNDS(lane >= K || mine + (C - 1) * (int)plane + (PS - 1) * rs + PS - 1 < C * (int)plane,
                                   &st->error))
                    continue;  // (the check build: the staged region would be overrun)
#pragma unroll
                for (int k = 0; k < K; ++k) off[k] = __shfl_sync(FULL, mine, k);
                my_votes += vote_group<C, K>(vreg, plane, rs, off, gamma_rank, r, list, st);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) off[k] = __shfl_sync(FULL, pos, k);
                my_votes += vote_group<C, K>(img, HW, W, off, gamma_rank, r, list, st);
            }
        }
    }
    if (lane == 0) atomicAdd(&s_votes, my_votes);
    __syncthreads();
    if (tid == 0) atomicAdd(&st->votes, s_votes);
}

// The groups k_vote could not settle, decided in FP64: a cluster of VX
// blocks per listed group, block b summing the components of slice b (one
// thread per component, fixed-order block sum); block 0 adds the slices'
// sums in slice order through distributed shared memory.  FP64 runs at a
// small fraction of the FP32 rate on this part, so a group's components are
// spread over VX SMs.
constexpr int VX = 4;

template <int C>
__host__ __device__ constexpr int vx_threads() {
    return ((C * NPIX + VX - 1) / VX + 31) / 32 * 32;
}

template <int C, int K>
__global__ void __launch_bounds__(vx_threads<C>()) k_vote_exact(const float *__restrict__ img, int H, int W,
                                                                const int32_t *__restrict__ idx, double gamma_rank,
                                                                const int32_t *__restrict__ list, DevState *st) {
    namespace cg = cooperative_groups;
    constexpr int NM = K / 2 + 1;
    constexpr int D = C * NPIX, SL = (D + VX - 1) / VX;
    __shared__ double sm[(vx_threads<C>() / 32) * NM];
    __shared__ double lam[NM];
    cg::cluster_group cl = cg::this_cluster();
    const int b = (int)cl.block_rank();
    const int ncl = gridDim.x / VX, cid = blockIdx.x / VX;
    const int n = *(volatile int *)&st->vote_uncertain;
    for (int g = cid; g < n; g += ncl) {
        const int r = list[g];
        lambda64_partial<C, K>(img, H, W, idx + (size_t)r * K, b * SL, min(D, (b + 1) * SL), sm, lam);
        cl.sync();  // every slice's sums are in its block's shared memory
        if (b == 0 && threadIdx.x == 0) {
            double tot[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) tot[m] = 0.0;
            for (int q = 0; q < VX; ++q) {
                const double *pl = cl.map_shared_rank(lam, q);
#pragma unroll
                for (int m = 0; m < NM; ++m) tot[m] += pl[m];
            }
            int a = 1;  // rank of lambda_{K/2} among all K (m and K-m share a value)
#pragma unroll
            for (int m = 0; m < K; ++m) {
                const int mm = (m <= K / 2) ? m : K - m;
                if (m != K / 2 && tot[mm] < tot[K / 2]) ++a;
            }
            if ((double)a <= gamma_rank) atomicAdd(&st->votes, 1);
        }
        cl.sync();  // block 0 has read every slice
    }
}

__global__ void k_sigma_final(DevState *st, int nref, int adjust, double beta, double tau_scale) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double se = st->sigma_est;
    const int adj = (adjust && 2 * st->votes > nref) ? 1 : 0;
    const double sh = adj ? se / beta : se;
    st->adjusted = adj;
    st->sigma_hat = sh;
    st->tau = tau_scale * sh;
    st->tau32 = (float)(tau_scale * sh);
    st->nref = nref;
}

__global__ void k_set_sigma(DevState *st, double sigma, int nref, double tau_scale) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->sigma_est = sigma;
    st->sigma_hat = sigma;
    st->adjusted = 0;
    st->votes = 0;
    st->vote_uncertain = 0;
    st->tau = tau_scale * sigma;
    st->tau32 = (float)(tau_scale * sigma);
    st->nref = nref;
}


template <int C, int K>
hts_status launch_vote(const float *img, const Geom &g, const int32_t *idx, double gamma_rank, int32_t *list,
                       DevState *st, cudaStream_t s) {
    // the largest tile region: VT x VT references, their windows and patches, cut to the image
    const int rh = std::min(g.H, (VT - 1) * g.step + 2 * g.R + PS), rw = std::min(g.W, (VT - 1) * g.step + 2 * g.R + PS);
    const size_t smem = (size_t)C * rh * vote_stride(rw) * sizeof(float);
    const void *fn = reinterpret_cast<const void *>(k_vote<C, K>);
    if (hts_status e = allow_smem(fn, smem); e != HTS_OK) return e;
    int dev = 0, nsm = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, VNT, smem);
    const int ntiles = ((g.nx + VT - 1) / VT) * ((g.ny + VT - 1) / VT);
    const int blocks = std::max(1, std::min(ntiles, nsm * std::max(per_sm, 1)));
    {
        KTimer kt("k_vote", s);
        k_vote<C, K><<<blocks, VNT, smem, s>>>(img, g.H, g.W, idx, g.nx, g.ny, g.step, g.R, gamma_rank, list, st);
    }
    if (hts_status e = check_launch("k_vote"); e != HTS_OK) return e;
    {
        KTimer kt("k_vote_exact", s);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(152);  // 38 clusters of VX blocks
        cfg.blockDim = dim3(vx_threads<C>());
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = VX;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_vote_exact<C, K>, img, g.H, g.W, idx, gamma_rank, list, st);
        if (e != cudaSuccess) return report(HTS_ECUDA, cudaGetErrorString(e));
    }
    return check_launch("k_vote_exact");
}

}  // namespace

double tau_scale(const Geom &g, const hts_params &p) {
    return p.tau_mult * sqrt(2.0 * log((double)g.C * g.K * PS * PS));
}

hts_status launch_sigma_floor(const Geom &g, const hts_params &p, const double *eig, DevState *st, cudaStream_t s) {
    const int ns = g.C / 2 + 1;
    {
        KTimer kt("k_sigma_est", s);
        k_sigma_est<<<1, 32, 0, s>>>(eig, ns * 2 * 8, g.nref, p.mp_correct, st);
    }
    return check_launch("k_sigma_est");
}

hts_status launch_sigma_vote(const float *img, const Geom &g, const hts_params &p, const int32_t *idx,
                             int32_t *list, DevState *st, cudaStream_t s) {
    const double gamma = p.gamma_rank > 0 ? p.gamma_rank : 13.0 * g.K / 32.0;
    if (p.adjust_rank) {
        hts_status e = HTS_EUNSUPPORTED;
#define HTS_VOTE_CASE(CC, KK) \
    if (g.C == CC && g.K == KK) e = launch_vote<CC, KK>(img, g, idx, gamma, list, st, s);
        HTS_VOTE_CASE(1, 2) HTS_VOTE_CASE(1, 4) HTS_VOTE_CASE(1, 8) HTS_VOTE_CASE(1, 16) HTS_VOTE_CASE(1, 32)
        HTS_VOTE_CASE(3, 2) HTS_VOTE_CASE(3, 4) HTS_VOTE_CASE(3, 8) HTS_VOTE_CASE(3, 16) HTS_VOTE_CASE(3, 32)
#undef HTS_VOTE_CASE
        if (e != HTS_OK) return e;
    }
    return HTS_OK;
}

hts_status launch_sigma_final(const Geom &g, const hts_params &p, DevState *st, cudaStream_t s) {
    {
        KTimer kt("k_sigma_final", s);
        k_sigma_final<<<1, 32, 0, s>>>(st, g.nref, p.adjust_rank, p.beta, tau_scale(g, p));
    }
    return check_launch("k_sigma_final");
}

hts_status launch_sigma(const float *img, const Geom &g, const hts_params &p, const double *eig, const int32_t *idx,
                        int32_t *list, DevState *st, cudaStream_t s) {
    if (hts_status e = launch_sigma_floor(g, p, eig, st, s); e != HTS_OK) return e;
    if (hts_status e = launch_sigma_vote(img, g, p, idx, list, st, s); e != HTS_OK) return e;
    return launch_sigma_final(g, p, st, s);
}

hts_status launch_set_sigma(double sigma, const Geom &g, const hts_params &p, DevState *st, cudaStream_t s) {
    {
        KTimer kt("k_set_sigma", s);
        k_set_sigma<<<1, 32, 0, s>>>(st, sigma, g.nref, tau_scale(g, p));
    }
    return check_launch("k_set_sigma");
}

}  // namespace hts
