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
    st->sigma_est = sqrt(s2);
    st->votes = 0;
    st->vote_uncertain = 0;
    st->nref = nref;
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

template <int C, int K>
__global__ void __launch_bounds__(128) k_vote(const float *__restrict__ img, int H, int W,
                                              const int32_t *__restrict__ idx, int nref, double gamma_rank,
                                              DevState *st) {
    constexpr int D = C * NPIX;
    constexpr int NM = K / 2 + 1;
    __shared__ int s_votes, s_unc;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_votes = 0;
        s_unc = 0;
    }
    __syncthreads();
    float twc[K], tws[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double c, s;
        twiddle64(j, K, c, s);
        twc[j] = (float)c;
        tws[j] = (float)s;
    }
    const size_t HW = (size_t)H * W;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int my_votes = 0, my_unc = 0;
    for (int r = gw; r < nref; r += nw) {
        int off[K];
        {
            const int mine = (lane < K) ? idx[(size_t)r * K + lane] : 0;
#pragma unroll
            for (int k = 0; k < K; ++k) off[k] = __shfl_sync(FULL, mine, k);
        }
        float lam[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) lam[m] = 0.f;
        float e0sq = 0.f, esq = 0.f;
        for (int d = lane; d < D; d += 32) {
            const int c = d / NPIX, e = d - c * NPIX;
            const size_t base = (size_t)c * HW + (size_t)(e >> 3) * W + (e & 7);
            float p[K];
#pragma unroll
            for (int k = 0; k < K; ++k) p[k] = __ldg(img + base + off[k]);
            float x0 = 0.f, a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                x0 += p[k];
                a0 += fabsf(p[k]);
            }
            lam[0] = fmaf(x0, x0, lam[0]);
            e0sq = fmaf(a0, a0, e0sq);
            float q[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                q[k] = p[k] - p[0];
                a1 += fabsf(q[k]);
            }
            esq = fmaf(a1, a1, esq);
#pragma unroll
            for (int m = 1; m < NM; ++m) {
                float xr = 0.f, xi = 0.f;
#pragma unroll
                for (int k = 1; k < K; ++k) {
                    const int j = (m * k) % K;
                    xr = fmaf(q[k], twc[j], xr);
                    xi = fmaf(q[k], tws[j], xi);
                }
                lam[m] = fmaf(xr, xr, fmaf(xi, xi, lam[m]));
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int m = 0; m < NM; ++m) lam[m] += __shfl_xor_sync(FULL, lam[m], o);
            e0sq += __shfl_xor_sync(FULL, e0sq, o);
            esq += __shfl_xor_sync(FULL, esq, o);
        }
        // rigorous bound on |lambda32 - lambda|
        const float dx0 = 1.4143f * (float)(K + 3) * U32 * sqrtf(e0sq) * 1.01f;
        const float dx = 1.4143f * (float)(K + 3) * U32 * sqrtf(esq) * 1.01f;
        float bnd[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const float dd = (m == 0) ? dx0 : dx;
            const float sl = sqrtf(fmaxf(lam[m], 0.f) * 1.02f);
            bnd[m] = (2.f * sl * dd + dd * dd) * 1.01f + 16.f * U32 * lam[m] + 1e-30f;
        }
        const float lh = lam[K / 2], bh = bnd[K / 2];
        int sure = 0, unc = 0;
#pragma unroll
        for (int m = 0; m < K / 2; ++m) {
            const int mult = (m == 0) ? 1 : 2;
            if (lam[m] + bnd[m] < lh - bh) sure += mult;
            else if (lam[m] - bnd[m] >= lh + bh) {
            } else unc += mult;
        }
        int vote;
        if ((double)(1 + sure + unc) <= gamma_rank) vote = 1;
        else if ((double)(1 + sure) > gamma_rank) vote = 0;
        else {
            // FP64: lambda_m for all m, rank of lambda_{K/2} (ties rank lowest)
            double l64[K];
#pragma unroll
            for (int m = 0; m < K; ++m) l64[m] = 0.0;
            for (int d = lane; d < D; d += 32) {
                const int c = d / NPIX, e = d - c * NPIX;
                const size_t base = (size_t)c * HW + (size_t)(e >> 3) * W + (e & 7);
                double p[K];
#pragma unroll
                for (int k = 0; k < K; ++k) p[k] = (double)__ldg(img + base + off[k]);
                for (int m = 0; m < K; ++m) {
                    double xr = 0.0, xi = 0.0;
                    for (int k = 0; k < K; ++k) {
                        double cc, ss;
                        twiddle64(m * k, K, cc, ss);
                        xr += p[k] * cc;
                        xi += p[k] * ss;
                    }
                    l64[m] += xr * xr + xi * xi;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1)
#pragma unroll
                for (int m = 0; m < K; ++m) l64[m] += __shfl_xor_sync(FULL, l64[m], o);
            int a = 1;
#pragma unroll
            for (int m = 0; m < K; ++m)
                if (m != K / 2 && l64[m] < l64[K / 2]) ++a;
            vote = ((double)a <= gamma_rank) ? 1 : 0;
            ++my_unc;
        }
        my_votes += vote;
    }
    if (lane == 0) {
        atomicAdd(&s_votes, my_votes);
        atomicAdd(&s_unc, my_unc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&st->votes, s_votes);
        atomicAdd(&st->vote_uncertain, s_unc);
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

double tau_scale(const Geom &g, const hts_params &p) {
    return p.tau_mult * sqrt(2.0 * log((double)g.C * g.K * PS * PS));
}

template <int C, int K>
hts_status launch_vote(const float *img, const Geom &g, const int32_t *idx, double gamma_rank, DevState *st,
                       cudaStream_t s) {
    int blocks = (g.nref + 3) / 4;
    if (blocks > 152 * 8) blocks = 152 * 8;
    {
        KTimer kt("k_vote", s);
        k_vote<C, K><<<blocks, 128, 0, s>>>(img, g.H, g.W, idx, g.nref, gamma_rank, st);
    }
    return check_launch("k_vote");
}

}  // namespace

hts_status launch_sigma(const float *img, const Geom &g, const hts_params &p, const double *eig, const int32_t *idx,
                        DevState *st, cudaStream_t s) {
    const int ns = g.C / 2 + 1;
    {
        KTimer kt("k_sigma_est", s);
        k_sigma_est<<<1, 32, 0, s>>>(eig, ns * 2 * 8, g.nref, p.mp_correct, st);
    }
    if (hts_status e = check_launch("k_sigma_est"); e != HTS_OK) return e;
    const double gamma = p.gamma_rank > 0 ? p.gamma_rank : 13.0 * g.K / 32.0;
    if (p.adjust_rank) {
        hts_status e = HTS_EUNSUPPORTED;
#define HTS_VOTE_CASE(CC, KK) \
    if (g.C == CC && g.K == KK) e = launch_vote<CC, KK>(img, g, idx, gamma, st, s);
        HTS_VOTE_CASE(1, 2) HTS_VOTE_CASE(1, 4) HTS_VOTE_CASE(1, 8) HTS_VOTE_CASE(1, 16) HTS_VOTE_CASE(1, 32)
        HTS_VOTE_CASE(3, 2) HTS_VOTE_CASE(3, 4) HTS_VOTE_CASE(3, 8) HTS_VOTE_CASE(3, 16) HTS_VOTE_CASE(3, 32)
#undef HTS_VOTE_CASE
        if (e != HTS_OK) return e;
    }
    {
        KTimer kt("k_sigma_final", s);
        k_sigma_final<<<1, 32, 0, s>>>(st, g.nref, p.adjust_rank, p.beta, tau_scale(g, p));
    }
    return check_launch("k_sigma_final");
}

hts_status launch_set_sigma(double sigma, const Geom &g, const hts_params &p, DevState *st, cudaStream_t s) {
    {
        KTimer kt("k_set_sigma", s);
        k_set_sigma<<<1, 32, 0, s>>>(st, sigma, g.nref, tau_scale(g, p));
    }
    return check_launch("k_set_sigma");
}

}  // namespace hts
