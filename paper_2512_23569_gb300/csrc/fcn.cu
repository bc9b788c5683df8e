// The enhancement strategy's network on sm_103a (RA-Haar-tSVD, Eq. 24-25):
// a plain fully connected network that refines the mean patch of every
// group, trained by the library's own kernels with residual learning.
//
// The mean patch enters in the image's transform coordinates (k_mean_coefs:
// Eq. 19 without the Haar factor, [S^(1), sqrt 2 Re S^(2), sqrt 2 Im S^(2)],
// orthonormal, canonical eigenvector phases), where it is sparse, in units of
// its noise level s = sigma / sqrt(K).  Input: g(c / s), g(x) = x / (1 + |x|
// / 16), then sigma / 255, zero-padded to a multiple of 16; two hidden layers
// of 128 ReLU units; a linear output of C x 64 values, the residual in noise
// units: refined = c + s x output.  FP32 weights and arithmetic.  The layers are GEMMs
// over a batch of groups (k_gemm: 64 x 64 output tiles, 16-deep slabs in
// shared memory, 4 x 4 outputs per thread); the weight gradients reduce
// over the batch with a split of the reduction and a fixed-order sum of the
// parts, so training is deterministic.
//
// Denoising (hts_denoise_ra): the mean patch of every group (k_group_means),
// its coordinates, the network with the call's estimated sigma, the refined
// patch back in pixels (k_coefs_to_patch), and the refined patches go to the
// tensor-core filter, which drops each group's first Haar row and
// adds the refined mean to every member's estimate instead (the same as
// replacing that row by sqrt(K) times the refined mean's transform and not
// thresholding it).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hts_internal.h"

namespace hts {
namespace {

constexpr int HID = 128;
constexpr int NL = 3;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;
constexpr int TM = 64, TN = 64, TK = 16;  // GEMM tile
constexpr float SAT = 16.f;                // saturation of the input compression
constexpr float K3F = 0.57735026918962576f;  // 1/sqrt(3)
constexpr float SQ2 = 1.41421356237309505f;

}  // namespace
}  // namespace hts

struct hts_fcn {
    int C = 1, K = 16, device = 0, nparams = 0, t = 0, din = 0, dout = 0;
    int off[3] = {}, nin[3] = {}, nout[3] = {};
    float *w = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    size_t cap = 0;                       // samples the activation buffers hold
    float *X = nullptr;                   // features [n][din]
    float *act[3] = {};                   // layer outputs [n][nout[l]]
    float *d0 = nullptr, *d1 = nullptr;   // gradients of layer outputs [n][HID or dout]
    size_t cap_part = 0;
    float *part = nullptr;                // split-reduction parts
    double *loss = nullptr;               // accumulated loss
    double *lpart = nullptr;              // per-block loss parts
    float *sig = nullptr;                 // the call's sigma for the features (denoising)
};

namespace hts {
namespace {

#define HTS_TRY(expr)                \
    do {                             \
        hts_status _s = (expr);      \
        if (_s != HTS_OK) return _s; \
    } while (0)

hts_status cu(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HTS_OK;
    char buf[160];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return report(e == cudaErrorMemoryAllocation ? HTS_ENOMEM : HTS_ECUDA, buf);
}

// C(m, n) = sum_k A(m, k) B(n, k), A(m, k) = A[m * am + k * ak], B(n, k) = B[n * bn + k * bk].
// parts == nullptr: Cout[m * ldc + n] = act(C + bias[n]) (act: 1 = ReLU, 2 = times (mask[m * ldc + n] > 0));
// else the reduction range [z * kchunk, (z + 1) * kchunk) of block z goes to parts[z][m][n] as it is.
__global__ void __launch_bounds__(256) k_gemm(const float *__restrict__ A, long am, long ak, const float *__restrict__ B,
                                              long bn, long bk, int M, int N, int K, int kchunk,
                                              const float *__restrict__ bias, int act, const float *__restrict__ mask,
                                              float *__restrict__ Cout, int ldc, float *__restrict__ parts) {
    __shared__ float sA[TK][TM + 4], sB[TK][TN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int k0 = blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
    float acc[4][4] = {};
    for (int kb = k0; kb < k1; kb += TK) {
        for (int e = tid; e < TK * TM; e += 256) {
            const int kk = e / TM, mm = e - kk * TM;  // consecutive threads: consecutive m
            const int gm = m0 + mm, gk = kb + kk;
            sA[kk][mm] = (gm < M && gk < k1) ? A[(long)gm * am + (long)gk * ak] : 0.f;
        }
        for (int e = tid; e < TK * TN; e += 256) {
            const int kk = e / TN, nn = e - kk * TN;
            const int gn = n0 + nn, gk = kb + kk;
            sB[kk][nn] = (gn < N && gk < k1) ? B[(long)gn * bn + (long)gk * bk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = sA[kk][ty * 4 + i];
                b[i] = sB[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            if (parts) {
                parts[((long)blockIdx.z * M + gm) * N + gn] = acc[i][j];
            } else {
                float r = acc[i][j] + (bias ? bias[gn] : 0.f);
                if (act == 1) r = fmaxf(r, 0.f);
                if (act == 2) r = mask[(long)gm * ldc + gn] > 0.f ? r : 0.f;
                Cout[(long)gm * ldc + gn] = r;
            }
        }
    }
}

// out[e] += sum over z of parts[z][e], in z order.
__global__ void k_sum_parts(const float *__restrict__ parts, int nz, long ne, float *__restrict__ out) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ne; e += (long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < nz; ++z) s += parts[(long)z * ne + e];
        out[e] += s;
    }
}

// db[o] += sum over n of dY[n][o], n in order.
__global__ void k_bias_grad(const float *__restrict__ dY, int n, int o, float *__restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= o) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += dY[(long)i * o + j];
    db[j] += s;
}

// Mean patch of group r (channel t, pixel (u, v)) over its K members, members in order.
__global__ void k_group_means(const float *__restrict__ img, int H, int W, int C, const int32_t *__restrict__ idx, int K,
                              int nref, float *__restrict__ means) {
    const long total = (long)nref * C * 64;
    const size_t HW = (size_t)H * W;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / (C * 64)), e = (int)(i - (long)r * C * 64);
        const int t = e >> 6, u = (e >> 3) & 7, v = e & 7;
        float s = 0.f;
        for (int k = 0; k < K; ++k) {
            const int pos = idx[(long)r * K + k];
            s += img[t * HW + (size_t)pos + (size_t)u * W + v];
        }
        means[i] = s / (float)K;
    }
}

// Features: g(coordinate / s) with s = sigma / sqrt(K), g(x) = x / (1 + |x| / SAT); sigma / 255
// (sigma[i * sstride]); zeros.
__global__ void k_features(const float *__restrict__ coords, const float *__restrict__ sigma, int sstride, int n,
                           int d, int din, float rsqrt_k, float *__restrict__ X) {
    const long total = (long)n * din;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int s = (int)(i / din), c = (int)(i - (long)s * din);
        const float sg = sigma[(long)s * sstride];
        float v = 0.f;
        if (c < d) {
            const float x = coords[(long)s * d + c] / (sg * rsqrt_k);
            v = x / (1.f + fabsf(x) * (1.f / SAT));
        } else if (c == d) {
            v = sg * (1.f / 255.f);
        }
        X[i] = v;
    }
}

// sigma of the call (double in the state) as a float for the features.
__global__ void k_state_sigma(const DevState *st, float *out) { *out = (float)st->sigma_hat; }

// Loss parts: block b sums (out - (clean - noisy) / s)^2 over its stride (s = sigma / sqrt(K) of the
// sample, d values per sample); dout = 2 (out - target) / total.
__global__ void __launch_bounds__(256) k_fcn_loss(const float *__restrict__ out, const float *__restrict__ noisy,
                                                  const float *__restrict__ clean, const float *__restrict__ sigma,
                                                  int d, float rsqrt_k, long total, float *__restrict__ dout,
                                                  double *lpart) {
    __shared__ double red[8];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const float e = out[i] - (clean[i] - noisy[i]) / (sigma[i / d] * rsqrt_k);
        dout[i] = 2.f * e / (float)total;
        s += (double)e * e;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        lpart[blockIdx.x] = t;
    }
}

__global__ void k_loss_sum(const double *lpart, int nb, long total, double *loss) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += lpart[b];
    *loss += t / (double)total;
}

__global__ void k_fcn_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int n, float lr, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = ADAM_B1 * m[i] + (1.f - ADAM_B1) * gi;
        const float vi = ADAM_B2 * v[i] + (1.f - ADAM_B2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + ADAM_EPS);
    }
}

// refined[i] = coords[i] + s out[i], s = sigma[sample * sstride] / sqrt(K)
__global__ void k_refine(const float *__restrict__ coords, const float *__restrict__ out, const float *__restrict__ sigma,
                         int sstride, int d, float rsqrt_k, long total, float *__restrict__ refined) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
        refined[i] = coords[i] + sigma[(i / d) * sstride] * rsqrt_k * out[i];
}

// Column c of an 8x8 basis (element (r, c) at r * 8 + c) multiplied by the conjugate phase of its
// largest-magnitude entry (ties to the lower row): the entry becomes real positive.  Eigenvectors are
// defined up to that phase; the network's coordinates need one fixed choice.
__device__ void canon_column(float *re, float *im, int c) {
    int best = 0;
    float bm = -1.f;
    for (int r = 0; r < 8; ++r) {
        const float x = re[r * 8 + c], y = im ? im[r * 8 + c] : 0.f;
        const float m2 = x * x + y * y;
        if (m2 > bm) {
            bm = m2;
            best = r;
        }
    }
    const float x = re[best * 8 + c], y = im ? im[best * 8 + c] : 0.f;
    const float inv = bm > 0.f ? rsqrtf(bm) : 1.f;
    const float pr = x * inv, pi = y * inv;  // phase; multiply the column by its conjugate
    for (int r = 0; r < 8; ++r) {
        const float a = re[r * 8 + c], b = im ? im[r * 8 + c] : 0.f;
        re[r * 8 + c] = a * pr + b * pi;
        if (im) im[r * 8 + c] = b * pr - a * pi;
    }
}

// Basis slices of the FP32 device copy ([j][U/V][8][8][re/im]) in shared memory, columns in the
// canonical phase (canon_column).
template <int C>
__device__ void load_bases(const float *__restrict__ b32, float (&u0)[64], float (&v0)[64], float (&u1r)[64],
                           float (&u1i)[64], float (&v1r)[64], float (&v1i)[64]) {
    const int t = threadIdx.x;
    u0[t] = b32[(0 * 64 + t) * 2];
    v0[t] = b32[(1 * 64 + t) * 2];
    if (C == 3) {
        u1r[t] = b32[(2 * 64 + t) * 2];
        u1i[t] = b32[(2 * 64 + t) * 2 + 1];
        v1r[t] = b32[(3 * 64 + t) * 2];
        v1i[t] = b32[(3 * 64 + t) * 2 + 1];
    }
    __syncthreads();
    if (t < 8) canon_column(u0, nullptr, t);
    else if (t < 16) canon_column(v0, nullptr, t - 8);
    else if (C == 3 && t < 24) canon_column(u1r, u1i, t - 16);
    else if (C == 3 && t < 32) canon_column(v1r, v1i, t - 24);
}

// Coordinates of patch r (one block of 64 threads per patch, thread = pixel / coefficient (a, b)):
// the DFT along the channels, T = Phat V, S = U^H T (Eq. 19 without the Haar factor); out
// [S^(1) | sqrt 2 Re S^(2) | sqrt 2 Im S^(2)] (orthonormal).
template <int C>
__global__ void __launch_bounds__(64) k_mean_coefs(const float *__restrict__ means, const float *__restrict__ b32,
                                                   float *__restrict__ coefs) {
    __shared__ float u0[64], v0[64], u1r[64], u1i[64], v1r[64], v1i[64];
    __shared__ float p0[64], pr[64], pi[64], t0[64], tr[64], ti[64];
    const int t = threadIdx.x, r = blockIdx.x;
    load_bases<C>(b32, u0, v0, u1r, u1i, v1r, v1i);
    const float *m = means + (size_t)r * C * 64;
    if (C == 1) {
        p0[t] = m[t];
    } else {
        const float R = m[t], G = m[64 + t], B = m[128 + t];
        p0[t] = ((R + G) + B) * K3F;
        pr[t] = (R - 0.5f * (G + B)) * K3F;
        pi[t] = (B - G) * 0.5f;
    }
    __syncthreads();
    const int hi = t >> 3, lo = t & 7;
    {  // T[i][b] = sum_j Phat[i][j] V[j][b], thread (i, b) = (hi, lo)
        float a0 = 0.f, ar = 0.f, ai = 0.f;
        for (int j = 0; j < 8; ++j) {
            a0 = fmaf(p0[hi * 8 + j], v0[j * 8 + lo], a0);
            if (C == 3) {
                const float xr = pr[hi * 8 + j], xi = pi[hi * 8 + j], yr = v1r[j * 8 + lo], yi = v1i[j * 8 + lo];
                ar = fmaf(xr, yr, fmaf(-xi, yi, ar));
                ai = fmaf(xr, yi, fmaf(xi, yr, ai));
            }
        }
        t0[t] = a0;
        tr[t] = ar;
        ti[t] = ai;
    }
    __syncthreads();
    {  // S[a][b] = sum_i conj(U[i][a]) T[i][b], thread (a, b) = (hi, lo)
        float s0 = 0.f, sr = 0.f, si = 0.f;
        for (int i = 0; i < 8; ++i) {
            s0 = fmaf(u0[i * 8 + hi], t0[i * 8 + lo], s0);
            if (C == 3) {
                const float ur = u1r[i * 8 + hi], ui = u1i[i * 8 + hi], xr = tr[i * 8 + lo], xi = ti[i * 8 + lo];
                sr = fmaf(ur, xr, fmaf(ui, xi, sr));
                si = fmaf(ur, xi, fmaf(-ui, xr, si));
            }
        }
        float *o = coefs + (size_t)r * C * 64;
        o[t] = s0;
        if (C == 3) {
            o[64 + t] = SQ2 * sr;
            o[128 + t] = SQ2 * si;
        }
    }
}

// Inverse of k_mean_coefs: Phat = U S V^H per slice, then the inverse DFT along the channels.
template <int C>
__global__ void __launch_bounds__(64) k_coefs_to_patch(const float *__restrict__ coefs, const float *__restrict__ b32,
                                                       float *__restrict__ patches) {
    __shared__ float u0[64], v0[64], u1r[64], u1i[64], v1r[64], v1i[64];
    __shared__ float s0[64], sr[64], si[64], q0[64], qr[64], qi[64];
    const int t = threadIdx.x, r = blockIdx.x;
    load_bases<C>(b32, u0, v0, u1r, u1i, v1r, v1i);
    const float *c = coefs + (size_t)r * C * 64;
    s0[t] = c[t];
    if (C == 3) {
        sr[t] = c[64 + t] * (1.f / SQ2);
        si[t] = c[128 + t] * (1.f / SQ2);
    }
    __syncthreads();
    const int hi = t >> 3, lo = t & 7;
    {  // Q[a][j] = sum_b S[a][b] conj(V[j][b]), thread (a, j) = (hi, lo)
        float a0 = 0.f, ar = 0.f, ai = 0.f;
        for (int b = 0; b < 8; ++b) {
            a0 = fmaf(s0[hi * 8 + b], v0[lo * 8 + b], a0);
            if (C == 3) {
                const float xr = sr[hi * 8 + b], xi = si[hi * 8 + b], yr = v1r[lo * 8 + b], yi = v1i[lo * 8 + b];
                ar = fmaf(xr, yr, fmaf(xi, yi, ar));
                ai = fmaf(xi, yr, fmaf(-xr, yi, ai));
            }
        }
        q0[t] = a0;
        qr[t] = ar;
        qi[t] = ai;
    }
    __syncthreads();
    {  // Phat[i][j] = sum_a U[i][a] Q[a][j], thread (i, j) = (hi, lo); then the inverse channel DFT
        float f0 = 0.f, fr = 0.f, fi = 0.f;
        for (int a = 0; a < 8; ++a) {
            f0 = fmaf(u0[hi * 8 + a], q0[a * 8 + lo], f0);
            if (C == 3) {
                const float ur = u1r[hi * 8 + a], ui = u1i[hi * 8 + a], xr = qr[a * 8 + lo], xi = qi[a * 8 + lo];
                fr = fmaf(ur, xr, fmaf(-ui, xi, fr));
                fi = fmaf(ur, xi, fmaf(ui, xr, fi));
            }
        }
        float *o = patches + (size_t)r * C * 64;
        if (C == 1) {
            o[t] = f0;
        } else {
            o[t] = (f0 + 2.f * fr) * K3F;
            o[64 + t] = (f0 - fr - 1.7320508075688772f * fi) * K3F;
            o[128 + t] = (f0 - fr + 1.7320508075688772f * fi) * K3F;
        }
    }
}

constexpr int LOSS_BLOCKS = 304;

void layout(hts_fcn *f) {
    f->din = (f->C * 64 + 1 + 15) / 16 * 16;
    f->dout = f->C * 64;
    const int ins[NL] = {f->din, HID, HID}, outs[NL] = {HID, HID, f->dout};
    int o = 0;
    for (int l = 0; l < NL; ++l) {
        f->nin[l] = ins[l];
        f->nout[l] = outs[l];
        f->off[l] = o;
        o += ins[l] * outs[l] + outs[l];
    }
    f->nparams = o;
}

hts_status ensure(hts_fcn *f, size_t n) {
    if (n > f->cap) {
        cudaFree(f->X);
        for (float *&p : f->act) {
            cudaFree(p);
            p = nullptr;
        }
        cudaFree(f->d0);
        cudaFree(f->d1);
        f->X = f->d0 = f->d1 = nullptr;
        f->cap = 0;
        HTS_TRY(cu(dev_malloc(&f->X, n * f->din * sizeof(float)), "cudaMalloc(fcn)"));
        for (int l = 0; l < NL; ++l) HTS_TRY(cu(dev_malloc(&f->act[l], n * f->nout[l] * sizeof(float)), "cudaMalloc(fcn)"));
        const size_t wd = std::max(HID, f->dout);
        HTS_TRY(cu(dev_malloc(&f->d0, n * wd * sizeof(float)), "cudaMalloc(fcn)"));
        HTS_TRY(cu(dev_malloc(&f->d1, n * wd * sizeof(float)), "cudaMalloc(fcn)"));
        f->cap = n;
    }
    return HTS_OK;
}

int nsm() {
    int dev = 0, n = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

hts_status gemm(const float *A, long am, long ak, const float *B, long bn, long bk, int M, int N, int K,
                const float *bias, int act, const float *mask, float *Cout, int ldc, cudaStream_t s) {
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, 1);
    {
        KTimer kt("k_fcn_gemm", s);
        k_gemm<<<grid, 256, 0, s>>>(A, am, ak, B, bn, bk, M, N, K, K, bias, act, mask, Cout, ldc, nullptr);
    }
    return check_launch("k_fcn_gemm");
}

// out[M][N] += sum_k A(m, k) B(n, k) with the reduction split over blocks and summed in a fixed order.
hts_status gemm_acc(hts_fcn *f, const float *A, long am, long ak, const float *B, long bn, long bk, int M, int N,
                    int K, float *out, cudaStream_t s) {
    const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
    int nz = std::max(1, std::min((2 * nsm() + tiles - 1) / tiles, (K + 255) / 256));
    const int kchunk = ((K + nz - 1) / nz + TK - 1) / TK * TK;
    nz = (K + kchunk - 1) / kchunk;
    const size_t need = (size_t)nz * M * N;
    if (need > f->cap_part) {
        cudaFree(f->part);
        f->part = nullptr;
        f->cap_part = 0;
        HTS_TRY(cu(dev_malloc(&f->part, need * sizeof(float)), "cudaMalloc(fcn)"));
        f->cap_part = need;
    }
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, nz);
    {
        KTimer kt("k_fcn_gemm", s);
        k_gemm<<<grid, 256, 0, s>>>(A, am, ak, B, bn, bk, M, N, K, kchunk, nullptr, 0, nullptr, nullptr, 0, f->part);
    }
    HTS_TRY(check_launch("k_fcn_gemm"));
    const long ne = (long)M * N;
    {
        KTimer kt("k_sum_parts", s);
        k_sum_parts<<<(unsigned)std::min<long>((ne + 255) / 256, 1024), 256, 0, s>>>(f->part, nz, ne, out);
    }
    return check_launch("k_sum_parts");
}

// Forward of n samples whose features are in f->X; output in f->act[2].
hts_status forward(hts_fcn *f, int n, cudaStream_t s) {
    const float *in = f->X;
    for (int l = 0; l < NL; ++l) {
        HTS_TRY(gemm(in, f->nin[l], 1, f->w + f->off[l], f->nin[l], 1, n, f->nout[l], f->nin[l],
                     f->w + f->off[l] + f->nout[l] * f->nin[l], l < NL - 1 ? 1 : 0, nullptr, f->act[l], f->nout[l],
                     s));
        in = f->act[l];
    }
    return HTS_OK;
}

hts_status features(hts_fcn *f, const float *means, const float *sigma, int sstride, int n, cudaStream_t s) {
    const long total = (long)n * f->din;
    {
        KTimer kt("k_fcn_features", s);
        k_features<<<(unsigned)std::min<long>((total + 255) / 256, 4096), 256, 0, s>>>(
            means, sigma, sstride, n, f->dout, f->din, 1.f / std::sqrt((float)f->K), f->X);
    }
    return check_launch("k_fcn_features");
}

hts_status upload(hts_fcn *f, const float *host) {
    HTS_TRY(cu(cudaMemcpy(f->w, host, f->nparams * sizeof(float), cudaMemcpyHostToDevice), "cudaMemcpy"));
    for (float *p : {f->grad, f->m, f->v}) HTS_TRY(cu(cudaMemset(p, 0, f->nparams * sizeof(float)), "cudaMemset"));
    f->t = 0;
    return HTS_OK;
}

void free_fcn(hts_fcn *f) {
    if (!f) return;
    for (float *p : {f->w, f->grad, f->m, f->v, f->X, f->d0, f->d1, f->part}) cudaFree(p);
    for (float *p : f->act) cudaFree(p);
    cudaFree(f->loss);
    cudaFree(f->lpart);
    cudaFree(f->sig);
    delete f;
}

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

hts_status launch_group_means(const float *img, const Geom &g, const int32_t *idx, float *means, cudaStream_t s) {
    const long total = (long)g.nref * g.C * 64;
    {
        KTimer kt("k_group_means", s);
        k_group_means<<<(unsigned)std::min<long>((total + 255) / 256, 8192), 256, 0, s>>>(img, g.H, g.W, g.C, idx,
                                                                                          g.K, g.nref, means);
    }
    return check_launch("k_group_means");
}

hts_status launch_mean_transform(const float *in, int n, int C, const float *b32, bool inverse, float *out,
                                 cudaStream_t s) {
    if (n == 0) return HTS_OK;
    KTimer kt(inverse ? "k_coefs_to_patch" : "k_mean_coefs", s);
    if (C == 1) {
        if (inverse) k_coefs_to_patch<1><<<n, 64, 0, s>>>(in, b32, out);
        else k_mean_coefs<1><<<n, 64, 0, s>>>(in, b32, out);
    } else {
        if (inverse) k_coefs_to_patch<3><<<n, 64, 0, s>>>(in, b32, out);
        else k_mean_coefs<3><<<n, 64, 0, s>>>(in, b32, out);
    }
    return check_launch(inverse ? "k_coefs_to_patch" : "k_mean_coefs");
}

// Refined mean patches (pixels) of the groups whose mean patches are in buf (n x C x 64; overwritten),
// with the call's sigma from the state; result in out (n x C x 64).
hts_status fcn_refine_state(hts_fcn *f, float *buf, int n, const DevState *st, const float *b32, float *out,
                            cudaStream_t s) {
    HTS_TRY(ensure(f, n));
    HTS_TRY(launch_mean_transform(buf, n, f->C, b32, false, out, s));  // coordinates in out
    {
        KTimer kt("k_state_sigma", s);
        k_state_sigma<<<1, 1, 0, s>>>(st, f->sig);
    }
    HTS_TRY(check_launch("k_state_sigma"));
    HTS_TRY(features(f, out, f->sig, 0, n, s));
    HTS_TRY(forward(f, n, s));
    const long total = (long)n * f->dout;
    {
        KTimer kt("k_fcn_refine", s);
        k_refine<<<(unsigned)std::min<long>((total + 255) / 256, 8192), 256, 0, s>>>(
            out, f->act[NL - 1], f->sig, 0, f->dout, 1.f / std::sqrt((float)f->K), total, buf);
    }
    HTS_TRY(check_launch("k_fcn_refine"));
    return launch_mean_transform(buf, n, f->C, b32, true, out, s);  // refined patch in pixels
}

}  // namespace hts

using namespace hts;

extern "C" int hts_fcn_num_params(int C) {
    if (C != 1 && C != 3) return 0;
    hts_fcn f;
    f.C = C;
    layout(&f);
    return f.nparams;
}

extern "C" int hts_fcn_channels(const hts_fcn *f) { return f ? f->C : 0; }

extern "C" int hts_fcn_group_size(const hts_fcn *f) { return f ? f->K : 0; }

extern "C" hts_status hts_fcn_create(int C, int K, uint64_t seed, hts_fcn **out) {
    if (!out) return report(HTS_EINVAL, "NULL pointer");
    if (C != 1 && C != 3) return report(HTS_EINVAL, "C must be 1 or 3");
    if (K < 2 || K > 32 || (K & (K - 1))) return report(HTS_EINVAL, "K must be a power of 2 in 2..32");
    hts_fcn *f = new hts_fcn();
    f->C = C;
    f->K = K;
    layout(f);
    hts_status st = cu(cudaGetDevice(&f->device), "cudaGetDevice");
    for (float **p : {&f->w, &f->grad, &f->m, &f->v})
        if (st == HTS_OK) st = cu(dev_malloc(p, f->nparams * sizeof(float)), "cudaMalloc(fcn)");
    if (st == HTS_OK) st = cu(dev_malloc(&f->loss, sizeof(double)), "cudaMalloc(fcn)");
    if (st == HTS_OK) st = cu(cudaMemset(f->loss, 0, sizeof(double)), "cudaMemset");
    if (st == HTS_OK) st = cu(dev_malloc(&f->lpart, LOSS_BLOCKS * sizeof(double)), "cudaMalloc(fcn)");
    if (st == HTS_OK) st = cu(dev_malloc(&f->sig, sizeof(float)), "cudaMalloc(fcn)");
    if (st != HTS_OK) {
        free_fcn(f);
        return st;
    }
    // He initialisation of the hidden layers, the output layer 0.1x smaller (starts near the identity
    // refinement), biases zero; Box-Muller on a splitmix64 stream
    std::vector<float> h(f->nparams, 0.f);
    uint64_t x = seed;
    for (int l = 0; l < NL; ++l) {
        const double sd = std::sqrt(2.0 / f->nin[l]) * (l == NL - 1 ? 0.1 : 1.0);
        for (int i = 0; i < f->nout[l] * f->nin[l]; ++i) {
            const double u1 = ((splitmix64(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            const double u2 = ((splitmix64(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            h[f->off[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    st = upload(f, h.data());
    if (st != HTS_OK) {
        free_fcn(f);
        return st;
    }
    *out = f;
    return HTS_OK;
}

extern "C" hts_status hts_fcn_free(hts_fcn *f) {
    free_fcn(f);
    return HTS_OK;
}

extern "C" hts_status hts_fcn_get_params(const hts_fcn *f, float *host) {
    if (!f || !host) return report(HTS_EINVAL, "NULL pointer");
    return cu(cudaMemcpy(host, f->w, f->nparams * sizeof(float), cudaMemcpyDeviceToHost), "cudaMemcpy");
}

extern "C" hts_status hts_fcn_set_params(hts_fcn *f, const float *host) {
    if (!f || !host) return report(HTS_EINVAL, "NULL pointer");
    return upload(f, host);
}

extern "C" hts_status hts_group_means(const float *img, int H, int W, int C, const hts_params *p, const int32_t *idx,
                                      float *means, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!img || !idx || !means) return report(HTS_EINVAL, "NULL pointer");
    return launch_group_means(img, g, idx, means, static_cast<cudaStream_t>(stream));
}

extern "C" hts_status hts_mean_coefs(const float *in, int n, int C, const hts_basis *basis, int inverse, float *out,
                                     void *stream) {
    if (!in || !basis || !out) return report(HTS_EINVAL, "NULL pointer");
    if (n < 0) return report(HTS_EINVAL, "n < 0");
    if (C != basis->C) return report(HTS_EINVAL, "basis built for another channel count");
    return launch_mean_transform(in, n, C, basis->b32, inverse != 0, out, static_cast<cudaStream_t>(stream));
}

extern "C" hts_status hts_fcn_refine(hts_fcn *f, const float *means, const float *sigma, int n, float *refined,
                                     void *stream) {
    if (!f || !means || !sigma || !refined) return report(HTS_EINVAL, "NULL pointer");
    if (n < 0) return report(HTS_EINVAL, "n < 0");
    if (n == 0) return HTS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(ensure(f, n));
    HTS_TRY(features(f, means, sigma, 1, n, s));
    HTS_TRY(forward(f, n, s));
    const long total = (long)n * f->dout;
    {
        KTimer kt("k_fcn_refine", s);
        k_refine<<<(unsigned)std::min<long>((total + 255) / 256, 8192), 256, 0, s>>>(
            means, f->act[NL - 1], sigma, 1, f->dout, 1.f / std::sqrt((float)f->K), total, refined);
    }
    return check_launch("k_fcn_refine");
}

extern "C" hts_status hts_fcn_zero_grad(hts_fcn *f, void *stream) {
    if (!f) return report(HTS_EINVAL, "NULL pointer");
    return cu(cudaMemsetAsync(f->grad, 0, f->nparams * sizeof(float), static_cast<cudaStream_t>(stream)),
              "cudaMemsetAsync");
}

extern "C" hts_status hts_fcn_accumulate_grad(hts_fcn *f, const float *noisy_means, const float *clean_means,
                                              const float *sigma, int n, void *stream) {
    if (!f || !noisy_means || !clean_means || !sigma) return report(HTS_EINVAL, "NULL pointer");
    if (n <= 0) return report(HTS_EINVAL, "n must be > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(ensure(f, n));
    HTS_TRY(features(f, noisy_means, sigma, 1, n, s));
    HTS_TRY(forward(f, n, s));
    const long total = (long)n * f->dout;
    {
        KTimer kt("k_fcn_loss", s);
        k_fcn_loss<<<LOSS_BLOCKS, 256, 0, s>>>(f->act[NL - 1], noisy_means, clean_means, sigma, f->dout,
                                               1.f / std::sqrt((float)f->K), total, f->d0, f->lpart);
        k_loss_sum<<<1, 32, 0, s>>>(f->lpart, LOSS_BLOCKS, total, f->loss);
    }
    HTS_TRY(check_launch("k_fcn_loss"));
    // layer l: dY (n x nout) in dcur; dW += dY^T X_l, db += column sums, dX = (dY W) * (X_l > 0)
    float *dcur = f->d0, *dnext = f->d1;
    for (int l = NL - 1; l >= 0; --l) {
        const float *xin = l == 0 ? f->X : f->act[l - 1];
        const int ni = f->nin[l], no = f->nout[l];
        HTS_TRY(gemm_acc(f, dcur, 1, no, xin, 1, ni, no, ni, n, f->grad + f->off[l], s));
        {
            KTimer kt("k_fcn_bias_grad", s);
            k_bias_grad<<<(no + 127) / 128, 128, 0, s>>>(dcur, n, no, f->grad + f->off[l] + no * ni);
        }
        HTS_TRY(check_launch("k_fcn_bias_grad"));
        if (l > 0) {
            HTS_TRY(gemm(dcur, no, 1, f->w + f->off[l], 1, ni, n, ni, no, nullptr, 2, xin, dnext, ni, s));
            std::swap(dcur, dnext);
        }
    }
    return HTS_OK;
}

extern "C" hts_status hts_fcn_take_loss(hts_fcn *f, double *loss_sum, void *stream) {
    if (!f || !loss_sum) return report(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(cu(cudaMemcpyAsync(loss_sum, f->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync"));
    HTS_TRY(cu(cudaMemsetAsync(f->loss, 0, sizeof(double), s), "cudaMemsetAsync"));
    return cu(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

extern "C" hts_status hts_fcn_get_grad(const hts_fcn *f, float *host, void *stream) {
    if (!f || !host) return report(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(cu(cudaMemcpyAsync(host, f->grad, f->nparams * sizeof(float), cudaMemcpyDeviceToHost, s),
               "cudaMemcpyAsync"));
    return cu(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

extern "C" hts_status hts_fcn_adam_step(hts_fcn *f, float lr, void *stream) {
    if (!f) return report(HTS_EINVAL, "NULL pointer");
    if (!(lr > 0.f) || !std::isfinite(lr)) return report(HTS_EINVAL, "lr must be > 0");
    f->t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B1, f->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B2, f->t)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        KTimer kt("k_fcn_adam", s);
        k_fcn_adam<<<(f->nparams + 255) / 256, 256, 0, s>>>(f->w, f->grad, f->m, f->v, f->nparams, lr, c1, c2);
    }
    return check_launch("k_fcn_adam");
}
