// Learned noise-level map on sm_103a: the convolutional estimate of the
// noise level that the paper's adaptive variant uses in place of a single
// global value (Sec. III-C), trained here by the library's own kernels.
// This file holds the FP32 training path (forward with FP32 activations,
// backward, Adam), the readout and the host interface; the forward pass used
// for denoising and the default (FP16) training step run on the tensor cores
// (cnn_tc.cu).
//
// Network: the noisy image scaled by 1/255 goes through five 3x3
// convolutions with zero padding (widths C -> 32 -> 32 -> 32 -> 32 -> 1,
// ReLU after the first four) to a map of log(sigma) on the [0, 255] scale; a
// reference patch with top-left corner (y, x) reads it at (y + 4, x + 4).
// Weights and biases are FP16 in the forward pass (FP32 master copy for
// Adam), activations and accumulation FP32.
//
// k_conv_fwd        one 16 x 16 output tile per block, one pixel per thread,
//                   all output channels in registers; the input tile with its
//                   halo and the layer's weights staged in shared memory.
// k_conv_bwd_data   gradient of the layer input (correlation of the output
//                   gradient with the flipped kernels) times the ReLU mask.
// k_conv_bwd_weight per-tile partial sums of the weight and bias gradients,
//                   added by k_reduce_grad in tile order (deterministic).
// k_loss            mean squared error of log(sigma) over the reference
//                   patches (map read at the patch centre) and its gradient map.
// k_window_rows/cols  noise level of every reference patch for denoising:
//                   exp of the mean of the map over an S x S window around the
//                   patch centre, as row sums then column sums (fixed order).
// k_learned_partial/final  the map against the eigenvalue estimate: geometric
//                   mean of the ratio, and the decision to use it.
// k_adam            Adam with bias correction; refreshes the FP16 copy.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "cnn_internal.h"
#include "hts_internal.h"

namespace hts {
namespace {

constexpr int WID = 32, DEPTH = 5, TS = 16, NTH = 256, HALO = TS + 2;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

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

// out[co][y][x] = b[co] + sum_ci sum_ky,kx w[co][ci][ky][kx] in[ci][y+ky-1][x+kx-1] (zero outside)
template <int COUT>
__global__ void __launch_bounds__(NTH) k_conv_fwd(const float *__restrict__ in, int cin, int H, int W, float in_scale,
                                                  const __half *__restrict__ wt, const __half *__restrict__ bias,
                                                  float *__restrict__ out, int relu) {
    extern __shared__ float sm[];
    float *sIn = sm;                     // [cin][HALO][HALO]
    float *sW = sm + cin * HALO * HALO;  // [COUT][cin][9]
    const int tid = threadIdx.x;
    const int ntx = (W + TS - 1) / TS;
    const int y0 = (blockIdx.x / ntx) * TS, x0 = (blockIdx.x % ntx) * TS;
    const size_t HWs = (size_t)H * W;
    for (int e = tid; e < cin * HALO * HALO; e += NTH) {
        const int c = e / (HALO * HALO), r = e - c * HALO * HALO, a = r / HALO, b = r - a * HALO;
        const int y = y0 - 1 + a, x = x0 - 1 + b;
        sIn[e] = (y >= 0 && y < H && x >= 0 && x < W) ? in[c * HWs + (size_t)y * W + x] * in_scale : 0.f;
    }
    for (int e = tid; e < COUT * cin * 9; e += NTH) sW[e] = __half2float(wt[e]);
    __syncthreads();
    const int ty = tid / TS, tx = tid - ty * TS;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = __half2float(bias[co]);
    for (int c = 0; c < cin; ++c) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float xv = sIn[c * HALO * HALO + (ty + k / 3) * HALO + tx + k % 3];
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(sW[(co * cin + c) * 9 + k], xv, acc[co]);
        }
    }
    const int y = y0 + ty, x = x0 + tx;
    if (y < H && x < W) {
#pragma unroll
        for (int co = 0; co < COUT; ++co) out[co * HWs + (size_t)y * W + x] = relu ? fmaxf(acc[co], 0.f) : acc[co];
    }
}

// dx[ci][y][x] = sum_co sum_ky,kx w[co][ci][ky][kx] dy[co][y-ky+1][x-kx+1], then times (x_in > 0):
// the layer input is the previous layer's ReLU output.
template <int COUT>
__global__ void __launch_bounds__(NTH) k_conv_bwd_data(const float *__restrict__ dy, int H, int W,
                                                       const __half *__restrict__ wt, const float *__restrict__ xin,
                                                       float *__restrict__ dx) {
    constexpr int CIN = WID;
    extern __shared__ float sm[];
    float *sD = sm;                       // [COUT][HALO][HALO]
    float *sW = sm + COUT * HALO * HALO;  // [COUT][CIN][9]
    const int tid = threadIdx.x;
    const int ntx = (W + TS - 1) / TS;
    const int y0 = (blockIdx.x / ntx) * TS, x0 = (blockIdx.x % ntx) * TS;
    const size_t HWs = (size_t)H * W;
    for (int e = tid; e < COUT * HALO * HALO; e += NTH) {
        const int c = e / (HALO * HALO), r = e - c * HALO * HALO, a = r / HALO, b = r - a * HALO;
        const int y = y0 - 1 + a, x = x0 - 1 + b;
        sD[e] = (y >= 0 && y < H && x >= 0 && x < W) ? dy[c * HWs + (size_t)y * W + x] : 0.f;
    }
    for (int e = tid; e < COUT * CIN * 9; e += NTH) sW[e] = __half2float(wt[e]);
    __syncthreads();
    const int ty = tid / TS, tx = tid - ty * TS;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int co = 0; co < COUT; ++co) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int ky = k / 3, kx = k % 3;
            const float dv = sD[co * HALO * HALO + (ty + 2 - ky) * HALO + tx + 2 - kx];
#pragma unroll
            for (int c = 0; c < CIN; ++c) acc[c] = fmaf(sW[(co * CIN + c) * 9 + k], dv, acc[c]);
        }
    }
    const int y = y0 + ty, x = x0 + tx;
    if (y < H && x < W) {
        const size_t o = (size_t)y * W + x;
#pragma unroll
        for (int c = 0; c < CIN; ++c) dx[c * HWs + o] = xin[c * HWs + o] > 0.f ? acc[c] : 0.f;
    }
}

// Per tile: dw[co][ci][ky][kx] = sum over the tile's pixels of dy[co][p] x[ci][p + (ky-1, kx-1)],
// db[co] = sum of dy[co][p]; written to part[tile][.].
template <int COUT>
__global__ void __launch_bounds__(NTH) k_conv_bwd_weight(const float *__restrict__ x, int cin, int H, int W,
                                                         float in_scale, const float *__restrict__ dy,
                                                         float *__restrict__ part) {
    extern __shared__ float sm[];
    float *sX = sm;                      // [cin][HALO][HALO]
    float *sD = sm + cin * HALO * HALO;  // [COUT][TS][TS]
    const int tid = threadIdx.x;
    const int ntx = (W + TS - 1) / TS;
    const int y0 = (blockIdx.x / ntx) * TS, x0 = (blockIdx.x % ntx) * TS;
    const size_t HWs = (size_t)H * W;
    for (int e = tid; e < cin * HALO * HALO; e += NTH) {
        const int c = e / (HALO * HALO), r = e - c * HALO * HALO, a = r / HALO, b = r - a * HALO;
        const int y = y0 - 1 + a, xx = x0 - 1 + b;
        sX[e] = (y >= 0 && y < H && xx >= 0 && xx < W) ? x[c * HWs + (size_t)y * W + xx] * in_scale : 0.f;
    }
    for (int e = tid; e < COUT * TS * TS; e += NTH) {
        const int c = e / (TS * TS), r = e - c * TS * TS, a = r / TS, b = r - a * TS;
        const int y = y0 + a, xx = x0 + b;
        sD[e] = (y < H && xx < W) ? dy[c * HWs + (size_t)y * W + xx] : 0.f;
    }
    __syncthreads();
    const int nw = COUT * cin * 9, ne = nw + COUT;
    float *dst = part + (size_t)blockIdx.x * ne;
    for (int e = tid; e < ne; e += NTH) {
        float s = 0.f;
        if (e < nw) {
            const int co = e / (cin * 9), rem = e - co * cin * 9, c = rem / 9, k = rem - c * 9;
            const float *d = sD + co * TS * TS;
            const float *xs = sX + c * HALO * HALO + (k / 3) * HALO + k % 3;
            for (int i = 0; i < TS; ++i)
#pragma unroll
                for (int j = 0; j < TS; ++j) s = fmaf(d[i * TS + j], xs[i * HALO + j], s);
        } else {
            const float *d = sD + (e - nw) * TS * TS;
            for (int i = 0; i < TS * TS; ++i) s += d[i];
        }
        dst[e] = s;
    }
}

// grad[e] += sum over tiles, in tile order.
__global__ void k_reduce_grad(const float *__restrict__ part, int ntiles, int ne, float *__restrict__ grad) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * ne + e];
        grad[e] += s;
    }
}

// Loss over the reference patches (one block): mean of (out[centre] - target)^2 added to *loss;
// dout[centre] = 2 (out - target) / N_ref (dout zeroed before).
__global__ void __launch_bounds__(1024) k_loss(const float *__restrict__ outm, int H, int W, int step, int nx,
                                               int nref, const float *__restrict__ target, float *__restrict__ dout,
                                               double *loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (int r = threadIdx.x; r < nref; r += blockDim.x) {
        const int gy = r / nx, gx = r - gy * nx;
        const size_t o = (size_t)(grid_pos(gy, H, step) + PS / 2) * W + grid_pos(gx, W, step) + PS / 2;
        const float d = outm[o] - target[r];
        dout[o] = 2.f * d / (float)nref;
        s += (double)d * d;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *loss += t / nref;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __half *__restrict__ w16, int n, float lr, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = ADAM_B1 * m[i] + (1.f - ADAM_B1) * gi;
        const float vi = ADAM_B2 * v[i] + (1.f - ADAM_B2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + ADAM_EPS);
        p[i] = pi;
        w16[i] = __float2half_rn(pi);
    }
}

__global__ void k_to_half(const float *__restrict__ p, __half *__restrict__ w16, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w16[i] = __float2half_rn(p[i]);
}

// Window of a reference patch along one axis: [c - S/2, c - S/2 + S) cut to [0, n), c = centre.
__host__ __device__ __forceinline__ void window_span(int c, int S, int n, int &lo, int &hi) {
    lo = c - S / 2;
    hi = lo + S;
    lo = lo < 0 ? 0 : lo;
    hi = hi > n ? n : hi;
}

// rows[y][gx] = sum of map[y][x] over the window columns of reference column gx.
__global__ void k_window_rows(const float *__restrict__ outm, int H, int W, int step, int nx, int S,
                              float *__restrict__ rows) {
    const size_t n = (size_t)H * nx;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(e / nx), gx = (int)(e - (size_t)y * nx);
        int lo, hi;
        window_span(grid_pos(gx, W, step) + PS / 2, S, W, lo, hi);
        const float *row = outm + (size_t)y * W;
        // four partial sums over 16-byte loads (the windows of grid columns start on multiples of 4 pixels)
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int x = lo;
        for (; x < hi && (reinterpret_cast<uintptr_t>(row + x) & 15) != 0; ++x) a0 += row[x];
        for (; x + 4 <= hi; x += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(row + x));
            a0 += v.x;
            a1 += v.y;
            a2 += v.z;
            a3 += v.w;
        }
        for (; x < hi; ++x) a0 += row[x];
        rows[e] = (a0 + a1) + (a2 + a3);
    }
}

// sigma_ref[r] = exp(sum of rows[y][gx] over the window rows of r / window area).
__global__ void k_window_cols(const float *__restrict__ rows, int H, int W, int step, int nx, int nref, int S,
                              float *__restrict__ sigma_ref) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nref; r += gridDim.x * blockDim.x) {
        const int gy = r / nx, gx = r - gy * nx;
        int ylo, yhi, xlo, xhi;
        window_span(grid_pos(gy, H, step) + PS / 2, S, H, ylo, yhi);
        window_span(grid_pos(gx, W, step) + PS / 2, S, W, xlo, xhi);
        float acc = 0.f;
        for (int y = ylo; y < yhi; ++y) acc += rows[(size_t)y * nx + gx];
        sigma_ref[r] = expf(acc / (float)((yhi - ylo) * (xhi - xlo)));
    }
}

// Per block: sum of log(sigma_ref) over a fixed stride of references (NaN if one is not finite and > 0).
__global__ void __launch_bounds__(256) k_learned_partial(const float *__restrict__ sigma_ref, int nref,
                                                         DevState *st) {
    __shared__ double red[8];
    double s = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nref; r += gridDim.x * blockDim.x) {
        const float v = sigma_ref[r];
        s += (v > 0.f && isfinite(v)) ? (double)logf(v) : (double)NAN;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        st->learned_part[blockIdx.x] = t;
    }
}

// Geometric-mean ratio of the map to the estimate; the map is used if it lies in [1/factor, factor].
__global__ void k_learned_final(int nref, double factor, DevState *st) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < LEARNED_PARTS; ++b) t += st->learned_part[b];
    const double est = st->sigma_hat;
    const double ratio = (est > 0.0 && isfinite(t)) ? exp(t / nref - log(est)) : 0.0;
    st->learned_ratio = ratio;
    st->learned = (ratio > 0.0 && ratio >= 1.0 / factor && ratio <= factor) ? 1 : 0;
}

}  // namespace

// The training loss over the reference patches and its gradient map (dout: H x W, zeroed here), for the
// tensor-core training path (cnn_tc.cu).
hts_status cnn_loss(const float *map, int H, int W, const Geom &g, const float *target, float *dout, double *loss,
                    cudaStream_t s) {
    HTS_TRY(cu(cudaMemsetAsync(dout, 0, (size_t)H * W * sizeof(float), s), "cudaMemsetAsync"));
    {
        KTimer kt("k_loss", s);
        k_loss<<<1, 1024, 0, s>>>(map, H, W, g.step, g.nx, g.nref, target, dout, loss);
    }
    return check_launch("k_loss");
}

namespace {

size_t fwd_smem(int cin, int cout) { return ((size_t)cin * HALO * HALO + (size_t)cout * cin * 9) * 4; }

uint64_t splitmix64(uint64_t &x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

double unit_uniform(uint64_t &x) { return ((splitmix64(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

hts_status ensure_ws(hts_cnn *n, int H, int W) {
    const size_t px = (size_t)H * W;
    if (px > n->cap_px) {
        for (int l = 0; l < DEPTH; ++l) {
            cudaFree(n->act[l]);
            n->act[l] = nullptr;
        }
        cudaFree(n->d0);
        cudaFree(n->d1);
        n->d0 = n->d1 = nullptr;
        n->cap_px = 0;
        for (int l = 0; l < DEPTH; ++l)
            HTS_TRY(cu(dev_malloc(&n->act[l], px * (l < DEPTH - 1 ? WID : 1) * sizeof(float)), "cudaMalloc(cnn)"));
        HTS_TRY(cu(dev_malloc(&n->d0, px * WID * sizeof(float)), "cudaMalloc(cnn)"));
        HTS_TRY(cu(dev_malloc(&n->d1, px * WID * sizeof(float)), "cudaMalloc(cnn)"));
        n->cap_px = px;
    }
    const size_t ntiles = ((size_t)(H + TS - 1) / TS) * ((W + TS - 1) / TS);
    const size_t need = ntiles * (WID * WID * 9 + WID);
    if (need > n->cap_part) {
        cudaFree(n->part);
        n->part = nullptr;
        n->cap_part = 0;
        HTS_TRY(cu(dev_malloc(&n->part, need * sizeof(float)), "cudaMalloc(cnn)"));
        n->cap_part = need;
    }
    return HTS_OK;
}

template <int COUT>
hts_status fwd_layer(const hts_cnn *n, int l, const float *in, float scale, int H, int W, float *out, int relu,
                     cudaStream_t s) {
    const size_t sm = fwd_smem(n->cin[l], COUT);
    HTS_TRY(allow_smem(reinterpret_cast<const void *>(k_conv_fwd<COUT>), sm));
    const int nt = ((H + TS - 1) / TS) * ((W + TS - 1) / TS);
    {
        KTimer kt("k_conv_fwd", s);
        k_conv_fwd<COUT><<<nt, NTH, sm, s>>>(in, n->cin[l], H, W, scale, n->w16 + n->off[l],
                                             n->w16 + n->off[l] + COUT * n->cin[l] * 9, out, relu);
    }
    return check_launch("k_conv_fwd");
}

hts_status forward(const hts_cnn *n, const float *img, int H, int W, cudaStream_t s) {
    HTS_TRY(fwd_layer<WID>(n, 0, img, 1.f / 255.f, H, W, n->act[0], 1, s));
    for (int l = 1; l < DEPTH - 1; ++l) HTS_TRY(fwd_layer<WID>(n, l, n->act[l - 1], 1.f, H, W, n->act[l], 1, s));
    return fwd_layer<1>(n, DEPTH - 1, n->act[DEPTH - 2], 1.f, H, W, n->act[DEPTH - 1], 0, s);
}

template <int COUT>
hts_status bwd_weight(hts_cnn *n, int l, const float *x, float scale, const float *dy, int H, int W, cudaStream_t s) {
    const int cin = n->cin[l];
    const size_t sm = ((size_t)cin * HALO * HALO + (size_t)COUT * TS * TS) * 4;
    HTS_TRY(allow_smem(reinterpret_cast<const void *>(k_conv_bwd_weight<COUT>), sm));
    const int nt = ((H + TS - 1) / TS) * ((W + TS - 1) / TS);
    const int ne = COUT * cin * 9 + COUT;
    {
        KTimer kt("k_conv_bwd_weight", s);
        k_conv_bwd_weight<COUT><<<nt, NTH, sm, s>>>(x, cin, H, W, scale, dy, n->part);
    }
    HTS_TRY(check_launch("k_conv_bwd_weight"));
    {
        KTimer kt("k_reduce_grad", s);
        k_reduce_grad<<<(ne + 255) / 256, 256, 0, s>>>(n->part, nt, ne, n->grad + n->off[l]);
    }
    return check_launch("k_reduce_grad");
}

template <int COUT>
hts_status bwd_data(const hts_cnn *n, int l, const float *dy, const float *xin, float *dx, int H, int W,
                    cudaStream_t s) {
    const size_t sm = ((size_t)COUT * HALO * HALO + (size_t)COUT * WID * 9) * 4;
    HTS_TRY(allow_smem(reinterpret_cast<const void *>(k_conv_bwd_data<COUT>), sm));
    const int nt = ((H + TS - 1) / TS) * ((W + TS - 1) / TS);
    {
        KTimer kt("k_conv_bwd_data", s);
        k_conv_bwd_data<COUT><<<nt, NTH, sm, s>>>(dy, H, W, n->w16 + n->off[l], xin, dx);
    }
    return check_launch("k_conv_bwd_data");
}

hts_status check_net(const hts_cnn *n, const float *img, int H, int W) {
    if (!n || !img) return report(HTS_EINVAL, "NULL pointer");
    if (H < PS || W < PS) return report(HTS_EINVAL, "image smaller than a patch");
    int dev = 0;
    HTS_TRY(cu(cudaGetDevice(&dev), "cudaGetDevice"));
    if (dev != n->device) return report(HTS_EINVAL, "network lives on another device");
    return HTS_OK;
}

void layout(hts_cnn *n) {
    int o = 0;
    for (int l = 0; l < DEPTH; ++l) {
        n->cin[l] = l == 0 ? n->C : WID;
        n->cout[l] = l == DEPTH - 1 ? 1 : WID;
        n->off[l] = o;
        o += n->cout[l] * n->cin[l] * 9 + n->cout[l];
    }
    n->nparams = o;
}

hts_status upload(hts_cnn *n, const float *host) {
    HTS_TRY(cu(cudaMemcpy(n->master, host, n->nparams * sizeof(float), cudaMemcpyHostToDevice), "cudaMemcpy"));
    HTS_TRY(cu(cudaMemset(n->m, 0, n->nparams * sizeof(float)), "cudaMemset"));
    HTS_TRY(cu(cudaMemset(n->v, 0, n->nparams * sizeof(float)), "cudaMemset"));
    HTS_TRY(cu(cudaMemset(n->grad, 0, n->nparams * sizeof(float)), "cudaMemset"));
    n->t = 0;
    k_to_half<<<(n->nparams + 255) / 256, 256>>>(n->master, n->w16, n->nparams);
    count_launch();
    HTS_TRY(check_launch("k_to_half"));
    return cu(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
}

void free_net(hts_cnn *n) {
    if (!n) return;
    cudaFree(n->master);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->w16);
    for (int l = 0; l < DEPTH; ++l) cudaFree(n->act[l]);
    cudaFree(n->d0);
    cudaFree(n->d1);
    cudaFree(n->part);
    cudaFree(n->loss);
    cudaFree(n->h16[0]);
    cudaFree(n->h16[1]);
    cudaFree(n->map);
    cudaFree(n->rows);
    cudaFree(n->err);
    for (int i = 0; i < 4; ++i) cudaFree(n->tr_act[i]);
    for (int i = 0; i < 2; ++i) cudaFree(n->tr_dy[i]);
    cudaFree(n->tr_wt);
    cudaFree(n->tr_map);
    cudaFree(n->tr_d0);
    cudaFree(n->tr_part);
    delete n;
}

}  // namespace

hts_status launch_learned_check(const float *sigma_ref, int nref, double factor, DevState *st, cudaStream_t s) {
    {
        KTimer kt("k_learned_partial", s);
        k_learned_partial<<<LEARNED_PARTS, 256, 0, s>>>(sigma_ref, nref, st);
    }
    HTS_TRY(check_launch("k_learned_partial"));
    {
        KTimer kt("k_learned_final", s);
        k_learned_final<<<1, 32, 0, s>>>(nref, factor, st);
    }
    return check_launch("k_learned_final");
}

// Noise level of every reference patch from the network through the readout window (device, N_ref).
hts_status cnn_sigma_refs(hts_cnn *n, const float *img, const Geom &g, float *sigma_ref, cudaStream_t s) {
    HTS_TRY(check_net(n, img, g.H, g.W));
    if (n->C != g.C) return report(HTS_EINVAL, "network built for another channel count");
    HTS_TRY(cnn_ensure_infer(n, g.H, g.W, g.nx));
    return cnn_sigma_refs_into(n, img, g, n->h16[0], n->h16[1], n->map, n->rows, sigma_ref, s);
}

hts_status cnn_sigma_refs_into(hts_cnn *n, const float *img, const Geom &g, __half *h0, __half *h1, float *map,
                               float *rows, float *sigma_ref, cudaStream_t s) {
    if (n->C != g.C) return report(HTS_EINVAL, "network built for another channel count");
    HTS_TRY(cnn_forward_tc_into(n, img, g.H, g.W, h0, h1, map, s));
    const size_t nrow = (size_t)g.H * g.nx;  // rows: H x nx row sums
    {
        KTimer kt("k_window_rows", s);
        k_window_rows<<<(unsigned)std::min<size_t>((nrow + 255) / 256, 152 * 16), 256, 0, s>>>(
            map, g.H, g.W, g.step, g.nx, n->window, rows);
    }
    HTS_TRY(check_launch("k_window_rows"));
    {
        KTimer kt("k_window_cols", s);
        k_window_cols<<<(g.nref + 255) / 256, 256, 0, s>>>(rows, g.H, g.W, g.step, g.nx, g.nref, n->window,
                                                           sigma_ref);
    }
    return check_launch("k_window_cols");
}

}  // namespace hts

using namespace hts;

extern "C" int hts_cnn_num_params(int C) {
    if (C != 1 && C != 3) return 0;
    hts_cnn n;
    n.C = C;
    layout(&n);
    return n.nparams;
}

extern "C" int hts_cnn_channels(const hts_cnn *net) { return net ? net->C : 0; }

extern "C" int hts_cnn_window(const hts_cnn *net) { return net ? net->window : 0; }

extern "C" hts_status hts_cnn_set_window(hts_cnn *net, int S) {
    if (!net) return report(HTS_EINVAL, "NULL pointer");
    if (S < 1 || S > 4096) return report(HTS_EINVAL, "window must be in [1, 4096]");
    net->window = S;
    return HTS_OK;
}

extern "C" hts_status hts_cnn_create(int C, uint64_t seed, hts_cnn **out) {
    if (!out) return report(HTS_EINVAL, "NULL pointer");
    if (C != 1 && C != 3) return report(HTS_EINVAL, "C must be 1 or 3");
    hts_cnn *n = new hts_cnn();
    n->C = C;
    layout(n);
    hts_status st = cu(cudaGetDevice(&n->device), "cudaGetDevice");
    const size_t b = n->nparams * sizeof(float);
    for (float **p : {&n->master, &n->grad, &n->m, &n->v})
        if (st == HTS_OK) st = cu(dev_malloc(p, b), "cudaMalloc(cnn)");
    if (st == HTS_OK) st = cu(dev_malloc(&n->w16, n->nparams * sizeof(__half)), "cudaMalloc(cnn)");
    if (st == HTS_OK) st = cu(dev_malloc(&n->loss, sizeof(double)), "cudaMalloc(cnn)");
    if (st == HTS_OK) st = cu(cudaMemset(n->loss, 0, sizeof(double)), "cudaMemset");
    if (st == HTS_OK) st = cu(dev_malloc(&n->err, sizeof(int)), "cudaMalloc(cnn)");
    if (st == HTS_OK) st = cu(cudaMemset(n->err, 0, sizeof(int)), "cudaMemset");
    if (st != HTS_OK) {
        free_net(n);
        return st;
    }
    // He initialisation N(0, 2 / fan_in) (Box-Muller on a splitmix64 stream); the output layer
    // starts small with bias log(10), i.e. sigma = 10 everywhere
    std::vector<float> h(n->nparams, 0.f);
    uint64_t x = seed;
    for (int l = 0; l < DEPTH; ++l) {
        const int nw = n->cout[l] * n->cin[l] * 9;
        const double sd = std::sqrt(2.0 / (n->cin[l] * 9)) * (l == DEPTH - 1 ? 0.1 : 1.0);
        for (int i = 0; i < nw; ++i) {
            const double u1 = unit_uniform(x), u2 = unit_uniform(x);
            h[n->off[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
        for (int i = 0; i < n->cout[l]; ++i) h[n->off[l] + nw + i] = l == DEPTH - 1 ? (float)std::log(10.0) : 0.f;
    }
    st = upload(n, h.data());
    if (st != HTS_OK) {
        free_net(n);
        return st;
    }
    *out = n;
    return HTS_OK;
}

extern "C" hts_status hts_cnn_free(hts_cnn *net) {
    if (net) batch_drop_net(net);
    free_net(net);
    return HTS_OK;
}

extern "C" hts_status hts_cnn_get_params(const hts_cnn *net, float *host_params) {
    if (!net || !host_params) return report(HTS_EINVAL, "NULL pointer");
    return cu(cudaMemcpy(host_params, net->master, net->nparams * sizeof(float), cudaMemcpyDeviceToHost),
              "cudaMemcpy");
}

extern "C" hts_status hts_cnn_set_params(hts_cnn *net, const float *host_params) {
    if (!net || !host_params) return report(HTS_EINVAL, "NULL pointer");
    return upload(net, host_params);
}

extern "C" hts_status hts_cnn_log_sigma_map(hts_cnn *net, const float *img, int H, int W, float *map_out,
                                           void *stream) {
    HTS_TRY(check_net(net, img, H, W));
    if (!map_out) return report(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(cnn_ensure_infer(net, H, W, 1));
    HTS_TRY(cnn_forward_tc(net, img, H, W, s));
    return cu(cudaMemcpyAsync(map_out, net->map, (size_t)H * W * sizeof(float), cudaMemcpyDeviceToDevice, s),
              "cudaMemcpyAsync");
}

extern "C" hts_status hts_cnn_sigma_refs(hts_cnn *net, const float *img, int H, int W, const hts_params *p,
                                        float *sigma_ref, void *stream) {
    HTS_TRY(check_net(net, img, H, W));
    if (!sigma_ref) return report(HTS_EINVAL, "NULL pointer");
    Geom g;
    HTS_TRY(validate(H, W, net->C, p, &g));
    return cnn_sigma_refs(net, img, g, sigma_ref, static_cast<cudaStream_t>(stream));
}

extern "C" hts_status hts_cnn_set_train_fp16(hts_cnn *net, int on) {
    if (!net) return report(HTS_EINVAL, "NULL pointer");
    net->train_tc = on ? 1 : 0;
    return HTS_OK;
}

extern "C" int hts_cnn_train_fp16(const hts_cnn *net) { return net ? net->train_tc : -1; }

extern "C" hts_status hts_cnn_zero_grad(hts_cnn *net, void *stream) {
    if (!net) return report(HTS_EINVAL, "NULL pointer");
    return cu(cudaMemsetAsync(net->grad, 0, net->nparams * sizeof(float), static_cast<cudaStream_t>(stream)),
              "cudaMemsetAsync");
}

extern "C" hts_status hts_cnn_accumulate_grad(hts_cnn *net, const float *img, int H, int W, const hts_params *p,
                                             const float *target_log_sigma, void *stream) {
    HTS_TRY(check_net(net, img, H, W));
    if (!target_log_sigma) return report(HTS_EINVAL, "NULL pointer");
    Geom g;
    HTS_TRY(validate(H, W, net->C, p, &g));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (net->train_tc) return cnn_grad_tc(net, img, H, W, g, target_log_sigma, s);
    HTS_TRY(ensure_ws(net, H, W));
    HTS_TRY(forward(net, img, H, W, s));
    const size_t px = (size_t)H * W;
    // loss and its gradient map (in d0)
    HTS_TRY(cu(cudaMemsetAsync(net->d0, 0, px * sizeof(float), s), "cudaMemsetAsync"));
    {
        KTimer kt("k_loss", s);
        k_loss<<<1, 1024, 0, s>>>(net->act[DEPTH - 1], H, W, g.step, g.nx, g.nref, target_log_sigma, net->d0,
                                  net->loss);
    }
    HTS_TRY(check_launch("k_loss"));
    // layer 4 (linear) back to layer 0; each bwd_data output is masked by the ReLU of its layer
    float *dcur = net->d0, *dnext = net->d1;
    HTS_TRY(bwd_weight<1>(net, DEPTH - 1, net->act[DEPTH - 2], 1.f, dcur, H, W, s));
    HTS_TRY(bwd_data<1>(net, DEPTH - 1, dcur, net->act[DEPTH - 2], dnext, H, W, s));
    for (int l = DEPTH - 2; l >= 1; --l) {
        std::swap(dcur, dnext);
        HTS_TRY(bwd_weight<WID>(net, l, net->act[l - 1], 1.f, dcur, H, W, s));
        HTS_TRY(bwd_data<WID>(net, l, dcur, net->act[l - 1], dnext, H, W, s));
    }
    std::swap(dcur, dnext);
    return bwd_weight<WID>(net, 0, img, 1.f / 255.f, dcur, H, W, s);
}

extern "C" hts_status hts_cnn_take_loss(hts_cnn *net, double *loss_sum, void *stream) {
    if (!net || !loss_sum) return report(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(cu(cudaMemcpyAsync(loss_sum, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync"));
    HTS_TRY(cu(cudaMemsetAsync(net->loss, 0, sizeof(double), s), "cudaMemsetAsync"));
    return cu(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

extern "C" hts_status hts_cnn_get_grad(const hts_cnn *net, float *host_grad, void *stream) {
    if (!net || !host_grad) return report(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HTS_TRY(cu(cudaMemcpyAsync(host_grad, net->grad, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, s),
               "cudaMemcpyAsync"));
    return cu(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

extern "C" hts_status hts_cnn_adam_step(hts_cnn *net, float lr, void *stream) {
    if (!net) return report(HTS_EINVAL, "NULL pointer");
    if (!(lr > 0.f) || !std::isfinite(lr)) return report(HTS_EINVAL, "lr must be > 0");
    net->t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B1, net->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)ADAM_B2, net->t)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        KTimer kt("k_adam", s);
        k_adam<<<(net->nparams + 255) / 256, 256, 0, s>>>(net->master, net->grad, net->m, net->v, net->w16,
                                                          net->nparams, lr, c1, c2);
    }
    return check_launch("k_adam");
}

extern "C" hts_status hts_cnn_save(const hts_cnn *net, const char *path) {
    if (!net || !path) return report(HTS_EINVAL, "NULL pointer");
    std::vector<float> h(net->nparams);
    HTS_TRY(hts_cnn_get_params(net, h.data()));
    FILE *f = fopen(path, "wb");
    if (!f) return report(HTS_EINVAL, "cannot open file");
    const char magic[8] = {'H', 'T', 'S', 'C', 'N', 'N', '2', 0};
    const int hdr[3] = {net->C, net->nparams, net->window};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 3, f) == 3 &&
              fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    return ok ? HTS_OK : report(HTS_EINVAL, "write failed");
}

extern "C" hts_status hts_cnn_load(const char *path, hts_cnn **out) {
    if (!path || !out) return report(HTS_EINVAL, "NULL pointer");
    FILE *f = fopen(path, "rb");
    if (!f) return report(HTS_EINVAL, "cannot open file");
    char magic[8];
    int hdr[3];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "HTSCNN2", 8) == 0 && fread(hdr, sizeof(int), 3, f) == 3 &&
              (hdr[0] == 1 || hdr[0] == 3) && hdr[1] == hts_cnn_num_params(hdr[0]) && hdr[2] >= 1 && hdr[2] <= 4096;
    std::vector<float> h(ok ? hdr[1] : 0);
    if (ok) ok = fread(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    if (!ok) return report(HTS_EINVAL, "not a network file");
    hts_cnn *n = nullptr;
    HTS_TRY(hts_cnn_create(hdr[0], 1, &n));
    n->window = hdr[2];
    const hts_status st = upload(n, h.data());
    if (st != HTS_OK) {
        free_net(n);
        return st;
    }
    *out = n;
    return HTS_OK;
}
