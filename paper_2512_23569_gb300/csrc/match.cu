// Grouping step of Haar-tSVD (Eq. 9, Alg. 1 step 1) on sm_103a.
//
// One warp per reference patch.  The warp stages its search region of the
// matching plane (gray image, green channel, or the channel sum R+G+B when
// Eq. 9 rejects green) in shared memory, computes FP32 squared distances of
// all candidates (each lane 4 horizontally adjacent candidates per item,
// register-blocked), keeps a per-lane sorted top-(K+3) list of 64-bit keys
// (distance bits, raster index) and merges the 32 lists.
//
// Exactness.  The group must equal the FP64 definition bit for bit: the K-1
// nearest candidates in ascending (distance, raster index), distances being
// the FP64 row-major sum of squared differences.  The FP32 distance d of a
// candidate whose FP64 distance is D obeys |d - D| <= eps D + beta sqrt(D) + g0
// (eps covers 66 roundings of the subtract / FMA chain; beta and g0 cover the
// rounding of the FP32 channel sum on the R+G+B plane, scaled by the largest
// |R|+|G|+|B| of the region; g0 also absorbs subnormal flushing).  If every
// adjacent pair among the first K FP32 entries is separated by that bound,
// the FP32 order is the FP64 order and nothing else runs.  Otherwise every
// entry that can still belong to the K-1 nearest is re-evaluated with the
// FP64 expression in the same operation order as the definition and ranked
// by (D, index); when even the list of K+3 cannot certify that it holds all
// of them, the reference goes to an exhaustive FP64 pass (flat, noiseless
// inputs with massive ties end up there).
#include "hts_internal.h"

namespace hts {
namespace {

constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24
constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t EMPTY = ~0ull;

struct MatchArgs {
    const float *img;
    int H, W, C, step, R, nx, nref;
    double gamma;
    int32_t *idx;
    uint8_t *green;
    int32_t *fb;
    DevState *st;
};

__device__ __forceinline__ uint64_t make_key(float d, int idx) {
    return ((uint64_t)__float_as_uint(d) << 32) | (uint32_t)idx;
}
__device__ __forceinline__ float key_dist(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int key_idx(uint64_t k) { return (int)(uint32_t)(k & 0xffffffffu); }

template <int M>
__device__ __forceinline__ void topm_insert(uint64_t (&lst)[M], uint64_t key) {
    if (key >= lst[M - 1]) return;
#pragma unroll
    for (int i = M - 1; i > 0; --i) {
        const uint64_t prev = lst[i - 1], cur = lst[i];
        lst[i] = prev > key ? prev : (cur < key ? cur : key);
    }
    lst[0] = lst[0] < key ? lst[0] : key;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(FULL, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Value of the matching plane in FP64, in the definition's operation order.
__device__ __forceinline__ double plane64(const float *__restrict__ img, size_t HW, int C, int green, size_t o) {
    if (C == 1) return (double)__ldg(img + o);
    if (green) return (double)__ldg(img + HW + o);
    return __dadd_rn(__dadd_rn((double)__ldg(img + o), (double)__ldg(img + HW + o)), (double)__ldg(img + 2 * HW + o));
}

// FP64 squared distance, row-major, no contraction (same order as the definition).
__device__ double exact_dist(const float *__restrict__ img, int W, size_t HW, int C, int green, int yr, int xr,
                             int yc, int xc) {
    double acc = 0.0;
    for (int u = 0; u < PS; ++u)
        for (int v = 0; v < PS; ++v) {
            const double a = plane64(img, HW, C, green, (size_t)(yr + u) * W + xr + v);
            const double b = plane64(img, HW, C, green, (size_t)(yc + u) * W + xc + v);
            const double d = __dsub_rn(a, b);
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        }
    return acc;
}

// Eq. 9 on the reference patch in FP64 (sequential row-major sums, as the
// definition).  Lanes 0..2 each sum one channel; all lanes get the flag.
__device__ int gcp_green(const float *__restrict__ img, int W, size_t HW, int y, int x, double gamma, int lane) {
    double n2 = 0.0;
    if (lane < 3) {
        const float *ch = img + (size_t)lane * HW;
        for (int u = 0; u < PS; ++u)
            for (int v = 0; v < PS; ++v) {
                const double a = (double)__ldg(ch + (size_t)(y + u) * W + x + v);
                n2 = __dadd_rn(n2, __dmul_rn(a, a));
            }
    }
    const double r2 = __shfl_sync(FULL, n2, 0), g2 = __shfl_sync(FULL, n2, 1), b2 = __shfl_sync(FULL, n2, 2);
    const double nR = __dsqrt_rn(r2), nG = __dsqrt_rn(g2), nB = __dsqrt_rn(b2);
    const double lim = fmax(__ddiv_rn(nR, gamma), __ddiv_rn(nB, gamma));
    return nG >= lim ? 1 : 0;
}

// Certified interval of the FP64 distance given the FP32 one.
struct Bound {
    float eps, beta, g0;
    __device__ __forceinline__ float upper(float d) const {
        if (beta == 0.f) return __fdiv_rn(d + g0, 1.f - eps) * (1.f + 4.f * U32);
        const float a = 1.f - eps;
        const float s = (beta + sqrtf(beta * beta + 4.f * a * (g0 + d))) / (2.f * a);
        return s * s * (1.f + 8.f * U32);
    }
    __device__ __forceinline__ float lower(float d) const {
        if (d <= g0) return 0.f;
        if (beta == 0.f) return __fdiv_rn(d - g0, 1.f + eps) * (1.f - 4.f * U32);
        const float a = 1.f + eps;
        const float s = (-beta + sqrtf(beta * beta + 4.f * a * (d - g0))) / (2.f * a);
        return s * s * (1.f - 8.f * U32);
    }
};

template <int K>
__global__ void __launch_bounds__(128) k_match(MatchArgs a) {
    constexpr int M = K + 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RW = 2 * a.R + PS;
    uint64_t *mer = reinterpret_cast<uint64_t *>(smem_raw) + warp * M;
    double *dex = reinterpret_cast<double *>(smem_raw) + nwarps * M + warp * M;
    float *reg = reinterpret_cast<float *>(smem_raw + (size_t)nwarps * M * 16) + warp * RW * RW;

    const int r = blockIdx.x * nwarps + warp;
    if (r >= a.nref) return;  // warp-uniform
    const size_t HW = (size_t)a.H * a.W;
    const int yr = grid_pos(r / a.nx, a.H, a.step), xr = grid_pos(r % a.nx, a.W, a.step);
    const int green = (a.C == 3) ? gcp_green(a.img, a.W, HW, yr, xr, a.gamma, lane) : 1;
    if (lane == 0 && a.green) a.green[r] = (uint8_t)green;

    const int cy0 = max(0, yr - a.R), cy1 = min(a.H - PS, yr + a.R);
    const int cx0 = max(0, xr - a.R), cx1 = min(a.W - PS, xr + a.R);
    const int nrow = cy1 - cy0 + 1, ncol = cx1 - cx0 + 1;
    const int rh = nrow + PS - 1, rw = ncol + PS - 1;
    const bool exact_plane = (a.C == 1) || green;

    float tmax = 0.f;
    for (int e = lane; e < rh * rw; e += 32) {
        const int yy = e / rw, xx = e - yy * rw;
        const size_t o = (size_t)(cy0 + yy) * a.W + (cx0 + xx);
        float v;
        if (a.C == 1) {
            v = __ldg(a.img + o);
        } else if (green) {
            v = __ldg(a.img + HW + o);
        } else {
            const float R = __ldg(a.img + o), G = __ldg(a.img + HW + o), B = __ldg(a.img + 2 * HW + o);
            v = __fadd_rn(__fadd_rn(R, G), B);
            tmax = fmaxf(tmax, fabsf(R) + fabsf(G) + fabsf(B));
        }
        reg[e] = v;
    }
    tmax = warp_max_f(tmax);
    __syncwarp();

    float ar[NPIX];
    {
        const float *rp = reg + (yr - cy0) * rw + (xr - cx0);
#pragma unroll
        for (int u = 0; u < PS; ++u)
#pragma unroll
            for (int v = 0; v < PS; ++v) ar[u * PS + v] = rp[u * rw + v];
    }

    uint64_t lst[M];
#pragma unroll
    for (int i = 0; i < M; ++i) lst[i] = EMPTY;

    const int nq = (ncol + 3) >> 2;
    const int nitems = nrow * nq;
    for (int it = lane; it < nitems; it += 32) {
        const int i = it / nq, cxb = (it - i * nq) * 4;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const float *row = reg + (i + u) * rw + cxb;
            float b[PS + 3];
#pragma unroll
            for (int t = 0; t < PS + 3; ++t) b[t] = (cxb + t < rw) ? row[t] : 0.f;
#pragma unroll
            for (int v = 0; v < PS; ++v) {
                const float av = ar[u * PS + v];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float e = __fsub_rn(av, b[v + t]);
                    d[t] = __fmaf_rn(e, e, d[t]);
                }
            }
        }
        const int gy = cy0 + i;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int cx = cxb + t;
            if (cx < ncol) {
                const int gx = cx0 + cx;
                if (gy != yr || gx != xr) topm_insert<M>(lst, make_key(d[t], gy * a.W + gx));
            }
        }
    }

    // merge the 32 sorted lists: M rounds of warp-wide minimum
    for (int j = 0; j < M; ++j) {
        const uint64_t h = lst[0];
        const uint64_t mn = warp_min_u64(h);
        if (lane == 0) mer[j] = mn;
        if (h == mn && mn != EMPTY) {
#pragma unroll
            for (int q = 0; q < M - 1; ++q) lst[q] = lst[q + 1];
            lst[M - 1] = EMPTY;
        }
    }
    __syncwarp();

    Bound bd;
    bd.eps = 100.f * U32;
    bd.beta = exact_plane ? 0.f : 72.f * U32 * tmax;
    bd.g0 = (exact_plane ? 0.f : 1200.f * U32 * U32 * tmax * tmax) + 1e-30f;

    int32_t *out = a.idx + (size_t)r * K;
    bool ok = true;
    for (int i = lane; i < K - 1; i += 32) {
        const uint64_t nx = mer[i + 1];
        if (nx != EMPTY) ok = ok && (bd.upper(key_dist(mer[i])) < bd.lower(key_dist(nx)));
    }
    const bool certified = __all_sync(FULL, ok);
    if (lane == 0) out[0] = yr * a.W + xr;
    if (certified) {
        for (int i = lane; i < K - 1; i += 32) out[1 + i] = key_idx(mer[i]);
        return;
    }
    // uncertain: FP64 re-rank of every entry that may belong to the K-1 nearest
    const float thr = bd.upper(key_dist(mer[K - 2]));
    const uint64_t last = mer[M - 1];
    if (last != EMPTY && bd.lower(key_dist(last)) <= thr) {
        if (lane == 0) {
            const int pos = atomicAdd(&a.st->match_fallback, 1);
            a.fb[pos] = r;
        }
        return;
    }
    int m = 0;
    for (int i = 0; i < M; ++i) {
        const uint64_t k = mer[i];
        if (k == EMPTY || bd.lower(key_dist(k)) > thr) break;
        m = i + 1;
    }
    for (int i = lane; i < m; i += 32) {
        const int id = key_idx(mer[i]);
        dex[i] = exact_dist(a.img, a.W, HW, a.C, green, yr, xr, id / a.W, id % a.W);
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
        const double di = dex[i];
        const int ii = key_idx(mer[i]);
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double dj = dex[j];
            const int ij = key_idx(mer[j]);
            rank += (dj < di || (dj == di && ij < ii)) ? 1 : 0;
        }
        if (rank < K - 1) out[1 + rank] = ii;
    }
    if (lane == 0) atomicAdd(&a.st->match_reranked, 1);
}

// Exhaustive FP64 matching of the references listed by k_match.
template <int K>
__global__ void __launch_bounds__(128) k_match_fallback(MatchArgs a) {
    constexpr int L = K - 1;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int count = *(volatile int *)&a.st->match_fallback;
    const size_t HW = (size_t)a.H * a.W;
    for (int f = gw; f < count; f += nw) {
        const int r = a.fb[f];
        const int yr = grid_pos(r / a.nx, a.H, a.step), xr = grid_pos(r % a.nx, a.W, a.step);
        const int green = (a.C == 3) ? gcp_green(a.img, a.W, HW, yr, xr, a.gamma, lane) : 1;
        const int cy0 = max(0, yr - a.R), cy1 = min(a.H - PS, yr + a.R);
        const int cx0 = max(0, xr - a.R), cx1 = min(a.W - PS, xr + a.R);
        const int ncol = cx1 - cx0 + 1, ncand = (cy1 - cy0 + 1) * ncol;
        double dl[L];
        int il[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            dl[i] = __longlong_as_double(0x7ff0000000000000ll);  // +inf
            il[i] = 0x7fffffff;
        }
        for (int c = lane; c < ncand; c += 32) {
            const int cy = cy0 + c / ncol, cx = cx0 + c % ncol;
            if (cy == yr && cx == xr) continue;
            const double D = exact_dist(a.img, a.W, HW, a.C, green, yr, xr, cy, cx);
            const int id = cy * a.W + cx;
            if (D > dl[L - 1] || (D == dl[L - 1] && id > il[L - 1])) continue;
            // insertion keeping (D, id) ascending
#pragma unroll
            for (int i = L - 1; i > 0; --i) {
                const bool shift = (dl[i - 1] > D) || (dl[i - 1] == D && il[i - 1] > id);
                const bool here = !shift && ((dl[i] > D) || (dl[i] == D && il[i] > id));
                if (shift) { dl[i] = dl[i - 1]; il[i] = il[i - 1]; }
                else if (here) { dl[i] = D; il[i] = id; }
            }
            if ((dl[0] > D) || (dl[0] == D && il[0] > id)) { dl[0] = D; il[0] = id; }
        }
        int32_t *out = a.idx + (size_t)r * K;
        if (lane == 0) out[0] = yr * a.W + xr;
        for (int j = 0; j < L; ++j) {
            double bd = dl[0];
            int bi = il[0];
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double od = __shfl_xor_sync(FULL, bd, o);
                const int oi = __shfl_xor_sync(FULL, bi, o);
                if (od < bd || (od == bd && oi < bi)) { bd = od; bi = oi; }
            }
            if (lane == 0) out[1 + j] = bi;
            if (il[0] == bi && dl[0] == bd) {
#pragma unroll
                for (int q = 0; q < L - 1; ++q) { dl[q] = dl[q + 1]; il[q] = il[q + 1]; }
                dl[L - 1] = __longlong_as_double(0x7ff0000000000000ll);
                il[L - 1] = 0x7fffffff;
            }
        }
    }
}

template <int K>
hts_status launch_k(const MatchArgs &a, cudaStream_t s) {
    constexpr int M = K + 3;
    const int nwarps = 4;
    const int RW = 2 * a.R + PS;
    const size_t smem = (size_t)nwarps * M * 16 + (size_t)nwarps * RW * RW * sizeof(float);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_match<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return check_launch("cudaFuncSetAttribute(k_match)");
    }
    const int blocks = (a.nref + nwarps - 1) / nwarps;
    {
        KTimer kt("k_match", s);
        k_match<K><<<blocks, nwarps * 32, smem, s>>>(a);
    }
    hts_status st = check_launch("k_match");
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_match_fallback", s);
        k_match_fallback<K><<<152, 128, 0, s>>>(a);
    }
    return check_launch("k_match_fallback");
}

}  // namespace

hts_status launch_match(const float *img, const Geom &g, double gamma_gcp, int32_t *idx, uint8_t *green,
                        int32_t *fallback_list, DevState *st, cudaStream_t s) {
    MatchArgs a;
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.C = g.C;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.nref = g.nref;
    a.gamma = gamma_gcp;
    a.idx = idx;
    a.green = green;
    a.fb = fallback_list;
    a.st = st;
    switch (g.K) {
        case 2: return launch_k<2>(a, s);
        case 4: return launch_k<4>(a, s);
        case 8: return launch_k<8>(a, s);
        case 16: return launch_k<16>(a, s);
        case 32: return launch_k<32>(a, s);
        default: return HTS_EUNSUPPORTED;
    }
}

}  // namespace hts
