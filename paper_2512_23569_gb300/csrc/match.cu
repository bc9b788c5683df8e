// Grouping step of Haar-tSVD (Eq. 9, Alg. 1 step 1) on sm_103a.
//
// A block of four warps takes a 2x2 block of reference patches and stages the
// union of their search regions of the matching planes in shared memory
// (gray image; for colour both the green channel and the channel sum R+G+B,
// since Eq. 9 picks one per reference).  Each warp takes one reference:
// lanes compute FP32 squared distances of 4 horizontally adjacent
// candidates per item (register-blocked), store every distance in shared
// memory and keep a sorted per-lane list of their 4 smallest keys (distance
// bits, raster index).  The (K-1)-th smallest key of the 32 lists bounds the
// true (K-1)-th from above; the warp then collects every candidate under the
// certified threshold (usually K-1 plus a few) and sorts only those.
//
// Exactness.  The group must equal the FP64 definition bit for bit: the K-1
// nearest candidates in ascending (distance, raster index), distances being
// the FP64 row-major sum of squared differences.  The FP32 distance d of a
// candidate whose FP64 distance is D obeys |d - D| <= eps D + beta sqrt(D) + g0
// (eps covers 66 roundings of the subtract / FMA chain; beta and g0 cover the
// rounding of the FP32 channel sum on the R+G+B plane, scaled by the largest
// |R|+|G|+|B| of the region; g0 also absorbs subnormal flushing).  If every
// adjacent pair among the first K sorted entries is separated by that bound,
// the FP32 order is the FP64 order.  Otherwise every entry that can still
// belong to the K-1 nearest is re-evaluated with the FP64 expression in the
// same operation order as the definition and ranked by (D, index).  When the
// candidate set exceeds what a warp handles (flat, noiseless inputs with
// massive ties), the reference goes to an exhaustive FP64 pass.
#include "hts_internal.h"

namespace hts {
namespace {

constexpr float U32 = 5.9604644775390625e-08f;  // 2^-24
constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t EMPTY = ~0ull;

struct MatchArgs {
    const float *img;
    int H, W, C, step, R, nx, ny, nref;
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

constexpr int MW = 4;      // warps per block = a 2x2 block of reference patches sharing one staged region
constexpr int LTOP = 4;    // per-lane short list that bounds the (K-1)-th distance from above
constexpr int PMAX = 64;   // largest candidate set a warp certifies or re-ranks itself

// Eq. 9 with FP32 channel norms (64-term sums, relative error < 40 u): the
// decision is certain when nG^2 gamma^2 and max(nR^2, nB^2) differ by more
// than 1e-5 relative; otherwise the FP64 sequential definition decides.
__device__ int gcp_green_fast(const float *__restrict__ img, int W, size_t HW, int y, int x, double gamma, int lane) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = lane + 32 * q;
        const size_t o = (size_t)(y + (e >> 3)) * W + x + (e & 7);
        const float r = __ldg(img + o), g = __ldg(img + HW + o), b = __ldg(img + 2 * HW + o);
        s0 = fmaf(r, r, s0);
        s1 = fmaf(g, g, s1);
        s2 = fmaf(b, b, s2);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(FULL, s0, o);
        s1 += __shfl_xor_sync(FULL, s1, o);
        s2 += __shfl_xor_sync(FULL, s2, o);
    }
    const float lhs = s1 * (float)(gamma * gamma), rhs = fmaxf(s0, s2);
    if (lhs > rhs * (1.f + 1e-5f) && lhs > 0.f) return 1;
    if (lhs < rhs * (1.f - 1e-5f)) return 0;
    return gcp_green(img, W, HW, y, x, gamma, lane);
}

template <int K>
__global__ void __launch_bounds__(MW * 32) k_match(MatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RHM = a.step + 2 * a.R + PS;          // region side bound
    const int NCM = (2 * a.R + 1) * (2 * a.R + 1);  // candidates per window bound
    uint64_t *plist = reinterpret_cast<uint64_t *>(smem_raw) + warp * 2 * PMAX;
    uint64_t *psort = plist + PMAX;
    double *pd64 = reinterpret_cast<double *>(smem_raw) + MW * 2 * PMAX + warp * PMAX;
    float *planeA = reinterpret_cast<float *>(smem_raw + (size_t)MW * 3 * PMAX * 8);
    float *planeS = planeA + RHM * RHM;
    float *dbuf = planeS + (a.C == 3 ? RHM * RHM : 0) + warp * NCM;
    __shared__ unsigned s_tmax;

    const int nbx = (a.nx + 1) >> 1;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    const int gy = 2 * by + (warp >> 1), gx = 2 * bx + (warp & 1);
    const size_t HW = (size_t)a.H * a.W;
    // region = union of the block's windows (plus the patch extent)
    const int ya = grid_pos(2 * by, a.H, a.step), yb = grid_pos(min(2 * by + 1, a.ny - 1), a.H, a.step);
    const int xa = grid_pos(2 * bx, a.W, a.step), xb = grid_pos(min(2 * bx + 1, a.nx - 1), a.W, a.step);
    const int ry0 = max(0, ya - a.R), ry1 = min(a.H - PS, yb + a.R) + PS - 1;
    const int rx0 = max(0, xa - a.R), rx1 = min(a.W - PS, xb + a.R) + PS - 1;
    const int rh = ry1 - ry0 + 1, rw = rx1 - rx0 + 1;
    if (threadIdx.x == 0) s_tmax = 0u;
    __syncthreads();
    float tmax = 0.f;
    for (int e = threadIdx.x; e < rh * rw; e += blockDim.x) {
        const int yy = e / rw, xx = e - yy * rw;
        const size_t o = (size_t)(ry0 + yy) * a.W + (rx0 + xx);
        if (a.C == 1) {
            planeA[e] = __ldg(a.img + o);
        } else {
            const float R = __ldg(a.img + o), G = __ldg(a.img + HW + o), B = __ldg(a.img + 2 * HW + o);
            planeA[e] = G;
            planeS[e] = __fadd_rn(__fadd_rn(R, G), B);
            tmax = fmaxf(tmax, fabsf(R) + fabsf(G) + fabsf(B));
        }
    }
    tmax = warp_max_f(tmax);
    if (lane == 0) atomicMax(&s_tmax, __float_as_uint(tmax));  // non-negative floats order as their bits
    __syncthreads();
    if (gy >= a.ny || gx >= a.nx) return;  // no block-wide barrier below

    const int r = gy * a.nx + gx;
    const int yr = grid_pos(gy, a.H, a.step), xr = grid_pos(gx, a.W, a.step);
    const int green = (a.C == 3) ? gcp_green_fast(a.img, a.W, HW, yr, xr, a.gamma, lane) : 1;
    if (lane == 0 && a.green) a.green[r] = (uint8_t)green;
    const bool exact_plane = (a.C == 1) || green;
    const float *plane = exact_plane ? planeA : planeS;
    const float T3 = exact_plane ? 0.f : __uint_as_float(s_tmax);

    const int cy0 = max(0, yr - a.R), cy1 = min(a.H - PS, yr + a.R);
    const int cx0 = max(0, xr - a.R), cx1 = min(a.W - PS, xr + a.R);
    const int nrow = cy1 - cy0 + 1, ncol = cx1 - cx0 + 1, nc = nrow * ncol;
    const int oy = cy0 - ry0, ox = cx0 - rx0;

    float ar[NPIX];
    {
        const float *rp = plane + (yr - ry0) * rw + (xr - rx0);
#pragma unroll
        for (int u = 0; u < PS; ++u)
#pragma unroll
            for (int v = 0; v < PS; ++v) ar[u * PS + v] = rp[u * rw + v];
    }
    uint64_t lst[LTOP];
#pragma unroll
    for (int i = 0; i < LTOP; ++i) lst[i] = EMPTY;

    const int nq = (ncol + 3) >> 2;
    const int nitems = nrow * nq;
    for (int it = lane; it < nitems; it += 32) {
        const int i = it / nq, cxb = (it - i * nq) * 4;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const float *base = plane + (oy + i) * rw + ox + cxb;
        const int lim = rw - ox - cxb;  // columns of the region right of this quad's first candidate
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const float *row = base + u * rw;
            float b[PS + 3];
#pragma unroll
            for (int t = 0; t < PS + 3; ++t) b[t] = (t < lim) ? row[t] : 0.f;
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
        const int gyy = cy0 + i;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int cx = cxb + t;
            if (cx < ncol) {
                const int gxx = cx0 + cx;
                if (gyy == yr && gxx == xr) {
                    dbuf[i * ncol + cx] = __int_as_float(0x7f800000);  // the reference itself: never collected
                } else {
                    dbuf[i * ncol + cx] = d[t];
                    topm_insert<LTOP>(lst, make_key(d[t], gyy * a.W + gxx));
                }
            }
        }
    }
    __syncwarp();

    // (K-1)-th smallest key of the union of the lane lists: an upper bound of the true one
    uint64_t tau = EMPTY;
    for (int j = 0; j < K - 1; ++j) {
        const uint64_t h = lst[0];
        const uint64_t mn = warp_min_u64(h);
        if (h == mn && mn != EMPTY) {
#pragma unroll
            for (int q = 0; q < LTOP - 1; ++q) lst[q] = lst[q + 1];
            lst[LTOP - 1] = EMPTY;
        }
        tau = mn;
    }
    int32_t *out = a.idx + (size_t)r * K;
    if (lane == 0) out[0] = yr * a.W + xr;
    Bound bd;
    bd.eps = 100.f * U32;
    bd.beta = exact_plane ? 0.f : 72.f * U32 * T3;
    bd.g0 = (exact_plane ? 0.f : 1200.f * U32 * U32 * T3 * T3) + 1e-30f;
    bool overflow = (tau == EMPTY);
    // collect every candidate whose distance may still matter
    int m = 0;
    if (!overflow) {
        const float T = bd.upper(bd.upper(key_dist(tau)));
        const unsigned lt = (1u << lane) - 1u;
        for (int c0 = 0; c0 < nc; c0 += 32) {
            const int c = c0 + lane;
            const float dv = (c < nc) ? dbuf[c] : __int_as_float(0x7f800000);
            const bool ok = dv <= T;
            const unsigned msk = __ballot_sync(FULL, ok);
            if (ok) {
                const int pos = m + __popc(msk & lt);
                if (pos < PMAX) {
                    const int ci = c / ncol;
                    plist[pos] = make_key(dv, (cy0 + ci) * a.W + cx0 + (c - ci * ncol));
                }
            }
            m += __popc(msk);
        }
        overflow = (m > PMAX) || (m < K - 1);
    }
    if (overflow) {
        if (lane == 0) {
            const int pos = atomicAdd(&a.st->match_fallback, 1);
            a.fb[pos] = r;
        }
        return;
    }
    __syncwarp();
    // rank sort of the collected keys (unique: the raster index is part of the key)
    for (int e = lane; e < m; e += 32) {
        const uint64_t key = plist[e];
        int rank = 0;
        for (int j = 0; j < m; ++j) rank += (plist[j] < key) ? 1 : 0;
        psort[rank] = key;
    }
    __syncwarp();
    bool ok = true;
    for (int i = lane; i < K - 1; i += 32)
        if (i + 1 < m) ok = ok && (bd.upper(key_dist(psort[i])) < bd.lower(key_dist(psort[i + 1])));
    if (__all_sync(FULL, ok)) {
        for (int i = lane; i < K - 1; i += 32) out[1 + i] = key_idx(psort[i]);
        return;
    }
    // uncertain order: FP64 re-rank of every entry that may belong to the K-1 nearest
    const float thr = bd.upper(key_dist(psort[K - 2]));
    int mp = 0;
    for (int i = 0; i < m; ++i) {
        if (bd.lower(key_dist(psort[i])) > thr) break;
        mp = i + 1;
    }
    for (int i = lane; i < mp; i += 32) {
        const int id = key_idx(psort[i]);
        pd64[i] = exact_dist(a.img, a.W, HW, a.C, green, yr, xr, id / a.W, id % a.W);
    }
    __syncwarp();
    for (int i = lane; i < mp; i += 32) {
        const double di = pd64[i];
        const int ii = key_idx(psort[i]);
        int rank = 0;
        for (int j = 0; j < mp; ++j) {
            const double dj = pd64[j];
            const int ij = key_idx(psort[j]);
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

// Exhaustive matching, in FP32, of the references the tensor-core matcher
// listed in a.fb (count in a.st->match_fallback): one block of four warps per
// reference, its search region staged in shared memory as FP32 plane values
// ((R + G) + B for the channel sum), distances as FP32 fused multiply-adds
// in the definition's (u, v) order -- the arithmetic of the tensor-core
// matcher's re-rank -- and the K-1 nearest by (distance, raster index).  The
// matching plane comes from a.green (Eq. 9 flags already decided).
template <int K>
__global__ void __launch_bounds__(128) k_match_rescue(MatchArgs a) {
    constexpr int L = K - 1;
    extern __shared__ float rs_plane[];  // (2R + 8)^2 region values, then the warps' lists
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int count = *(volatile int *)&a.st->match_fallback;
    const size_t HW = (size_t)a.H * a.W;
    const int side = 2 * a.R + PS;
    float *wd = rs_plane + (size_t)side * side;  // [4][L]
    int *wi = reinterpret_cast<int *>(wd + 4 * L);  // [4][L]
    for (int f = blockIdx.x; f < count; f += gridDim.x) {
        const int r = a.fb[f];
        const int yr = grid_pos(r / a.nx, a.H, a.step), xr = grid_pos(r % a.nx, a.W, a.step);
        const int green = (a.C == 3) ? (int)a.green[r] : 1;
        const int cy0 = max(0, yr - a.R), cy1 = min(a.H - PS, yr + a.R);
        const int cx0 = max(0, xr - a.R), cx1 = min(a.W - PS, xr + a.R);
        const int ncol = cx1 - cx0 + 1, ncand = (cy1 - cy0 + 1) * ncol;
        const int rw = ncol + PS - 1, rh = cy1 - cy0 + PS;  // staged rows and columns
        __syncthreads();  // the previous reference's lists are read
        for (int e = tid; e < rw * rh; e += 128) {
            const int y = e / rw, x = e - y * rw;
            const size_t o = (size_t)(cy0 + y) * a.W + cx0 + x;
            float v;
            if (a.C == 1) v = __ldg(a.img + o);
            else if (green) v = __ldg(a.img + HW + o);
            else v = (__ldg(a.img + o) + __ldg(a.img + HW + o)) + __ldg(a.img + 2 * HW + o);
            rs_plane[e] = v;
        }
        __syncthreads();
        const float *ref = rs_plane + (size_t)(yr - cy0) * rw + (xr - cx0);
        float dl[L];
        int il[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            dl[i] = __builtin_huge_valf();
            il[i] = 0x7fffffff;
        }
        for (int c = tid; c < ncand; c += 128) {
            const int cy = c / ncol, cx = c - cy * ncol;
            if (cy0 + cy == yr && cx0 + cx == xr) continue;
            const float *cand = rs_plane + (size_t)cy * rw + cx;
            float D = 0.f;
            for (int u = 0; u < PS; ++u)
#pragma unroll
                for (int v = 0; v < PS; ++v) {
                    const float d = ref[u * rw + v] - cand[u * rw + v];
                    D = fmaf(d, d, D);
                }
            const int id = (cy0 + cy) * a.W + cx0 + cx;
            if (D > dl[L - 1] || (D == dl[L - 1] && id > il[L - 1])) continue;
#pragma unroll
            for (int i = L - 1; i > 0; --i) {
                const bool shift = (dl[i - 1] > D) || (dl[i - 1] == D && il[i - 1] > id);
                const bool here = !shift && ((dl[i] > D) || (dl[i] == D && il[i] > id));
                if (shift) {
                    dl[i] = dl[i - 1];
                    il[i] = il[i - 1];
                } else if (here) {
                    dl[i] = D;
                    il[i] = id;
                }
            }
            if ((dl[0] > D) || (dl[0] == D && il[0] > id)) {
                dl[0] = D;
                il[0] = id;
            }
        }
        // each warp: the L smallest of its lanes' lists (L rounds of a warp arg-min over the list heads)
        for (int j = 0; j < L; ++j) {
            float bd = dl[0];
            int bi = il[0];
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const float od = __shfl_xor_sync(FULL, bd, o);
                const int oi = __shfl_xor_sync(FULL, bi, o);
                if (od < bd || (od == bd && oi < bi)) {
                    bd = od;
                    bi = oi;
                }
            }
            if (lane == 0) {
                wd[warp * L + j] = bd;
                wi[warp * L + j] = bi;
            }
            if (il[0] == bi && dl[0] == bd) {
#pragma unroll
                for (int t = 0; t < L - 1; ++t) {
                    dl[t] = dl[t + 1];
                    il[t] = il[t + 1];
                }
                dl[L - 1] = __builtin_huge_valf();
                il[L - 1] = 0x7fffffff;
            }
        }
        __syncthreads();
        if (tid == 0) {  // merge of the four warps' sorted lists
            int h[4] = {0, 0, 0, 0};
            int32_t *out = a.idx + (size_t)r * K;
            out[0] = yr * a.W + xr;
            for (int j = 0; j < L; ++j) {
                int bw = -1;
                float bd = 0.f;
                int bi = 0x7fffffff;
                for (int w = 0; w < 4; ++w) {
                    if (h[w] >= L) continue;
                    const float dv = wd[w * L + h[w]];
                    const int iv = wi[w * L + h[w]];
                    if (bw < 0 || dv < bd || (dv == bd && iv < bi)) {
                        bw = w;
                        bd = dv;
                        bi = iv;
                    }
                }
                ++h[bw];
                out[1 + j] = (bi == 0x7fffffff) ? out[0] : bi;
            }
        }
    }
}

template <int K>
hts_status launch_k(const MatchArgs &a, cudaStream_t s) {
    const int RHM = a.step + 2 * a.R + PS;
    const int NCM = (2 * a.R + 1) * (2 * a.R + 1);
    const size_t smem = (size_t)MW * 3 * PMAX * 8 + (size_t)(a.C == 3 ? 2 : 1) * RHM * RHM * sizeof(float) +
                        (size_t)MW * NCM * sizeof(float);
    {
        const hts_status st0 = allow_smem(reinterpret_cast<const void *>(k_match<K>), smem);
        if (st0 != HTS_OK) return st0;
    }
    const int blocks = ((a.ny + 1) / 2) * ((a.nx + 1) / 2);
    {
        KTimer kt("k_match", s);
        k_match<K><<<blocks, MW * 32, smem, s>>>(a);
    }
    hts_status st = check_launch("k_match");
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_match_fallback", s);
        k_match_fallback<K><<<152, 128, 0, s>>>(a);
    }
    return check_launch("k_match_fallback");
}

// Eq. 9 flag of every reference patch, for the tensor-core matching path, which reads the flags instead of
// deciding them itself: two references per warp (a half-warp each, four pixels of the 8 x 8 patch per lane),
// the FP32 screen of gcp_green_fast (the same sums in another order, inside the same margin), and the FP64
// decision by the whole warp for a reference the screen leaves open.
__global__ void __launch_bounds__(128) k_gcp_flags(const float *__restrict__ img, int H, int W, int step, int nx,
                                                   int nref, double gamma, uint8_t *__restrict__ green) {
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const size_t HW = (size_t)H * W;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2; r0 < nref; r0 += 2 * nwarp) {
        const int r = min(r0 + half, nref - 1);  // the last odd reference is decided twice, identically
        const int gy = r / nx, gx = r - gy * nx;
        const int yr = grid_pos(gy, H, step), xr = grid_pos(gx, W, step);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = hl + 16 * q;
            const size_t o = (size_t)(yr + (e >> 3)) * W + xr + (e & 7);
            const float rv = __ldg(img + o), gv = __ldg(img + HW + o), bv = __ldg(img + 2 * HW + o);
            s0 = fmaf(rv, rv, s0);
            s1 = fmaf(gv, gv, s1);
            s2 = fmaf(bv, bv, s2);
        }
#pragma unroll
        for (int o = 8; o; o >>= 1) {
            s0 += __shfl_xor_sync(FULL, s0, o);
            s1 += __shfl_xor_sync(FULL, s1, o);
            s2 += __shfl_xor_sync(FULL, s2, o);
        }
        const float lhs = s1 * (float)(gamma * gamma), rhs = fmaxf(s0, s2);
        int flag = -1;  // -1: open
        if (lhs > rhs * (1.f + 1e-5f) && lhs > 0.f) flag = 1;
        else if (lhs < rhs * (1.f - 1e-5f)) flag = 0;
        const unsigned open = __ballot_sync(FULL, flag < 0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (open & (1u << (16 * h))) {  // the whole warp decides reference r0 + h in FP64
                const int rh = min(r0 + h, nref - 1);
                const int gyh = rh / nx, gxh = rh - gyh * nx;
                const int f = gcp_green(img, W, HW, grid_pos(gyh, H, step), grid_pos(gxh, W, step), gamma, lane);
                if (half == h) flag = f;
            }
        }
        if (hl == 0 && r0 + half < nref) green[r] = (uint8_t)flag;
    }
}

}  // namespace

hts_status launch_gcp_flags(const float *img, const Geom &g, double gamma_gcp, uint8_t *green, cudaStream_t s) {
    int blocks = (g.nref + 7) / 8;  // four warps of two references
    if (blocks > 152 * 16) blocks = 152 * 16;
    {
        KTimer kt("k_gcp_flags", s);
        k_gcp_flags<<<blocks, 128, 0, s>>>(img, g.H, g.W, g.step, g.nx, g.nref, gamma_gcp, green);
    }
    return check_launch("k_gcp_flags");
}

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
    a.ny = g.ny;
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

hts_status launch_match_rescue(const float *img, const Geom &g, int32_t *idx, const uint8_t *green,
                               int32_t *fallback_list, DevState *st, cudaStream_t s) {
    MatchArgs a;
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.C = g.C;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nref = g.nref;
    a.gamma = 0.0;
    a.idx = idx;
    a.green = const_cast<uint8_t *>(green);
    a.fb = fallback_list;
    a.st = st;
    const size_t side = 2 * (size_t)g.R + PS;
    const size_t smem = side * side * sizeof(float) + 4 * 32 * (sizeof(float) + sizeof(int));
    const void *fn = nullptr;
    switch (g.K) {
        case 2: fn = reinterpret_cast<const void *>(k_match_rescue<2>); break;
        case 4: fn = reinterpret_cast<const void *>(k_match_rescue<4>); break;
        case 8: fn = reinterpret_cast<const void *>(k_match_rescue<8>); break;
        case 16: fn = reinterpret_cast<const void *>(k_match_rescue<16>); break;
        case 32: fn = reinterpret_cast<const void *>(k_match_rescue<32>); break;
        default: return HTS_EUNSUPPORTED;
    }
    {
        const hts_status st0 = allow_smem(fn, smem);
        if (st0 != HTS_OK) return st0;
    }
    const int blocks = 4 * 152;
    {
        KTimer kt("k_match_rescue", s);
        switch (g.K) {
            case 2: k_match_rescue<2><<<blocks, 128, smem, s>>>(a); break;
            case 4: k_match_rescue<4><<<blocks, 128, smem, s>>>(a); break;
            case 8: k_match_rescue<8><<<blocks, 128, smem, s>>>(a); break;
            case 16: k_match_rescue<16><<<blocks, 128, smem, s>>>(a); break;
            default: k_match_rescue<32><<<blocks, 128, smem, s>>>(a); break;
        }
    }
    return check_launch("k_match_rescue");
}

}  // namespace hts
