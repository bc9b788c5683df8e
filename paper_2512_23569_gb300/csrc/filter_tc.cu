// Collaborative filtering of the precision form on the sm_103a tensor cores
// (Eq. 19-21, Alg. 1 steps 2-3), FP32 threshold decisions.
//
// The unitary DFT along the channels (Eq. 4-5) and the separable projection
// Shat = U^H Phat V of every Fourier slice (Eq. 19) are linear in the patch's
// raw pixels, so together they are one real orthogonal matrix F (192 x 192
// for colour, 64 x 64 for gray) applied to the patch read as a vector of its
// R, G, B pixels, giving [S^(1) | sqrt2 Re S^(2) | sqrt2 Im S^(2)] (slice 3 is
// the conjugate of slice 2).  A batch of 128 group members (8 groups of K =
// 16) is one GEMM with the members as the MMA's M = 128 rows: D[m][coefficient]
// = sum_pixel A[m][pixel] F[coefficient][pixel], FP16 operands, FP32
// accumulation in tensor memory (tcgen05.mma kind::f16, N = 192).  The
// inverse (Eq. 21 and the inverse channel DFT) is F^T: the same shared-memory
// matrix read with the transpose bit (MN-major), giving the R, G, B pixels of
// every member directly.  Between the two, the coefficients go through shared
// memory (transposed, FP32) so that one thread holds a coefficient stream of a
// group: Haar along the group axis (Eq. 8), hard threshold (Eq. 20, modulus
// for the complex slice, the group's tau), inverse Haar; then FP16 again as
// the inverse GEMM's A operand.
//
// FP16 rather than BF16: pixels lie in a bounded range and the bases are
// orthonormal, so FP16's 11-bit significand fits the data, where BF16's 8
// bits would put a rounding error of up to one grey level on the input.
//
// Aggregation: fixed-point integer sums (value * 2^8, rounded) of the
// estimates in 32-bit shared-memory accumulators over the tile's region
// (at most 2^10 members of a tile cover a pixel: no overflow), flushed to
// the image-wide int64 sums (2^16 scale) once per tile; integer sums do not
// depend on the order of the additions, so the result is deterministic.
// Weights: every member adds 1 to the count of its patch origin (top-left
// pixel) instead of 1 to each of its 64 pixels; a pixel's weight is the sum of
// the origin counts over the 8 x 8 origins whose patch covers it, formed by
// k_normalize_box.  The MMA waits
// are bounded: a wait that gives up records DevState.error = 2, waits
// (bounded) for the MMAs, frees the tensor memory and leaves.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "filter_common.h"
#include "hts_internal.h"
#include "tc_ptx.h"

namespace hts {
namespace {

using fc::K3F;

// The Haar transform of Eq. 8 without its 1/sqrt(2) factors: sums and differences only.  In the row
// order of Eq. 8 (row 0 the sum, then the difference rows coarse to fine) coefficient k has passed
// l_k butterflies, l_0 = log2 K and l_k = log2 K - floor(log2 k) for k >= 1, and equals 2^(l_k / 2)
// times the orthonormal one.  A coefficient is kept iff the orthonormal value reaches tau, i.e. iff
// |x_k| >= tau 2^(l_k / 2); kept ones are scaled by 2^(-l_k) (exact), after which the unnormalised
// inverse butterflies give the orthonormal inverse.
template <int K>
__device__ __forceinline__ void haar_fwd_u(float (&x)[K]) {
#pragma unroll
    for (int n = K; n >= 2; n >>= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[i] = x[2 * i] + x[2 * i + 1];
            t[n / 2 + i] = x[2 * i] - x[2 * i + 1];
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

template <int K>
__device__ __forceinline__ void haar_inv_u(float (&x)[K]) {
#pragma unroll
    for (int n = 2; n <= K; n <<= 1) {
        float t[K];
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            t[2 * i] = x[i] + x[n / 2 + i];
            t[2 * i + 1] = x[i] - x[n / 2 + i];
        }
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = t[i];
    }
}

// Butterflies coefficient k of a K-long unnormalised Haar transform has passed.
template <int K>
__host__ __device__ constexpr int haar_level(int k) {
    int L = 0;
    while ((1 << L) < K) ++L;
    if (k == 0) return L;
    int f = 0;
    while ((2 << f) <= k) ++f;
    return L - f;
}

constexpr int NT = 512;   // 16 warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31, column quarter w / 4
constexpr int MB = 128;   // group members per batch = MMA M
constexpr int TS = MB + 4;  // row stride (floats) of the transpose buffer: conflict-free float4 reads
constexpr long long SPIN = 1ll << 24;

// Offset (in halves) of element (r, k) of a K-major FP16 operand block of 64
// columns, no swizzle: core matrices of 8 rows x 8 columns (128 B), 8-column
// groups 128 B apart (LBO), 8-row groups 1024 B apart (SBO).
__device__ __forceinline__ int cm_off(int r, int k) { return (((r >> 3) << 3) + (k >> 3)) * 64 + ((r & 7) << 3) + (k & 7); }

template <int C>
struct FtcLayout {
    static constexpr int NBLK = (C == 3) ? 3 : 1;  // 64-column blocks of the member operand
    // The FP16 transform F [coefficient][pixel] (CK x CK, CK = 64 C), K-major, core matrices of 8 rows x 8
    // columns, 8-column groups 128 B apart along K and 8-row groups CK * 16 B apart: the forward GEMM's B
    // operand, and with the transpose bit (K = coefficients, N = pixels, MN-major) the inverse's.
    static constexpr int CK = 64 * C;
    static constexpr int B_HALVES = CK * CK;
    static constexpr size_t a_off = 0;                               // [NBLK][128][64] FP16
    static constexpr size_t b_off = a_off + (size_t)NBLK * MB * 64 * 2;
    static constexpr size_t t_off = b_off + (size_t)B_HALVES * 2;    // [64][TS] FP32
    static constexpr size_t basis_off = t_off + (size_t)64 * TS * 4;  // 6 x 64 FP32
    static constexpr size_t misc_off = basis_off + (size_t)6 * 64 * 4;
    // misc, two buffers each: pos[MB] int, tau[32] float; 2 mbarrier words, tensor-memory slot
    static constexpr size_t job_off = misc_off + (size_t)2 * (MB * 4 + 32 * 4) + 16 + 16;  // the current job
    static constexpr size_t acc_off = job_off + 256;
    static constexpr uint32_t tcols = (C == 3) ? 256 : 64;
};

struct FtcArgs {
    const float *img;
    int H, W, step, R, nx, ny;
    const int32_t *idx;
    const float *b32;
    long long *acc;
    int *wcount;
    const float *sigma_ref;
    int map_judged;
    double tau_scale;
    const float *mean_est;  // [N_ref][C][64] refined mean patches (enhancement strategy) or nullptr
    DevState *st;
    int ty, tx, nty, ntx, ntiles, rh_max, rw_max;
};

// A launch over the images of a batch (same C and K): jobs (device array of every image's arguments with
// its tile shape) and their tiles taken in turn; job j owns tiles tile_start[j] .. tile_start[j+1]-1.
struct FtcBatch {
    const FtcArgs *jobs;
    const int *tile_start;
    int njobs, ntiles;
    int rh_max, rw_max;  // the largest tile region over the jobs
};

// BATCH: the tiles of every job of `bt` (a0 unused); else the tiles of the one image a0 (bt unused).
template <int C, int K, bool BATCH>
__global__ void __launch_bounds__(NT, 1) k_filter_tc(const __grid_constant__ FtcArgs a0,
                                                     const __grid_constant__ FtcBatch bt) {
    using L = FtcLayout<C>;
    static_assert(sizeof(FtcArgs) <= 256, "the job fits its shared-memory slot");
    constexpr int GPB = MB / K;  // groups per batch
    extern __shared__ __align__(1024) unsigned char smem[];
    __half *sA = reinterpret_cast<__half *>(smem + L::a_off);
    __half *sB = reinterpret_cast<__half *>(smem + L::b_off);
    float *sT = reinterpret_cast<float *>(smem + L::t_off);
    float *sBas = reinterpret_cast<float *>(smem + L::basis_off);
    int *sPos = reinterpret_cast<int *>(smem + L::misc_off);  // [2][MB] members' top-left pixels
    float *sTau = reinterpret_cast<float *>(sPos + 2 * MB);    // [2][32] groups' thresholds
    uint64_t *bar = reinterpret_cast<uint64_t *>(sTau + 64);  // 8-byte aligned: misc_off + 1280
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
    int *accs = reinterpret_cast<int *>(smem + L::acc_off);
    FtcArgs *sjob = reinterpret_cast<FtcArgs *>(smem + L::job_off);
    const FtcArgs &a = BATCH ? *sjob : a0;  // the current job's arguments
    const int RA = BATCH ? bt.rh_max * bt.rw_max : a0.rh_max * a0.rw_max;
    int *acc_v = accs, *acc_w = accs + C * RA;  // [C][RA] sums of value * 2^8, [RA] patch-origin counts
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---- bases (row-major 8x8, element (r, c) at r * 8 + c) and the transform F of the current job
    constexpr int CK = L::CK;
    auto build_f = [&]() {
        for (int t = tid; t < 64; t += NT) {
            sBas[t] = a.b32[(0 * 64 + t) * 2];        // U0
            sBas[64 + t] = a.b32[(1 * 64 + t) * 2];   // V0
            if (C == 3) {
                sBas[128 + t] = a.b32[(2 * 64 + t) * 2];      // U1 re
                sBas[192 + t] = a.b32[(2 * 64 + t) * 2 + 1];  // U1 im
                sBas[256 + t] = a.b32[(3 * 64 + t) * 2];      // V1 re
                sBas[320 + t] = a.b32[(3 * 64 + t) * 2 + 1];  // V1 im
            }
        }
        __syncthreads();
        // F: the unitary DFT along the channels (Eq. 4-5) followed by the slices' projections (Eq. 19), as one real
        // orthogonal map of the raw R, G, B pixels (column t * 64 + (i, j)) to [S^(1) | sqrt2 Re S^(2) |
        // sqrt2 Im S^(2)] (row (a, b), 64 + (a, b), 128 + (a, b)); its inverse (Eq. 21) is its transpose.
        // Slice 1: P^(1) = (R + w G + w^2 B) / sqrt3, w = exp(-2 pi i / 3), projected by conj(U1[i][a]) V1[j][b].
        for (int e = tid; e < CK * CK; e += NT) {
            const int n = e / CK, k = e - n * CK;  // n: coefficient row, k: channel t = k / 64, pixel (i, j)
            const int t = k >> 6, px = k & 63, nc = n & 63, sl = n >> 6;
            const int ia = (px >> 3) * 8 + (nc >> 3), jb = (px & 7) * 8 + (nc & 7);
            float f;
            if (sl == 0) {
                f = sBas[ia] * sBas[64 + jb];  // U0[i][a] V0[j][b]
                if (C == 3) f *= K3F;
            } else {
                const float ur = sBas[128 + ia], ui = sBas[192 + ia], vr = sBas[256 + jb], vi = sBas[320 + jb];
                const float mr = ur * vr + ui * vi, mi = ur * vi - ui * vr;  // conj(U1[i][a]) V1[j][b]
                // channel weights of Re and Im of P^(1): (1, -1/2, -1/2) / sqrt3 and (0, -1/2, 1/2)
                const float cr = (t == 0) ? K3F : -0.5f * K3F, ci = (t == 0) ? 0.f : (t == 1 ? -0.5f : 0.5f);
                const float v = (sl == 1) ? (mr * cr - mi * ci) : (mr * ci + mi * cr);
                f = v * 1.41421356237309505f;
            }
            sB[(((n >> 3) * (CK / 8) + (k >> 3)) << 6) + ((n & 7) << 3) + (k & 7)] = __float2half_rn(f);
        }
    };
    if (!BATCH) build_f();
    if (tid == 0) {
        tc::bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(slot, L::tcols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idf = tc::idesc_f16(MB, L::CK, false);                 // forward: B K-major
    const uint32_t idi = tc::idesc_f16(MB, L::CK, false) | (1u << 16);    // inverse: B transposed (MN-major)
    const int q = warp & 3, wq = warp >> 2;  // tensor-memory lane quarter, column quarter
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    uint32_t phase = 0;
    bool ok = true;

    // issue the MMAs of one GEMM stage and wait for them; false if the wait gave up
    auto run_stage = [&](bool inverse) -> bool {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::su32(sA), b0 = tc::su32(sB);
            // A: [NBLK][128][64] K-major (K step kk: block kk / 4, two core matrices at (kk % 4) * 256 B).
            // Forward B = F: K = pixels, core matrices 128 B apart along K, CK * 16 B along N (coefficients).
            // Inverse B = F^T read in place: K = coefficients (core matrices CK * 16 B apart: LBO), N = pixels
            // (128 B apart: SBO), the MN-major convention.
#pragma unroll
            for (int kk = 0; kk < CK / 16; ++kk) {
                const uint64_t ad = tc::sdesc(a0 + (kk >> 2) * (MB * 64 * 2) + (kk & 3) * 256, 128, 1024);
                const uint64_t bd = inverse ? tc::sdesc(b0 + kk * 2 * (CK * 16), CK * 16, 128)
                                            : tc::sdesc(b0 + kk * 256, 128, CK * 16);
                tc::mma_f16(tbase, ad, bd, inverse ? idi : idf, kk > 0 ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
        const bool done = tc::bar_wait(bar, phase, SPIN);
        if (__syncthreads_or(!done)) {
            if (tid == 0) {
                tc::bar_wait(bar, phase, SPIN);  // the MMAs must end before the memory is released
                atomicExch(&a.st->error, 2);
            }
            return false;
        }
        phase ^= 1u;
        tc::fence_after();
        return true;
    };

    // gather mapping: per step it, thread tid loads pixel (row, px) of member m(it); a warp covers one
    // patch row of 4 consecutive members (4 coalesced 32-byte segments)
    const int g_px = tid & 7, g_ml = (tid >> 3) & 3, g_row = (tid >> 5) & 7, g_mh = tid >> 8;
    constexpr int NPF = MB * 64 / NT;  // pixels per thread per batch
    int cur_job = -1;
    const int total = BATCH ? bt.ntiles : a0.ntiles;
    for (int gt = blockIdx.x; gt < total && ok; gt += gridDim.x) {
        int tile = gt;
        if (BATCH) {
            int lo = 0, hi = bt.njobs - 1;  // the job owning the tile: the last j with tile_start[j] <= gt
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bt.tile_start[mid] <= gt) lo = mid;
                else hi = mid - 1;
            }
            tile = gt - bt.tile_start[lo];
            if (lo != cur_job) {  // the job's arguments and its transform F (the previous MMAs have completed)
                const int *src = reinterpret_cast<const int *>(bt.jobs + lo);
                int *dst = reinterpret_cast<int *>(sjob);
                for (int w = tid; w < (int)(sizeof(FtcArgs) / 4); w += NT) dst[w] = src[w];
                cur_job = lo;
                __syncthreads();
                build_f();
                tc::fence_async_smem();
                __syncthreads();
            }
        }
        const size_t HW = (size_t)a.H * a.W;
        const bool use_map = a.sigma_ref && (!a.map_judged || a.st->learned);
        const bool ra = a.mean_est != nullptr;
        const int gpt = a.ty * a.tx;
        const int nbatch = (gpt + GPB - 1) / GPB;
        const int tyi = tile / a.ntx, txi = tile - tyi * a.ntx;
        const int gy0 = tyi * a.ty, gx0 = txi * a.tx;
        const int gy1 = min(a.ny, gy0 + a.ty) - 1, gx1 = min(a.nx, gx0 + a.tx) - 1;
        const int Y0 = grid_pos(gy0, a.H, a.step), Y1 = grid_pos(gy1, a.H, a.step);
        const int X0 = grid_pos(gx0, a.W, a.step), X1 = grid_pos(gx1, a.W, a.step);
        const int ry0 = max(0, Y0 - a.R), ry1 = min(a.H - 1, Y1 + a.R + PS - 1);
        const int rx0 = max(0, X0 - a.R), rx1 = min(a.W - 1, X1 + a.R + PS - 1);
        const int rh = ry1 - ry0 + 1, rw = rx1 - rx0 + 1;
        for (int e = tid; e < (C + 1) * RA; e += NT) accs[e] = 0;
        // the thresholds of batch bb's groups into buffer buf
        auto setup = [&](int bb, int buf) {
            if (tid < GPB) {
                const int lg = bb * GPB + tid;
                const int gy = gy0 + lg / a.tx, gx = gx0 + lg % a.tx;
                const bool valid = lg < gpt && gy <= gy1 && gx <= gx1;
                sTau[32 * buf + tid] = !valid ? 0.f
                                       : use_map ? (float)(a.tau_scale * (double)a.sigma_ref[gy * a.nx + gx])
                                                 : a.st->tau32;
            }
        };
        // member m (= tid < MB) of batch bb: its patch's top-left pixel, -1 for an empty group slot
        auto member_pos = [&](int bb) -> int {
            const int g = tid / K, k = tid - g * K;
            const int lg = bb * GPB + g;
            const int gy = gy0 + lg / a.tx, gx = gx0 + lg % a.tx;
            const bool valid = lg < gpt && gy <= gy1 && gx <= gx1;
            return valid ? __ldg(a.idx + (size_t)(gy * a.nx + gx) * K + k) : -1;
        };
        // this thread's pixels of the batch whose positions are in buffer buf, into registers
        float pf[NPF][C];
        auto prefetch = [&](int buf) {
#pragma unroll
            for (int it = 0; it < NPF; ++it) {
                const int m = 4 * (2 * it + g_mh) + g_ml;
                const int pos = sPos[MB * buf + m];
                const float *src = a.img + (pos >= 0 ? pos : 0) + g_row * a.W + g_px;  // a valid address either way
#pragma unroll
                for (int c = 0; c < C; ++c) pf[it][c] = pos >= 0 ? __ldg(src + c * HW) : 0.f;
            }
        };
        // registers -> FP16, member rows of the operand (channel c in block c; F applies the channel DFT)
        auto commit = [&]() {
#pragma unroll
            for (int it = 0; it < NPF; ++it) {
                const int m = 4 * (2 * it + g_mh) + g_ml;
                const int o = cm_off(m, g_row * 8 + g_px);
#pragma unroll
                for (int c = 0; c < C; ++c) sA[c * MB * 64 + o] = __float2half_rn(pf[it][c]);
            }
        };
        setup(0, 0);
        int posreg = -1;
        if (tid < MB) {
            sPos[tid] = member_pos(0);
            sPos[MB + tid] = nbatch > 1 ? member_pos(1) : -1;
            posreg = nbatch > 2 ? member_pos(2) : -1;
        }
        __syncthreads();
        prefetch(0);
        for (int b = 0; b < nbatch; ++b) {
            const int cur = b & 1;
            const float *bTau = sTau + 32 * cur;
            const int *bPos = sPos + MB * cur;
            commit();
            if (b + 1 < nbatch) setup(b + 1, cur ^ 1);  // read after the next batch's first barrier
            if (b >= 1 && b + 1 < nbatch && tid < MB) sPos[MB * (cur ^ 1) + tid] = posreg;  // batch b + 1
            // ---- forward transform (Eq. 4-5, 19): D[m] = [S0 | sqrt2 Re S1 | sqrt2 Im S1]
            if (!run_stage(false)) {
                ok = false;
                break;
            }
            if (b + 1 < nbatch) {  // the next batch's pixel loads go out now, and the positions of the one after
                prefetch(cur ^ 1);
                if (tid < MB && b + 2 < nbatch) posreg = member_pos(b + 2);
            }
            // ---- per 64-column chunk: tensor memory -> transposed FP32 buffer, Haar + threshold +
            //      inverse Haar per (group, coefficient) stream, FP16 into the inverse's operand.
            //      Chunk 0: S0 (columns 0..63); chunks 1, 2: complex coefficients c0 = 32 (ch - 1) .. + 31,
            //      real parts (columns 64 + c) as local columns 0..31, imaginary parts (128 + c) as 32..63.
            constexpr int NCHUNK = (C == 3) ? 3 : 1;
#pragma unroll 1
            for (int ch = 0; ch < NCHUNK; ++ch) {
                const bool cplx = ch >= 1;
                const int c0 = 32 * (ch - 1);
                const int col0 = !cplx ? 16 * wq : (wq < 2 ? 64 + c0 + 16 * wq : 128 + c0 + 16 * (wq - 2));
                {
                    uint32_t v[16];
                    tc::tmem_ld16(tbase + tlane + (uint32_t)col0, v);
                    tc::tmem_wait_ld();
                    const int m = 32 * q + lane;
#pragma unroll
                    for (int j = 0; j < 16; ++j) sT[(16 * wq + j) * TS + m] = __uint_as_float(v[j]);
                }
                __syncthreads();
                // 64 GPB streams (real) or half-streams (complex: lanes 2i, 2i + 1 hold the real and
                // imaginary part of one coefficient and exchange squares); whole warps take part
                for (int s2 = tid; s2 < 64 * GPB; s2 += NT) {
                    int col, g;
                    if (!cplx) {
                        col = s2 & 63;
                        g = s2 >> 6;
                    } else {
                        col = ((s2 >> 1) & 31) + 32 * (s2 & 1);
                        g = s2 >> 6;
                    }
                    const float tau = bTau[g];  // 0 for an empty slot: its zeros stay zeros
                    float *p = sT + col * TS + g * K;
                    float x[K];
#pragma unroll
                    for (int k = 0; k < K; k += 4) {
                        const float4 t4 = *reinterpret_cast<const float4 *>(p + k);
                        x[k] = t4.x;
                        x[k + 1] = t4.y;
                        x[k + 2] = t4.z;
                        x[k + 3] = t4.w;
                    }
                    haar_fwd_u<K>(x);
                    if (!cplx) {
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const int l = haar_level<K>(k);
                            // |x| >= tau 2^(l/2): tau times sqrt(2) for odd l, times 2^(l/2) exactly
                            const float tl = (l & 1) ? tau * (float)(1 << (l >> 1)) * 1.41421356237309505f
                                                     : tau * (float)(1 << (l >> 1));
                            x[k] = (fabsf(x[k]) >= tl) ? x[k] * (1.f / (float)(1 << l)) : 0.f;
                        }
                    } else {
                        // modulus test on squares: the streams hold sqrt2 Re and sqrt2 Im (F's rows), so
                        // |S| >= tau iff re^2 + im^2 >= 2 tau^2 2^l (lanes 2i, 2i + 1 hold the real and imaginary
                        // stream of one coefficient; the sum is formed in one order on both)
                        const bool im = s2 & 1;
                        const float tau2 = 2.f * tau * tau;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const int l = haar_level<K>(k);
                            const float sq = x[k] * x[k];
                            const float other = __shfl_xor_sync(0xffffffffu, sq, 1);
                            const float m2 = im ? (other + sq) : (sq + other);
                            x[k] = (m2 >= tau2 * (float)(1 << l)) ? x[k] * (1.f / (float)(1 << l)) : 0.f;
                        }
                    }
                    if (ra) x[0] = 0.f;  // Haar row 0 (Eq. 8 order): its refined value is added after the inverse
                    haar_inv_u<K>(x);
#pragma unroll
                    for (int k = 0; k < K; k += 4)
                        *reinterpret_cast<float4 *>(p + k) = make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
                }
                __syncthreads();
                // FP16 into the inverse GEMM's operand: member m, 8 consecutive local columns 8 jg ..
#pragma unroll
                for (int it = 0; it < MB * 8 / NT; ++it) {
                    const int e2 = it * NT + tid;
                    const int m = e2 & (MB - 1), jg = e2 >> 7;
                    const int gc = !cplx ? 8 * jg : (jg < 4 ? 64 + c0 + 8 * jg : 128 + c0 + 8 * (jg - 4));
                    __align__(16) __half hv[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) hv[e] = __float2half_rn(sT[(8 * jg + e) * TS + m]);
                    *reinterpret_cast<uint4 *>(sA + (gc >> 6) * (MB * 64) + cm_off(m, gc & 63)) =
                        *reinterpret_cast<const uint4 *>(hv);
                }
                tc::fence_before();
                __syncthreads();
            }
            // ---- inverse transform (Eq. 21 and the inverse channel DFT): D[m] = [R | G | B] pixels
            if (!run_stage(true)) {
                ok = false;
                break;
            }
            // ---- aggregation: member m = 32 q + lane, patch rows
            //      2 wq, 2 wq + 1
            {
                const int m = 32 * q + lane;
                const int pos = bPos[m];
                const int py = pos >= 0 ? pos / a.W : 0, px = pos >= 0 ? pos - py * a.W : 0;
                const float *mrow = nullptr;  // the member's group's refined mean patch (enhancement strategy)
                if (ra && pos >= 0) {
                    const int lg = b * GPB + m / K;
                    mrow = a.mean_est + (size_t)((gy0 + lg / a.tx) * a.nx + gx0 + lg % a.tx) * (C * 64);
                }
#pragma unroll 1
                for (int rr = 0; rr < 2; ++rr) {
                    const int row = 2 * wq + rr;
                    uint32_t p0[8], p1[8] = {}, p2[8] = {};
                    tc::tmem_ld8(tbase + tlane + (uint32_t)(row * 8), p0);
                    if constexpr (C == 3) {
                        tc::tmem_ld8(tbase + tlane + (uint32_t)(64 + row * 8), p1);
                        tc::tmem_ld8(tbase + tlane + (uint32_t)(128 + row * 8), p2);
                    }
                    tc::tmem_wait_ld();
                    if (pos < 0) continue;
                    float out[C][8];  // the inverse transform (F^T) gives the channels' pixels directly
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        out[0][v] = __uint_as_float(p0[v]);
                        if constexpr (C == 3) {
                            out[1][v] = __uint_as_float(p1[v]);
                            out[2][v] = __uint_as_float(p2[v]);
                        }
                    }
                    if (mrow) {  // first Haar row replaced (Eq. 24-25): the refined mean joins every member
#pragma unroll
                        for (int c = 0; c < C; ++c)
#pragma unroll
                            for (int v = 0; v < 8; ++v) out[c][v] += __ldg(mrow + c * 64 + row * 8 + v);
                    }
                    const int ly = py + row - ry0, lx = px - rx0;
                    if (ly >= 0 && ly < rh && lx >= 0 && lx + 7 < rw) {
                        const int o = ly * rw + lx;
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
#pragma unroll
                            for (int c = 0; c < C; ++c) atomicAdd(acc_v + c * RA + o + v, __float2int_rn(out[c][v] * 256.f));
                        }
                        if (row == 0) atomicAdd(acc_w + o, 1);  // the patch's origin: its 64 pixels' weight
                    } else {
                        atomicExch(&a.st->error, 1);
                    }
                }
            }
            tc::fence_before();
            __syncthreads();
        }
        if (!ok) break;
        // flush the tile's sums to the image-wide int64 sums and its origin counts to the image-wide ones
        // (k_normalize_box turns those into pixel weights)
        for (int e = tid; e < rh * rw; e += NT) {
            const int w = acc_w[e];
            const int yy = e / rw, xx = e - yy * rw;
            const size_t gpix = (size_t)(ry0 + yy) * a.W + (rx0 + xx);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int v = acc_v[c * RA + e];
                if (v == 0) continue;
                const long long s = (long long)v * 256ll;  // to the image-wide 2^16 scale
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + c * HW + gpix), (unsigned long long)s);
            }
            if (w != 0) atomicAdd(a.wcount + gpix, w);
        }
        __syncthreads();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

constexpr int NSHAPES_TC = 7;
constexpr int SHAPES_TC[NSHAPES_TC][2] = {{8, 8}, {4, 8}, {4, 4}, {2, 4}, {2, 2}, {1, 2}, {1, 1}};
// Relative time per batch of a tile of each shape (halo staging and flushing grow as tiles shrink),
// measured on the colour 512^2, 1024^2 and 3840x2160 workloads (8x8: 1, 4x4: 1.06, 2x4: 1.13).
constexpr double SHAPE_WEIGHT_TC[NSHAPES_TC] = {1.0, 1.02, 1.06, 1.13, 1.3, 1.6, 2.0};

// The tile shape of geometry g: among the shapes that fit, the one that minimises the rounds of tiles over
// the SMs x batches per tile x the shape's relative batch time (ties: the larger shape); ty = 0 if none fits.
// force >= 0: shape SHAPES_TC[force] where it fits (else the model's choice).
template <int C, int K>
void ftc_shape(const Geom &g, int nsm, int &ty, int &tx, int &rh, int &rw, size_t &need, int force = -1) {
    using L = FtcLayout<C>;
    const size_t budget = std::min((size_t)smem_optin(), (size_t)227 * 1024);
    need = 0;
    ty = tx = rh = rw = 0;
    double best = 0.0;
    if (force >= 0 && force < NSHAPES_TC) {
        const int h = std::min(g.H, (SHAPES_TC[force][0] - 1) * g.step + 2 * g.R + PS);
        const int w = std::min(g.W, (SHAPES_TC[force][1] - 1) * g.step + 2 * g.R + PS);
        const size_t n = L::acc_off + (size_t)(C + 1) * h * w * 4;
        if (n <= budget) {
            ty = SHAPES_TC[force][0];
            tx = SHAPES_TC[force][1];
            rh = h;
            rw = w;
            need = n;
            return;
        }
    }
    for (int i = 0; i < NSHAPES_TC; ++i) {
        const int h = std::min(g.H, (SHAPES_TC[i][0] - 1) * g.step + 2 * g.R + PS);
        const int w = std::min(g.W, (SHAPES_TC[i][1] - 1) * g.step + 2 * g.R + PS);
        const size_t n = L::acc_off + (size_t)(C + 1) * h * w * 4;
        if (n > budget) continue;
        const long long ntiles = (long long)((g.ny + SHAPES_TC[i][0] - 1) / SHAPES_TC[i][0]) *
                                 ((g.nx + SHAPES_TC[i][1] - 1) / SHAPES_TC[i][1]);
        const int nb = (SHAPES_TC[i][0] * SHAPES_TC[i][1] * K + MB - 1) / MB;
        const double cost = (double)((ntiles + nsm - 1) / nsm) * nb * SHAPE_WEIGHT_TC[i];
        if (ty == 0 || cost < best) {
            best = cost;
            ty = SHAPES_TC[i][0];
            tx = SHAPES_TC[i][1];
            rh = h;
            rw = w;
            need = n;
        }
    }
}

template <int C, int K>
hts_status launch_ftc(FtcArgs a, const Geom &g, cudaStream_t s, bool *used) {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    size_t need = 0;
    int ty = 0, tx = 0, rh = 0, rw = 0;
    ftc_shape<C, K>(g, nsm, ty, tx, rh, rw, need);
    *used = false;
    if (ty == 0) return HTS_OK;  // the window is too large for a tile: the SIMT filter takes it
    const void *k = reinterpret_cast<const void *>(k_filter_tc<C, K, false>);
    const hts_status st = allow_smem(k, need);
    if (st != HTS_OK) return st;
    a.ty = ty;
    a.tx = tx;
    a.nty = (g.ny + ty - 1) / ty;
    a.ntx = (g.nx + tx - 1) / tx;
    a.ntiles = a.nty * a.ntx;
    a.rh_max = rh;
    a.rw_max = rw;
    const int grid = std::max(1, std::min(a.ntiles, nsm));
    const FtcBatch none{};
    {
        KTimer kt("k_filter_tc", s);
        k_filter_tc<C, K, false><<<grid, NT, need, s>>>(a, none);
    }
    *used = true;
    return check_launch("k_filter_tc");
}

template <int C, int K>
hts_status launch_ftc_batch(const FtcBatch &bt, int grid, cudaStream_t s) {
    using L = FtcLayout<C>;
    const size_t need = L::acc_off + (size_t)(C + 1) * bt.rh_max * bt.rw_max * 4;
    const void *k = reinterpret_cast<const void *>(k_filter_tc<C, K, true>);
    const hts_status st = allow_smem(k, need);
    if (st != HTS_OK) return st;
    const FtcArgs none{};
    {
        KTimer kt("k_filter_tc", s);
        k_filter_tc<C, K, true><<<grid, NT, need, s>>>(none, bt);
    }
    return check_launch("k_filter_tc");
}

}  // namespace

size_t filter_tc_job_size() { return sizeof(FtcArgs); }

int filter_tc_job(const float *img, const Geom &g, const int32_t *idx, const float *b32, long long *acc, int *wcount,
                  DevState *st, const float *sigma_ref, int map_judged, double tau_scale, int nsm, void *job,
                  int force_shape) {
    FtcArgs a{};
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.ny = g.ny;
    a.idx = idx;
    a.b32 = b32;
    a.acc = acc;
    a.wcount = wcount;
    a.sigma_ref = sigma_ref;
    a.map_judged = map_judged;
    a.tau_scale = tau_scale;
    a.mean_est = nullptr;
    a.st = st;
    size_t need = 0;
    int ty = 0, tx = 0, rh = 0, rw = 0;
#define HTS_FTC_SHAPE(CC, KK) \
    if (g.C == CC && g.K == KK) ftc_shape<CC, KK>(g, nsm, ty, tx, rh, rw, need, force_shape);
    HTS_FTC_SHAPE(1, 8) HTS_FTC_SHAPE(1, 16) HTS_FTC_SHAPE(1, 32) HTS_FTC_SHAPE(3, 8) HTS_FTC_SHAPE(3, 16)
    HTS_FTC_SHAPE(3, 32)
#undef HTS_FTC_SHAPE
    if (ty == 0) return -1;  // not for the tensor-core filter
    a.ty = ty;
    a.tx = tx;
    a.nty = (g.ny + ty - 1) / ty;
    a.ntx = (g.nx + tx - 1) / tx;
    a.ntiles = a.nty * a.ntx;
    a.rh_max = rh;
    a.rw_max = rw;
    std::memcpy(job, &a, sizeof(FtcArgs));
    return a.ntiles;
}

hts_status launch_filter_tc_batch(int C, int K, const void *jobs_host, const void *jobs_dev, const int *tile_start_dev,
                                  int njobs, int ntiles, int grid, cudaStream_t s) {
    FtcBatch bt{};
    bt.jobs = static_cast<const FtcArgs *>(jobs_dev);
    bt.tile_start = tile_start_dev;
    bt.njobs = njobs;
    bt.ntiles = ntiles;
    const FtcArgs *jh = static_cast<const FtcArgs *>(jobs_host);
    int area = 0;
    for (int j = 0; j < njobs; ++j)
        if (jh[j].rh_max * jh[j].rw_max > area) {
            area = jh[j].rh_max * jh[j].rw_max;
            bt.rh_max = jh[j].rh_max;
            bt.rw_max = jh[j].rw_max;
        }
    grid = std::max(1, std::min(grid, ntiles));
#define HTS_FTC_BATCH(CC, KK) \
    if (C == CC && K == KK) return launch_ftc_batch<CC, KK>(bt, grid, s);
    HTS_FTC_BATCH(1, 8) HTS_FTC_BATCH(1, 16) HTS_FTC_BATCH(1, 32) HTS_FTC_BATCH(3, 8) HTS_FTC_BATCH(3, 16)
    HTS_FTC_BATCH(3, 32)
#undef HTS_FTC_BATCH
    return HTS_EUNSUPPORTED;
}

hts_status launch_filter_tc(const float *img, const Geom &g, const int32_t *idx, const float *b32, long long *acc,
                            int *wcount, DevState *st, const float *sigma_ref, int map_judged, double tau_scale,
                            const float *mean_est, cudaStream_t s, bool *used) {
    *used = false;
    FtcArgs a{};
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.ny = g.ny;
    a.idx = idx;
    a.b32 = b32;
    a.acc = acc;
    a.wcount = wcount;
    a.sigma_ref = sigma_ref;
    a.map_judged = map_judged;
    a.tau_scale = tau_scale;
    a.mean_est = mean_est;
    a.st = st;
#define HTS_FTC_CASE(CC, KK) \
    if (g.C == CC && g.K == KK) return launch_ftc<CC, KK>(a, g, s, used);
    HTS_FTC_CASE(1, 8) HTS_FTC_CASE(1, 16) HTS_FTC_CASE(1, 32) HTS_FTC_CASE(3, 8) HTS_FTC_CASE(3, 16)
    HTS_FTC_CASE(3, 32)
#undef HTS_FTC_CASE
    return HTS_OK;  // other group sizes: the SIMT filter
}

}  // namespace hts
