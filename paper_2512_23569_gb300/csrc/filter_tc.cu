// Collaborative filtering of the precision form on the sm_103a tensor cores
// (Eq. 19-21, Alg. 1 steps 2-3), FP32 threshold decisions.
//
// The unitary DFT along the channels (Eq. 4-5), in its real orthonormal form
// [P^(1) | sqrt2 Re P^(2) | sqrt2 Im P^(2)] (slice 3 is the conjugate of
// slice 2), is applied to the gathered pixels in FP32 registers.  The
// separable projection Shat = U^H Phat V of each slice (Eq. 19) is then one
// real orthogonal matrix per slice: F0 (64 x 64) for the real slice 1 and,
// for colour, F1 (128 x 128, the real form [[Re M, -Im M], [Im M, Re M]] of
// the unitary M = conj(U) (x) V of the complex slice 2), giving
// [S^(1) | sqrt2 Re S^(2) | sqrt2 Im S^(2)].  The Haar transform along the
// group axis (Eq. 8) acts on the members, the DFT and F on each member's
// pixels: they commute, so the kernel applies the DFT and Haar first, in
// FP32 registers (a thread holds one pixel of all the group's members), and
// two GEMMs then give the 3-D coefficients: with the 128 Haar rows of a
// batch (8 groups of K = 16) as the MMA's M, D[row][coefficient] =
// sum_pixel A[row][pixel] F[coefficient][pixel] per slice, FP16 operands,
// FP32 accumulation in tensor memory (tcgen05.mma kind::f16, N = 64 and
// 128).  A thread per row thresholds its coefficients in place (Eq. 20; the
// complex slice's real and imaginary parts lie in the same row) and writes
// them as the inverse GEMMs' operand; the inverse (Eq. 21) is F0^T and F1^T,
// the same shared-memory matrices read with the transpose bit (MN-major),
// giving each Haar row's slice values.  One transposed pass per slice hands
// a (group, pixel) pair to a thread, which applies the inverse Haar along
// the group and adds the members' estimates to the tile's sums of that
// slice; slice 1's pass runs while the tensor cores compute slice 2's
// inverse.  The sums are kept per slice, and the inverse channel DFT is
// applied once per pixel when they are normalised (k_normalize_box): the
// aggregation and the DFT are both linear.
//
// FP16 rather than BF16: pixels lie in a bounded range and the bases are
// orthonormal, so FP16's 11-bit significand fits the data, where BF16's 8
// bits would put a rounding error of up to one grey level on the input.
//
// Aggregation: fixed-point integer sums (value * 2^8, rounded) of the
// estimates in 32-bit shared-memory accumulators over the tile's region
// (at most 2^10 members of a tile cover a pixel: no overflow), flushed to
// the image-wide int64 sums (2^16 scale) once per tile; integer sums do not
// depend on the order of the additions, so the result is deterministic.  A
// warp adds 4 rows x 8 pixels of one member's patch, in 32 distinct banks
// (row stride 8 mod 32).  Weights: every member adds 1 to the count of its
// patch origin (top-left pixel) instead of 1 to each of its 64 pixels; a
// pixel's weight is the sum of the origin counts over the 8 x 8 origins whose
// patch covers it, formed by k_normalize_box.  The MMA waits are bounded: a
// wait that gives up records DevState.error = 2, waits (bounded) for the
// MMAs, frees the tensor memory and leaves.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "filter_common.h"
#include "hts_internal.h"
#include "tc_ptx.h"

namespace hts {
namespace {

using fc::K3F;
using fc::K23F;
constexpr float K12F = fc::R2F;

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

constexpr int NT = 512;   // 16 warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31, column quarter w / 4
constexpr int MB = 128;   // Haar rows per batch (8 groups of K = 16) = MMA M
constexpr int TS = MB + 4;  // row stride (floats) of the transposed buffer: conflict-free float4 reads
constexpr long long SPIN = 1ll << 24;

// The row operands of the two GEMMs (forward: the groups' Haar rows of raw pixels, inverse: the thresholded
// coefficients), FP16, K-major without swizzle: core matrices of 8 rows x 8 columns (128 B); adjacent core
// matrices along K 144 B apart (16 B of padding, so that the four core matrices a warp's 32 consecutive
// columns touch fall in distinct banks), 8-row groups 8 x 144 B apart, 64-column blocks of 128 rows.
constexpr int LBO_A = 144;
constexpr int SBO_A = 8 * LBO_A;
constexpr int BLK_A = 16 * SBO_A;

// Byte offset of element (row r, column k) of a row operand.
__device__ __forceinline__ int a_off(int r, int k) {
    return (k >> 6) * BLK_A + (r >> 3) * SBO_A + ((k & 63) >> 3) * LBO_A + ((r & 7) << 4) + ((k & 7) << 1);
}

// Row stride (elements) of the tile's staged region (FP16) and shared sums (int32): the region width rounded
// up to 8 mod 64.  A warp reads or adds to 4 rows x 8 pixels of one patch: in the region four 16-byte row
// pieces whose starts are 16 B apart modulo the banks' 128 bytes, in the sums four 32-byte row pieces 32 B
// apart: distinct banks.
__host__ __device__ constexpr int acc_stride(int rw) { return rw + ((8 - rw) & 63); }

// Fixed-point value * 2^8 rounded to the nearest integer (ties to even), as __float2int_rn(v * 256), for the
// range the tile's 32-bit sums hold (|v| < 2^13; values beyond it are clamped): v * 256 + 1.5 * 2^23 lies in
// [2^23, 2^24), where FP32 spacing is 1, so the fused multiply-add rounds once to the integer and leaves it in
// the low mantissa bits.
__device__ __forceinline__ int fix8(float v) {
    v = fminf(fmaxf(v, -8191.f), 8191.f);
    return __float_as_int(fmaf(v, 256.f, 12582912.f)) - 0x4B400000;
}

template <int C>
struct FtcLayout {
    // The FP16 transforms F0 [coefficient][pixel] (64 x 64) and, for colour, F1 (128 x 128) right after it,
    // K-major, core matrices of 8 rows x 8 columns, 8-column groups 128 B apart along K and 8-row groups
    // (64 or 128) * 16 B apart: the forward GEMMs' B operands, and with the transpose bit (K = coefficients,
    // N = pixels, MN-major) the inverse's.
    static constexpr int F0_HALVES = 64 * 64;
    static constexpr int B_HALVES = (C == 3) ? F0_HALVES + 128 * 128 : F0_HALVES;
    static constexpr size_t a_bytes = (size_t)C * BLK_A;  // the row operand
    static constexpr size_t a_off = 0;
    static constexpr size_t t_off = a_off + a_bytes;  // the transposed FP32 buffer [64][TS] of one slice
    static constexpr size_t b_off = t_off + (size_t)64 * TS * 4;
    static constexpr size_t basis_off = b_off + (size_t)B_HALVES * 2;  // 6 x 64 FP32
    static constexpr size_t misc_off = basis_off + (size_t)6 * 64 * 4;
    // misc: tau[2][32] float, off[2][MB] int, 4 mbarrier words (forward; inverse of slice 1; inverse of
    // slices 2-3), tensor-memory slot
    static constexpr size_t job_off = misc_off + (size_t)2 * 32 * 4 + 2 * MB * 4 + 32 + 16;
    // then the tile's sums [C][RA] int32 (per slice) and its staged region [C][RA] FP16 (per channel; RA =
    // rows x acc_stride(width))
    static constexpr size_t acc_off = job_off + 256;
    static constexpr size_t bytes(int rh, int rw) { return acc_off + (size_t)C * rh * acc_stride(rw) * 6; }
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
//
// Per batch of MB Haar rows (GPB = MB / K groups):
//  1. gather: a thread holds, for one (group, pixel) pair, that pixel of the group's K members (for K = 32
//     two threads hold 16 members each), applies the channel DFT and the unnormalised Haar transform along
//     the group axis in FP32 registers and writes the K Haar rows' slice values to the row operand (FP16);
//  2. forward GEMMs: D[row][coefficient] = sum_pixel A[row][pixel] F[coefficient][pixel] per slice
//     (tensor memory);
//  3. threshold: a thread per row (tensor-memory lane) keeps or drops its coefficients against the level's
//     threshold (modulus for the complex slice, both parts in the same lane), rescales the kept ones by
//     2^-l and writes them as the inverse GEMMs' row operand (FP16);
//  4. inverse GEMMs with F0^T, then F1^T (two commits): the rows' slice values, still in the Haar domain;
//  5. per slice, once its inverse has completed: tensor memory -> transposed FP32 buffer; a thread per
//     (group, pixel) pair applies the unnormalised inverse Haar and adds the K members' estimates of that
//     pixel to the tile's sums of the slice.
template <int C, int K, bool BATCH>
__global__ void __launch_bounds__(NT, 1) k_filter_tc(const __grid_constant__ FtcArgs a0,
                                                     const __grid_constant__ FtcBatch bt) {
    using L = FtcLayout<C>;
    static_assert(sizeof(FtcArgs) <= 256, "the job fits its shared-memory slot");
    constexpr int GPB = MB / K;                 // groups per batch
    constexpr int KM = K < 16 ? K : 16;         // members a thread holds per (group, pixel) pair
    constexpr int TPP = K / KM;                 // threads per pair
    constexpr int PPT = GPB * 64 * TPP / NT;    // pairs per thread
    static_assert(PPT * NT == GPB * 64 * TPP && TPP <= 2, "pairs cover the threads");
    constexpr int LOGK = (K == 8) ? 3 : (K == 16) ? 4 : 5;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem + L::a_off;
    float *sT = reinterpret_cast<float *>(smem + L::t_off);
    __half *sB = reinterpret_cast<__half *>(smem + L::b_off);
    float *sBas = reinterpret_cast<float *>(smem + L::basis_off);
    float *sTau = reinterpret_cast<float *>(smem + L::misc_off);  // [2][32] groups' thresholds
    int *sOff = reinterpret_cast<int *>(sTau + 64);  // [2][MB] members' patch origins in the tile region (-1: none)
    uint64_t *bar = reinterpret_cast<uint64_t *>(sOff + 2 * MB);  // [3], 8-byte aligned
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 4);
    int *accs = reinterpret_cast<int *>(smem + L::acc_off);
    FtcArgs *sjob = reinterpret_cast<FtcArgs *>(smem + L::job_off);
    const FtcArgs &a = BATCH ? *sjob : a0;  // the current job's arguments
    const int RA = BATCH ? bt.rh_max * acc_stride(bt.rw_max) : a0.rh_max * acc_stride(a0.rw_max);
    int *acc_v = accs;                                         // [C][RA] the tile's sums of value * 2^8
    __half *sReg = reinterpret_cast<__half *>(accs + C * RA);  // [C][RA] the tile's region, FP16
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---- bases (row-major 8x8, element (r, c) at r * 8 + c) and the transform F of the current job
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
        // F0[(a, b)][(i, j)] = U0[i][a] V0[j][b] (S^(1) = U0^T P^(1) V0, Eq. 19).  Colour, F1: with M = conj(U1[i][a])
        // V1[j][b] = Mr + i Mi, rows Re S^(2) then Im S^(2), columns Re P^(2) then Im P^(2) (both sides times
        // sqrt2): F1 = [[Mr, -Mi], [Mi, Mr]].
        for (int e = tid; e < L::B_HALVES; e += NT) {
            int n, k, idx;
            float f;
            if (e < L::F0_HALVES) {
                n = e >> 6;
                k = e & 63;
                f = sBas[(k >> 3) * 8 + (n >> 3)] * sBas[64 + (k & 7) * 8 + (n & 7)];
                idx = (((n >> 3) * 8 + (k >> 3)) << 6) + ((n & 7) << 3) + (k & 7);
            } else {
                const int e1 = e - L::F0_HALVES;
                n = e1 >> 7;
                k = e1 & 127;
                const int nc = n & 63, px = k & 63;
                const int ia = (px >> 3) * 8 + (nc >> 3), jb = (px & 7) * 8 + (nc & 7);
                const float ur = sBas[128 + ia], ui = sBas[192 + ia], vr = sBas[256 + jb], vi = sBas[320 + jb];
                const float mr = ur * vr + ui * vi, mi = ur * vi - ui * vr;
                f = (n < 64) ? ((k < 64) ? mr : -mi) : ((k < 64) ? mi : mr);
                idx = L::F0_HALVES + (((n >> 3) * 16 + (k >> 3)) << 6) + ((n & 7) << 3) + (k & 7);
            }
            sB[idx] = __float2half_rn(f);
        }
    };
    if (!BATCH) build_f();
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) tc::bar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(slot, L::tcols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idf0 = tc::idesc_f16(MB, 64, false), idf1 = tc::idesc_f16(MB, 128, false);  // B K-major
    const uint32_t idi0 = idf0 | (1u << 16), idi1 = idf1 | (1u << 16);  // inverse: B transposed (MN-major)
    const int q = warp & 3, wq = warp >> 2;  // tensor-memory lane quarter, column quarter
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    uint32_t phase = 0;  // parity of the batches done: every barrier completes once per batch
    bool ok = true;

    // A K step kk of the row operand: columns 16 kk .. 16 kk + 15, two core matrices at (kk % 4) * 2 * LBO_A
    // in 64-column block kk / 4.
    auto a_desc = [&](uint32_t a0, int kk) { return tc::sdesc(a0 + (kk >> 2) * BLK_A + (kk & 3) * 2 * LBO_A, LBO_A, SBO_A); };
    // Issues the MMAs of the forward GEMMs (commit on bar[0]) or of the inverse ones (slice 1's commit on
    // bar[1], then slices 2-3's on bar[2]), after every thread's shared-memory writes; thread 0 only.
    // Forward B = F: K = pixels, core matrices 128 B apart along K, (64 or 128) * 16 B along N (coefficients).
    // Inverse B = F^T read in place: K = coefficients ((64 or 128) * 16 B apart: LBO), N = pixels (128 B
    // apart: SBO), the MN-major convention.
    auto issue = [&](bool inverse) {
        tc::fence_after();
        const uint32_t a0 = tc::su32(sA), f0 = tc::su32(sB), f1 = f0 + L::F0_HALVES * 2;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = inverse ? tc::sdesc(f0 + kk * 2 * 1024, 1024, 128) : tc::sdesc(f0 + kk * 256, 128, 1024);
            tc::mma_f16(tbase, a_desc(a0, kk), bd, inverse ? idi0 : idf0, kk > 0 ? 1u : 0u);
        }
        if (inverse) tc::mma_commit(&bar[1]);
        if constexpr (C == 3) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const uint64_t bd =
                    inverse ? tc::sdesc(f1 + kk * 2 * 2048, 2048, 128) : tc::sdesc(f1 + kk * 256, 128, 2048);
                tc::mma_f16(tbase + 64, a_desc(a0, 4 + kk), bd, inverse ? idi1 : idf1, kk > 0 ? 1u : 0u);
            }
            if (inverse) tc::mma_commit(&bar[2]);
        }
        if (!inverse) tc::mma_commit(&bar[0]);
    };
    // Every thread: the row operand written, then thread 0 issues the GEMMs.
    auto launch_stage = [&](bool inverse) {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) issue(inverse);
    };
    // Waits for barrier i of this batch; false (error 2 recorded) if the wait gave up, after thread 0 has
    // waited (bounded) for every MMA this batch issued, so that the memory can be released.
    auto wait_bar = [&](int i) -> bool {
        const bool done = tc::bar_wait(&bar[i], phase, SPIN);
        if (__syncthreads_or(!done)) {
            if (tid == 0) {
                for (int j = i; j < (i == 0 ? 1 : (C == 3 ? 3 : 2)); ++j) tc::bar_wait(&bar[j], phase, SPIN);
                atomicExch(&a.st->error, 2);
            }
            return false;
        }
        tc::fence_after();
        return true;
    };

    // pair slot i of this thread: group g, pixel p (patch row p >> 3, column p & 7), half h of the group's
    // members (K = 32).  A warp covers 32 consecutive pixels of one group (4 patch rows: 4 coalesced 32-byte
    // segments per member); for K = 32 16 pixels of both halves, the partner half in lane ^ 16.
    auto slot_of = [&](int i, int &g, int &p, int &h) {
        const int s = tid + i * NT;
        int pair;
        if (TPP == 1) {
            pair = s;
            h = 0;
        } else {
            h = (s >> 4) & 1;
            pair = ((s >> 5) << 4) | (s & 15);
        }
        g = pair >> 6;
        p = pair & 63;
    };
    // Haar row (Eq. 8 order) of local row r of half h when two threads share a group (K = 32): after the
    // exchange of the halves' sums row 0 of half 0 is global row 0, of half 1 global row 1; local detail rows
    // of level size n (r in [n, 2n)) go to global rows 2n + h n + (r - n).
    auto grow = [](int r, int h) -> int {
        if (TPP == 1) return r;
        if (r == 0) return h;
        const int n = r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1;
        return 2 * n + h * n + (r - n);
    };

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
        const int rh = ry1 - ry0 + 1, rw = rx1 - rx0 + 1, rwp = acc_stride(rw);
        const int RP = rh * rwp;  // elements per channel plane of the region and of the sums
        for (int e = tid; e < C * RP; e += NT) acc_v[e] = 0;
        // the tile's region, FP16: row y of channel c at (c * rh + y) * rwp; consecutive threads take consecutive
        // pixels of a row, eight loads in flight per thread
        {
            // element e = tid + i NT: column x, region row `row` = channel c, row y; advanced by NT per step
            const int dq = NT / rw, dr = NT - dq * rw;
            int row = tid / rw, x = tid - row * rw;
            int c = row / rh, y = row - c * rh;
            for (int e0 = 0; e0 < C * rh * rw; e0 += 8 * NT) {
                float v[8];
                int d[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool in = c < C;
                    d[i] = in ? row * rwp + x : -1;
                    v[i] = in ? __ldg(a.img + c * HW + (size_t)(ry0 + y) * a.W + rx0 + x) : 0.f;
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
                    if (d[i] >= 0) sReg[d[i]] = __float2half_rn(v[i]);
            }
        }
        // the block's next tile's region into L2 while this tile runs (its staging then reads L2, not HBM):
        // per channel and row, one address every 128 bytes from the first column, and the last column
        if (!BATCH && gt + (int)gridDim.x < total) {
            const int nt = gt + (int)gridDim.x;
            const int nyi = nt / a.ntx, nxi = nt - nyi * a.ntx;
            const int ngy0 = nyi * a.ty, ngx0 = nxi * a.tx;
            const int ngy1 = min(a.ny, ngy0 + a.ty) - 1, ngx1 = min(a.nx, ngx0 + a.tx) - 1;
            const int py0 = max(0, grid_pos(ngy0, a.H, a.step) - a.R);
            const int py1 = min(a.H - 1, grid_pos(ngy1, a.H, a.step) + a.R + PS - 1);
            const int px0 = max(0, grid_pos(ngx0, a.W, a.step) - a.R);
            const int px1 = min(a.W - 1, grid_pos(ngx1, a.W, a.step) + a.R + PS - 1);
            const int nl = (px1 - px0) / 32 + 2, prow = py1 - py0 + 1;
            for (int e = tid; e < C * prow * nl; e += NT) {
                const int c = e / (prow * nl), rem = e - c * (prow * nl), y = rem / nl, l = rem - y * nl;
                const int x = min(px0 + 32 * l, px1);
                tc::prefetch_l2(a.img + c * HW + (size_t)(py0 + y) * a.W + x);
            }
        }
        // group tid (< GPB) of batch bb: its noise level (the map's, else 1), loaded a batch ahead of its use
        // (nothing reads the loaded value until then: no wait), and whether the slot holds a group
        const float tau_all = use_map ? 0.f : a.st->tau32;
        auto sig_of = [&](int bb, bool &valid) -> float {
            const int lg = bb * GPB + tid;
            const int gy = gy0 + lg / a.tx, gx = gx0 + lg % a.tx;
            valid = lg < gpt && gy <= gy1 && gx <= gx1;
            return use_map ? __ldg(a.sigma_ref + (valid ? gy * a.nx + gx : 0)) : 1.f;
        };
        auto tau_from = [&](float sig, bool valid) -> float {
            return !valid ? 0.f : use_map ? (float)(a.tau_scale * (double)sig) : tau_all;
        };
        // member m (= tid < MB) of batch bb: its patch's top-left pixel (loaded; read a batch later) and
        // whether the slot holds a group
        auto member_pos = [&](int bb, bool &valid) -> int {
            const int g = tid / K, k = tid - g * K;
            const int lg = bb * GPB + g;
            const int gy = gy0 + lg / a.tx, gx = gx0 + lg % a.tx;
            valid = lg < gpt && gy <= gy1 && gx <= gx1;
            return __ldg(a.idx + (size_t)(valid ? gy * a.nx + gx : 0) * K + k);
        };
        // member tid (< MB) at pixel pos into buffer buf: its patch origin in the region (-1: empty slot), and
        // its origin count (the weight of the patch's 64 pixels, formed by k_normalize_box)
        auto member_off = [&](int pos, int buf) {
            int o = -1;
            if (pos >= 0) {
                const int py = pos / a.W, px = pos - py * a.W;
                const int ly = py - ry0, lx = px - rx0;
                if (ly >= 0 && ly + PS <= rh && lx >= 0 && lx + PS <= rw) {
                    o = ly * rwp + lx;
                    atomicAdd(a.wcount + pos, 1);
                } else {
                    atomicExch(&a.st->error, 1);
                }
            }
            sOff[MB * buf + tid] = o;
        };
        // the batch's pixels (offsets in buffer buf) from the staged region, Haar along the group axis (Eq. 8,
        // unnormalised) in FP32, FP16 rows of the operand
        auto commit = [&](int buf) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                int g, p, h;
                slot_of(i, g, p, h);
                const int *offs = sOff + MB * buf + g * K + h * KM;
                const __half *src = sReg + (p >> 3) * rwp + (p & 7);
                float v[KM][C];
#pragma unroll
                for (int j = 0; j < KM; ++j) {
                    const int o = offs[j];
                    const bool in = o >= 0 && HTS_IN_BOUNDS(o + (p >> 3) * rwp + (p & 7) < RP, &a.st->error);
#pragma unroll
                    for (int c = 0; c < C; ++c) v[j][c] = in ? __half2float(src[c * RP + o]) : 0.f;
                }
                if constexpr (C == 3) {  // the channel DFT (Eq. 4-5), real orthonormal form: v[j][s] = slice value s
#pragma unroll
                    for (int j = 0; j < KM; ++j) {
                        const float r = v[j][0], gb = v[j][1] + v[j][2], d = v[j][2] - v[j][1];
                        v[j][0] = K3F * (r + gb);
                        v[j][1] = K23F * fmaf(-0.5f, gb, r);
                        v[j][2] = K12F * d;
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float x[KM];
#pragma unroll
                    for (int j = 0; j < KM; ++j) x[j] = v[j][c];
                    haar_fwd_u<KM>(x);
                    if (TPP == 2) {  // the top level across the halves: sum and difference of their sums
                        const float o = __shfl_xor_sync(0xffffffffu, x[0], 16);
                        x[0] = h ? (o - x[0]) : (x[0] + o);
                    }
                    unsigned char *col = sA + a_off(g * K, c * 64 + p);
#pragma unroll
                    for (int r = 0; r < KM; ++r) {
                        const int row = grow(r, h);  // within the group: g * K + row, whose 8-row groups are SBO_A apart
                        *reinterpret_cast<__half *>(col + (row >> 3) * SBO_A + ((row & 7) << 4)) = __float2half_rn(x[r]);
                    }
                }
            }
        };
        int posreg = -1;
        float sigreg = 0.f;
        bool pvalid = false, svalid = false;
        if (tid < GPB) {
            const float s0 = sig_of(0, svalid);
            sTau[tid] = tau_from(s0, svalid);
            if (nbatch > 1) sigreg = sig_of(1, svalid);
        }
        if (tid < MB) {
            const int p0 = member_pos(0, pvalid);
            member_off(pvalid ? p0 : -1, 0);
            if (nbatch > 1) posreg = member_pos(1, pvalid);
        }
        __syncthreads();
        for (int b = 0; b < nbatch; ++b) {
            const int cur = b & 1;
            const float *bTau = sTau + 32 * cur;
            commit(cur);
            if (b + 1 < nbatch) {  // the next batch's thresholds and member offsets (read after the next barrier)
                if (tid < GPB) sTau[32 * (cur ^ 1) + tid] = tau_from(sigreg, svalid);
                if (tid < MB) member_off(pvalid ? posreg : -1, cur ^ 1);
            }
            // ---- forward transform (Eq. 19) of the Haar rows: D[row] = [S0 | sqrt2 Re S1 | sqrt2 Im S1]
            launch_stage(false);
            if (!wait_bar(0)) {
                ok = false;
                break;
            }
            if (b + 2 < nbatch) {  // the positions and noise levels of the batch after next
                if (tid < MB) posreg = member_pos(b + 2, pvalid);
                if (tid < GPB) sigreg = sig_of(b + 2, svalid);
            }
            // ---- hard threshold (Eq. 20) of row m = 32 q + lane: Haar row k of group m / K, level l_k.  The
            //      unnormalised coefficient is 2^(l/2) times the orthonormal one, so it is kept iff x^2 >= tau^2 2^l
            //      (complex: (sqrt2 Re)^2 + (sqrt2 Im)^2 >= 2 tau^2 2^l); kept ones are scaled by 2^-l (exact).
            {
                const int m = 32 * q + lane;
                const int k = m & (K - 1);
                const int l = k == 0 ? LOGK : LOGK - (31 - __clz(k));
                const float tau = bTau[m / K];  // 0 for an empty slot: its zeros stay zeros
                const float t2 = tau * tau * (float)(1 << l);
                const float sc = (ra && k == 0) ? 0.f : __int_as_float((127 - l) << 23);  // 2^-l; RA: row 0 replaced
                unsigned char *rowp = sA + (m >> 3) * SBO_A + ((m & 7) << 4);
                {
                    uint32_t v[16];
                    tc::tmem_ld16(tbase + tlane + (uint32_t)(16 * wq), v);
                    tc::tmem_wait_ld();
                    __align__(16) __half2 hv[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float x0 = __uint_as_float(v[2 * j]), x1 = __uint_as_float(v[2 * j + 1]);
                        hv[j] = __floats2half2_rn(x0 * x0 >= t2 ? x0 * sc : 0.f, x1 * x1 >= t2 ? x1 * sc : 0.f);
                    }
                    const uint4 *hp = reinterpret_cast<const uint4 *>(hv);
                    *reinterpret_cast<uint4 *>(rowp + (2 * wq) * LBO_A) = hp[0];
                    *reinterpret_cast<uint4 *>(rowp + (2 * wq + 1) * LBO_A) = hp[1];
                }
                if constexpr (C == 3) {
                    uint32_t vr[16], vi[16];
                    tc::tmem_ld16(tbase + tlane + (uint32_t)(64 + 16 * wq), vr);
                    tc::tmem_ld16(tbase + tlane + (uint32_t)(128 + 16 * wq), vi);
                    tc::tmem_wait_ld();
                    const float t2c = 2.f * t2;
                    __align__(16) __half2 hr[8], hi[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float o[2][2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float re = __uint_as_float(vr[2 * j + e]), im = __uint_as_float(vi[2 * j + e]);
                            const bool keep = fmaf(re, re, im * im) >= t2c;
                            o[0][e] = keep ? re * sc : 0.f;
                            o[1][e] = keep ? im * sc : 0.f;
                        }
                        hr[j] = __floats2half2_rn(o[0][0], o[0][1]);
                        hi[j] = __floats2half2_rn(o[1][0], o[1][1]);
                    }
                    const uint4 *rp = reinterpret_cast<const uint4 *>(hr);
                    const uint4 *ip = reinterpret_cast<const uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(rowp + BLK_A + (2 * wq) * LBO_A) = rp[0];
                    *reinterpret_cast<uint4 *>(rowp + BLK_A + (2 * wq + 1) * LBO_A) = rp[1];
                    *reinterpret_cast<uint4 *>(rowp + 2 * BLK_A + (2 * wq) * LBO_A) = ip[0];
                    *reinterpret_cast<uint4 *>(rowp + 2 * BLK_A + (2 * wq + 1) * LBO_A) = ip[1];
                }
            }
            // ---- inverse transform (Eq. 21): E[row] = the slices' values of the group's thresholded Haar rows,
            //      slice 1 first (its own commit), so that its aggregation overlaps the rest
            launch_stage(true);
            // ---- per slice: inverse Haar along the group axis and aggregation of the members' estimates
            int offs[PPT][KM];  // this thread's members' patch origins in the region (-1: empty slot)
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                int g, p, h;
                slot_of(i, g, p, h);
#pragma unroll
                for (int j = 0; j < KM; ++j) {
                    const int o = sOff[MB * cur + g * K + h * KM + j];
                    offs[i][j] = o >= 0 ? o + (p >> 3) * rwp + (p & 7) : -1;
                }
            }
#pragma unroll 1
            for (int c = 0; c < C; ++c) {
                if (c < 2 && !wait_bar(1 + c)) {  // slice c's inverse has completed (slices 2 and 3 together)
                    ok = false;
                    break;
                }
                {
                    uint32_t v[16];
                    tc::tmem_ld16(tbase + tlane + (uint32_t)(64 * c + 16 * wq), v);
                    tc::tmem_wait_ld();
                    const int m = 32 * q + lane;
#pragma unroll
                    for (int j = 0; j < 16; ++j) sT[(16 * wq + j) * TS + m] = __uint_as_float(v[j]);
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < PPT; ++i) {
                    int g, p, h;
                    slot_of(i, g, p, h);
                    const float *colp = sT + p * TS + g * K;
                    float x[KM];
                    if (TPP == 1) {
#pragma unroll
                        for (int r = 0; r < KM; r += 4) {
                            const float4 t4 = *reinterpret_cast<const float4 *>(colp + r);
                            x[r] = t4.x;
                            x[r + 1] = t4.y;
                            x[r + 2] = t4.z;
                            x[r + 3] = t4.w;
                        }
                    } else {
                        const float2 z = *reinterpret_cast<const float2 *>(colp);
                        x[0] = h ? (z.x - z.y) : (z.x + z.y);  // the top level: this half's sum
                        x[1] = colp[grow(1, h)];
                        const float2 u = *reinterpret_cast<const float2 *>(colp + grow(2, h));
                        x[2] = u.x;
                        x[3] = u.y;
#pragma unroll
                        for (int r = 4; r < KM; r += 4) {
                            const float4 t4 = *reinterpret_cast<const float4 *>(colp + grow(r, h));
                            x[r] = t4.x;
                            x[r + 1] = t4.y;
                            x[r + 2] = t4.z;
                            x[r + 3] = t4.w;
                        }
                    }
                    haar_inv_u<KM>(x);
                    if (ra) {  // first Haar row replaced (Eq. 24-25): the refined mean joins every member
                        const int lg = b * GPB + g;
                        const int gy = gy0 + lg / a.tx, gx = gx0 + lg % a.tx;
                        if (lg < gpt && gy <= gy1 && gx <= gx1) {
                            const float *mp = a.mean_est + (size_t)(gy * a.nx + gx) * (C * 64) + p;
                            float mu;  // slice c of the refined mean's pixel p
                            if (C == 1) {
                                mu = __ldg(mp);
                            } else {
                                const float r = __ldg(mp), gg = __ldg(mp + 64), bl = __ldg(mp + 128);
                                mu = c == 0 ? K3F * (r + (gg + bl)) : c == 1 ? K23F * fmaf(-0.5f, gg + bl, r) : K12F * (bl - gg);
                            }
#pragma unroll
                            for (int j = 0; j < KM; ++j) x[j] += mu;
                        }
                    }
                    int *dst = acc_v + c * RP;
#pragma unroll
                    for (int j = 0; j < KM; ++j)
                        if (offs[i][j] >= 0 && HTS_IN_BOUNDS(offs[i][j] < RP, &a.st->error))
                            atomicAdd(dst + offs[i][j], fix8(x[j]));
                }
                tc::fence_before();
                __syncthreads();
            }
            if (!ok) break;
            phase ^= 1u;
        }
        if (!ok) break;
        // flush the tile's sums (per slice) to the image-wide int64 sums
        for (int e = tid; e < rh * rw; e += NT) {
            const int yy = e / rw, xx = e - yy * rw;
            const int le = yy * rwp + xx;
            const size_t gpix = (size_t)(ry0 + yy) * a.W + (rx0 + xx);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int v = acc_v[c * RP + le];
                if (v == 0) continue;
                const long long s = (long long)v * 256ll;  // to the image-wide 2^16 scale
                atomicAdd(reinterpret_cast<unsigned long long *>(a.acc + c * HW + gpix), (unsigned long long)s);
            }
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
        const size_t n = L::bytes(h, w);
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
        const size_t n = L::bytes(h, w);
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
    const size_t need = L::bytes(bt.rh_max, bt.rw_max);
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
    int area = 0;  // the kernel's sums hold rh_max x acc_stride(rw_max) per plane: the largest over the jobs
    for (int j = 0; j < njobs; ++j)
        if (jh[j].rh_max * acc_stride(jh[j].rw_max) > area) {
            area = jh[j].rh_max * acc_stride(jh[j].rw_max);
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
