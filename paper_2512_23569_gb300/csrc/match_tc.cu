// Block matching of the precision form (Alg. 1 step 1 with Eq. 9 planes) on
// the sm_103a tensor cores.
//
// For a reference a and a candidate b of the same matching plane,
//   ||a - b||^2 = ||a||^2 + ||b||^2 - 2 a.b,
// and the cross terms of every candidate position of a tile's search region
// against the tile's 64 references (8 x 8 grid positions) form one BF16 GEMM
// with FP32 accumulation (tcgen05.mma, accumulator in TMEM):
//   D[p][r] = sum_{u<8, v<8} plane[y_p + u][x_p + v] * A[r][8u+v].
// No candidate matrix is materialised: the region is staged once as
// "row-8 vectors" Q[p] = plane[y_p][x_p .. x_p+7] (16 bytes, one core-matrix
// row), candidates are numbered p = y * Wc + x in the region, and the K slice
// of patch rows (u, u+1) of the M = 128 candidates p0 .. p0+127 is the
// shared-memory matrix starting at Q[p0 + u Wc] with core matrices 8 rows
// (128 bytes) apart along M and Wc rows (16 Wc bytes) apart along K.
//
// The candidates are the MMA's M dimension, so a warp reading 32 TMEM lanes
// (eight warps: two per lane quarter, each taking 32 of the reference
// columns) holds, for each reference, 32 candidates side by side: the
// filter "inside the reference's search window and below its threshold" is a
// warp ballot, and the passing candidates are appended to the reference's
// list at a prefix-sum position (one shared atomic per reference and warp).
// Four TMEM accumulators of 64 columns let the MMAs run up to three chunks
// ahead of the warps.  A reference's threshold starts at 1.5 times the
// (K-1)-th smallest BF16 distance to the positions around it (so its K-1
// nearest candidates always pass) and drops to its list's 2K-th smallest
// when the list is cut back (warp-cooperative bisection, between chunks).
// At the end every reference's kept candidates are re-ranked with FP32
// distances of the FP32 plane and the K-1 smallest (ties to the lower raster
// index) follow the reference in its group.  Eq. 9 picks the plane per
// reference: a colour tile runs once per plane that one of its references
// uses.
//
// Every mbarrier wait is bounded; a wait that gives up records error code 2
// in the call's state, and the block waits (bounded) for the MMAs it has
// issued, releases its tensor memory and leaves.
#include <cuda_bf16.h>

#include <algorithm>

#include "hts_internal.h"
#include "tc_ptx.h"

namespace hts {
namespace {

constexpr int TTY = 8, TTX = 8;  // reference tile (grid rows x grid columns)
constexpr int NR = TTY * TTX;    // references per tile = MMA N
constexpr int MC = 128;          // candidates per chunk = MMA M
constexpr int NBUF = 4;          // TMEM accumulators (NR columns each)
constexpr uint32_t TMEM_COLS = 256;
constexpr long long SPIN = 1ll << 24;
constexpr unsigned FULLM = 0xffffffffu;
constexpr int NT = 256;  // threads: warp w reads TMEM lanes 32 (w % 4) .. +31 (its candidates) and the
                         // columns of references 32 (w / 4) .. +31

// Offsets (dy, dx) of the positions around a reference whose distances seed
// its threshold, nearest first (the 7 x 7 square without its centre); the
// first 24 fill the 5 x 5 square.
constexpr int NSEED = 48;
__constant__ signed char c_seed[NSEED][2] = {
    {0, 1},  {1, 0},   {0, -1},  {-1, 0},  {1, 1},   {1, -1},  {-1, 1},  {-1, -1}, {0, 2},   {2, 0},
    {0, -2}, {-2, 0},  {1, 2},   {2, 1},   {-1, 2},  {2, -1},  {1, -2},  {-2, 1},  {-1, -2}, {-2, -1},
    {2, 2},  {2, -2},  {-2, 2},  {-2, -2}, {0, 3},   {3, 0},   {0, -3},  {-3, 0},  {1, 3},   {3, 1},
    {-1, 3}, {3, -1},  {1, -3},  {-3, 1},  {-1, -3}, {-3, -1}, {2, 3},   {3, 2},   {-2, 3},  {3, -2},
    {2, -3}, {-3, 2},  {-2, -3}, {-3, -2}, {3, 3},   {3, -3},  {-3, 3},  {-3, -3}};

struct TcArgs {
    const float *img;
    int H, W, C, step, R, nx, ny, nref;
    int32_t *idx;
    const uint8_t *green;
    DevState *st;
    int ntx, nty, ntiles;
    int hc_max, wc_max;  // bounds of the candidate region over all tiles
};

// Candidates kept per reference for the FP32 re-rank (the "2K"; 48 for K =
// 32) and the list capacity: a list is cut back to BUF once fewer than MC
// free slots (a whole chunk) remain, so cuts are rarer the larger CAP is.
template <int K>
struct ListCfg {
    static constexpr int BUF = (2 * K < 8) ? 8 : (2 * K > 48 ? 48 : 2 * K);
    static constexpr int CAP = BUF + MC + 48;
};

struct TcLayout {
    size_t q, a, e, ps, rn, bd, bp, ref, bar, total;
};

__host__ __device__ inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-reference record in shared memory.
struct RefRec {
    int wy0, wy1, wx0, wx1;  // search window, region coordinates
    int pself, mine, cnt, pad;
    float a2, thr, pad1, pad2;
};

// Shared memory: Q (row-8 vectors), A (references), E (squared norms), the
// FP32 plane Ps, the row norms rn (only needed while E is formed), the lists
// (overlaying rn), per-reference records, barriers.
template <int K>
__host__ __device__ inline TcLayout tc_layout(int hc_max, int wc_max) {
    TcLayout L;
    const size_t nch = ((size_t)hc_max * wc_max + MC - 1) / MC;
    const size_t nq = nch * MC + 7 * (size_t)wc_max;
    L.q = 0;
    L.a = up(L.q + nq * 16, 1024);
    L.e = L.a + (size_t)NR * 64 * 2;
    L.ps = up(L.e + nch * MC * 4, 16);
    L.rn = up(L.ps + (size_t)(hc_max + 7) * (wc_max + 7) * 4, 16);
    L.bd = L.rn;
    L.bp = L.bd + (size_t)NR * ListCfg<K>::CAP * 4;
    const size_t lists_end = L.bp + (size_t)NR * ListCfg<K>::CAP * 4;
    const size_t rn_end = L.rn + nq * 4;
    L.ref = up(lists_end > rn_end ? lists_end : rn_end, 16);
    L.bar = up(L.ref + (size_t)NR * sizeof(RefRec), 16);
    L.total = L.bar + 128;
    if (L.total < 120 * 1024) L.total = 120 * 1024;  // one block per SM
    return L;
}

using tc::bar_init;
using tc::mma_commit;
using tc::sdesc;
using tc::su32;
using tc::tmem_ld32;
using tc::tmem_wait_ld;
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) { return tc::idesc_f16(M, N, true); }
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    tc::mma_f16(d, ad, bd, id, acc);
}
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) { return tc::bar_wait(bar, parity, SPIN); }
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Squared distance of two row-8 BF16 vectors added to acc, in FP32.
__device__ __forceinline__ float row_dist2(uint4 x, uint4 y, float acc) {
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&xs[i]));
        const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ys[i]));
        const float d0 = fa.x - fb.x, d1 = fa.y - fb.y;
        acc = fmaf(d0, d0, acc);
        acc = fmaf(d1, d1, acc);
    }
    return acc;
}

// Warp-cooperative cut of reference j's list (n entries at j * CAP) back to
// `keep` entries containing every entry below the returned T (the smallest
// value, to a 12-step bisection of the list's range, with at least `keep`
// entries <= T); the kept entries stay in list order.
template <int CAP>
__device__ float cut_list_warp(float *bd, int *bp, int j, int n, int keep, int lane, int *n_out) {
    constexpr int PER = (CAP + 31) / 32;
    float dv[PER];
    int pv[PER];
    float lo = __builtin_huge_valf(), hi = -__builtin_huge_valf();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int i = t * 32 + lane;
        dv[t] = (i < n) ? bd[j * CAP + i] : __builtin_huge_valf();
        pv[t] = (i < n) ? bp[j * CAP + i] : 0;
        if (i < n) {
            lo = fminf(lo, dv[t]);
            hi = fmaxf(hi, dv[t]);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(FULLM, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(FULLM, hi, o));
    }
    for (int it = 0; it < 12; ++it) {  // invariant: count(<= hi) >= keep
        const float mid = 0.5f * (lo + hi);
        int c = 0;
#pragma unroll
        for (int t = 0; t < PER; ++t) c += __popc(__ballot_sync(FULLM, dv[t] <= mid));
        if (c >= keep) hi = mid;
        else lo = mid;
    }
    __syncwarp();
    int w = 0;
#pragma unroll
    for (int t = 0; t < PER; ++t) {  // stable compaction: entries <= hi, at most `keep`
        const bool k = dv[t] <= hi;
        const uint32_t m = __ballot_sync(FULLM, k);
        const int pos = w + __popc(m & ((1u << lane) - 1u));
        if (k && pos < keep) {
            bd[j * CAP + pos] = dv[t];
            bp[j * CAP + pos] = pv[t];
        }
        w += __popc(m);
    }
    __syncwarp();
    *n_out = w < keep ? w : keep;
    return hi;
}

template <int K>
__global__ void __launch_bounds__(NT, 1) k_match_tc(TcArgs a) {
    constexpr int BUF = ListCfg<K>::BUF, CAP = ListCfg<K>::CAP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const TcLayout L = tc_layout<K>(a.hc_max, a.wc_max);
    uint4 *Q = reinterpret_cast<uint4 *>(smem_raw + L.q);
    unsigned char *Abuf = smem_raw + L.a;
    float *E = reinterpret_cast<float *>(smem_raw + L.e);
    float *Ps = reinterpret_cast<float *>(smem_raw + L.ps);
    float *rn = reinterpret_cast<float *>(smem_raw + L.rn);
    float *bd = reinterpret_cast<float *>(smem_raw + L.bd);
    int *bp = reinterpret_cast<int *>(smem_raw + L.bp);
    RefRec *rec = reinterpret_cast<RefRec *>(smem_raw + L.ref);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L.bar);  // [NBUF]
    long long *issued_hi = reinterpret_cast<long long *>(full + NBUF);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(issued_hi + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wq4 = warp & 3, wcol = (warp >> 2) * 32;  // TMEM lane quarter, first reference column
    const size_t HW = (size_t)a.H * a.W;
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) bar_init(&full[b], 1);
        *issued_hi = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t idesc = idesc_bf16(MC, NR);
    long long gc = 0;  // chunks issued by this block so far (buffer = gc % NBUF, use = gc / NBUF)
    bool ok = true;

    for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
        const int tyi = tile / a.ntx, txi = tile - tyi * a.ntx;
        const int gy0 = tyi * TTY, gx0 = txi * TTX;
        const int gy1 = min(a.ny, gy0 + TTY) - 1, gx1 = min(a.nx, gx0 + TTX) - 1;
        const int cy0 = max(0, grid_pos(gy0, a.H, a.step) - a.R);
        const int cy1 = min(a.H - PS, grid_pos(gy1, a.H, a.step) + a.R);
        const int cx0 = max(0, grid_pos(gx0, a.W, a.step) - a.R);
        const int cx1 = min(a.W - PS, grid_pos(gx1, a.W, a.step) + a.R);
        const int Hc = cy1 - cy0 + 1, Wc = cx1 - cx0 + 1, PSW = Wc + 7;
        const int ncand = Hc * Wc;
        const int nch = (ncand + MC - 1) / MC;
        const int nq = nch * MC + 7 * Wc;

        for (int pass = 0; pass < (a.C == 3 ? 2 : 1) && ok; ++pass) {
            // ---- per-reference records (thread j < NR: reference j = row j/8, column j%8 of the tile)
            bool any = false;
            if (tid < NR) {
                const int ry = gy0 + (tid >> 3), rx = gx0 + (tid & 7);
                const bool valid = ry <= gy1 && rx <= gx1;
                const int r = valid ? ry * a.nx + rx : 0;
                const bool mine = valid && (a.C == 1 || (int)a.green[r] == (pass == 0 ? 1 : 0));
                const int yr = grid_pos(min(ry, gy1), a.H, a.step), xr = grid_pos(min(rx, gx1), a.W, a.step);
                RefRec q;
                q.wy0 = max(0, yr - a.R) - cy0;
                q.wy1 = min(a.H - PS, yr + a.R) - cy0;
                q.wx0 = max(0, xr - a.R) - cx0;
                q.wx1 = min(a.W - PS, xr + a.R) - cx0;
                q.pself = (yr - cy0) * Wc + (xr - cx0);
                q.mine = mine ? 1 : 0;
                q.cnt = 0;
                q.pad = 0;
                q.a2 = 0.f;
                q.thr = __builtin_huge_valf();
                q.pad1 = q.pad2 = 0.f;
                rec[tid] = q;
                any = mine;
            }
            if (!__syncthreads_or(any)) continue;
            // ---- stage the plane (FP32), the row-8 vectors and their norms, E, A
            for (int e = tid; e < (Hc + 7) * PSW; e += NT) {
                const int y = e / PSW, x = e - y * PSW;
                const size_t o = (size_t)(cy0 + y) * a.W + cx0 + x;
                float v;
                if (a.C == 1) v = __ldg(a.img + o);
                else if (pass == 0) v = __ldg(a.img + HW + o);
                else v = (__ldg(a.img + o) + __ldg(a.img + HW + o)) + __ldg(a.img + 2 * HW + o);
                Ps[e] = v;
            }
            __syncthreads();
            for (int q = tid; q < nq; q += NT) {
                const int y = q / Wc, x = q - y * Wc;
                uint4 w = make_uint4(0, 0, 0, 0);
                float n2 = 0.f;
                if (y < Hc + 7) {
                    const float *s = Ps + y * PSW + x;
#pragma unroll
                    for (int v = 0; v < PS; ++v) {
                        const float b = bf_round(s[v]);
                        n2 = fmaf(b, b, n2);
                    }
                    w = make_uint4(pack_bf16(s[0], s[1]), pack_bf16(s[2], s[3]), pack_bf16(s[4], s[5]),
                                   pack_bf16(s[6], s[7]));
                }
                Q[q] = w;
                rn[q] = n2;  // squared norm of the BF16 row-8 vector
            }
            __syncthreads();
            for (int p = tid; p < nch * MC; p += NT) {
                float e2 = 0.f;
                if (p < ncand) {
#pragma unroll
                    for (int u = 0; u < PS; ++u) e2 += rn[p + u * Wc];
                }
                E[p] = e2;
            }
            // A: row j = reference j, element 8u+v; core matrix (j/8, u) at (j/8)*1024 + u*128
            for (int e = tid; e < NR * PS; e += NT) {
                const int j = e >> 3, u = e & 7;
                const int ty_ = gy0 + (j >> 3), tx_ = gx0 + (j & 7);
                uint4 w = make_uint4(0, 0, 0, 0);
                if (ty_ <= gy1 && tx_ <= gx1) w = Q[rec[j].pself + u * Wc];
                *reinterpret_cast<uint4 *>(Abuf + (j >> 3) * 1024 + u * 128 + (j & 7) * 16) = w;
            }
            __syncthreads();  // rn is dead from here: the lists overlay it
            // ---- thresholds: 1.5 x the (K-1)-th smallest BF16 distance from the reference to the
            //      positions around it (an upper bound of its (K-1)-th nearest candidate, so those
            //      always pass), plus a margin for the different FP32 rounding of the MMA form
            if (tid < NR && rec[tid].mine) {
                constexpr int NS = (K + 8 > 24) ? ((K + 8 > NSEED) ? NSEED : K + 8) : 24;
                const RefRec q = rec[tid];
                const int ay = q.pself / Wc, ax = q.pself - ay * Wc;
                const float a2 = E[q.pself];
                float best[K - 1];
#pragma unroll
                for (int i = 0; i < K - 1; ++i) best[i] = __builtin_huge_valf();
                for (int sidx = 0; sidx < NS; ++sidx) {
                    const int y = ay + c_seed[sidx][0], x = ax + c_seed[sidx][1];
                    const bool in = y >= q.wy0 && y <= q.wy1 && x >= q.wx0 && x <= q.wx1;
                    const int pq = in ? y * Wc + x : q.pself;
                    float d = 0.f;
#pragma unroll
                    for (int u = 0; u < PS; ++u) d = row_dist2(Q[q.pself + u * Wc], Q[pq + u * Wc], d);
                    if (!in) d = __builtin_huge_valf();
#pragma unroll
                    for (int i = 0; i < K - 1; ++i) {  // branch-free insertion into the sorted seeds
                        const float lo = fminf(best[i], d);
                        d = fmaxf(best[i], d);
                        best[i] = lo;
                    }
                }
                const float t = best[K - 2];
                rec[tid].a2 = a2;
                rec[tid].thr = (t < __builtin_huge_valf()) ? t * 1.5f + 1e-6f * (4.f * a2 + 1.f)
                                                           : __builtin_huge_valf();
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();

            // ---- chunks of MC candidates: MMAs (thread 0), then every warp's 32 lanes
            auto issue = [&](int c, long long g) {
                const uint32_t b = (uint32_t)(g % NBUF);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t cd = sdesc(su32(Q + (size_t)c * MC + (size_t)2 * kk * Wc), 16u * Wc, 128);
                    const uint64_t rd = sdesc(su32(Abuf) + kk * 256, 128, 1024);
                    mma_bf16(tbase + b * NR, cd, rd, idesc, kk > 0 ? 1u : 0u);
                }
                mma_commit(&full[b]);
            };
            const long long g0 = gc;
            if (tid == 0) {
                tc_fence_after();
                for (int c = 0; c < nch && c < NBUF; ++c) issue(c, g0 + c);
                *issued_hi = g0 + min(nch, NBUF);
            }
            long long consumed = g0;
            for (int c = 0; c < nch; ++c) {
                const long long g = g0 + c;
                const uint32_t b = (uint32_t)(g % NBUF);
                if (bar_wait(&full[b], (uint32_t)((g / NBUF) & 1))) consumed = g + 1;
                else ok = false;
                ok = __all_sync(FULLM, ok);
                if (ok) {
                    tc_fence_after();
                    uint32_t v0[32];
                    tmem_ld32(tbase + ((uint32_t)(wq4 * 32) << 16) + b * NR + wcol, v0);
                    tmem_wait_ld();
                    // this lane's candidate
                    const int pw = c * MC + wq4 * 32;
                    const int p = pw + lane;
                    const bool cval = p < ncand;
                    const int prow = p / Wc, pcol = p - prow * Wc;
                    const float e = cval ? E[p] : 0.f;
                    const int rlo = pw / Wc, rhi = min(pw + 31, ncand - 1) / Wc;
                    (void)rlo;
                    (void)rhi;
                    auto scan = [&](int j, uint32_t raw) {
                        // no branch before the ballot, so the loads of consecutive references overlap
                        const int4 wq = *reinterpret_cast<const int4 *>(&rec[j].wy0);
                        const int4 wm = *reinterpret_cast<const int4 *>(&rec[j].pself);
                        const float2 at = *reinterpret_cast<const float2 *>(&rec[j].a2);
                        const float d = e + at.x - 2.f * __uint_as_float(raw);
                        const bool pass = wm.y && cval && prow >= wq.x && prow <= wq.y && pcol >= wq.z &&
                                          pcol <= wq.w && p != wm.x && d < at.y;
                        const uint32_t m = __ballot_sync(FULLM, pass);
                        if (!m) return;
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&rec[j].cnt, __popc(m));
                        base = __shfl_sync(FULLM, base, 0);
                        const int pos = base + __popc(m & ((1u << lane) - 1u));
                        if (pass && pos < CAP) {
                            bd[j * CAP + pos] = d;
                            bp[j * CAP + pos] = p;
                        }
                    };
#pragma unroll
                    for (int j = 0; j < 32; ++j) scan(wcol + j, v0[j]);
                }
                tc_fence_before();
                ok = !__syncthreads_or(!ok);
                if (!ok) break;
                // lists that the next chunk could overflow are cut back (reference j by warp j mod 4)
                if (c + 1 < nch) {
                    for (int j = warp; j < NR; j += NT / 32) {
                        const int n = rec[j].cnt;
                        if (n > CAP - MC) {
                            int n2 = 0;
                            const float t = cut_list_warp<CAP>(bd, bp, j, n < CAP ? n : CAP, BUF, lane, &n2);
                            if (lane == 0) {
                                rec[j].cnt = n2;
                                rec[j].thr = fminf(rec[j].thr, t);
                            }
                        }
                    }
                }
                __syncthreads();
                if (tid == 0 && c + NBUF < nch) {  // the buffer of chunk c is free: chunk c + NBUF goes there
                    tc_fence_after();
                    issue(c + NBUF, g + NBUF);
                    *issued_hi = g + NBUF + 1;
                }
            }
            if (!ok) {  // drain: wait (bounded) for the MMAs already issued before the memory is released
                for (long long g = consumed; g < *issued_hi; ++g)
                    bar_wait(&full[g % NBUF], (uint32_t)((g / NBUF) & 1));
                break;
            }
            gc = g0 + nch;

            // ---- per reference (one warp each): cut back to BUF, FP32 re-rank of the kept
            //      candidates, the K-1 nearest by (distance, raster index)
            for (int j = warp; j < NR; j += NT / 32) {
                if (!rec[j].mine) continue;
                int n = min(rec[j].cnt, CAP);
                if (n > BUF) cut_list_warp<CAP>(bd, bp, j, n, BUF, lane, &n);
                const int pself = rec[j].pself;
                const int ay = pself / Wc, ax = pself - ay * Wc;
                constexpr int PER = (BUF + 31) / 32;
                float dk[PER];
                int rk[PER];
#pragma unroll
                for (int t = 0; t < PER; ++t) {
                    const int i = t * 32 + lane;
                    dk[t] = __builtin_huge_valf();
                    rk[t] = 0x7fffffff;
                    if (i < n) {
                        const int pq = bp[j * CAP + i];
                        const int by = pq / Wc, bx = pq - by * Wc;
                        float d = 0.f;
                        for (int u = 0; u < PS; ++u) {
                            const float *ra = Ps + (ay + u) * PSW + ax, *rb = Ps + (by + u) * PSW + bx;
#pragma unroll
                            for (int v = 0; v < PS; ++v) {
                                const float df = ra[v] - rb[v];
                                d = fmaf(df, df, d);
                            }
                        }
                        dk[t] = d;
                        rk[t] = (cy0 + by) * a.W + cx0 + bx;
                    }
                }
                const int r = (gy0 + (j >> 3)) * a.nx + gx0 + (j & 7);
                int32_t *out = a.idx + (size_t)r * K;
                const int self = (cy0 + ay) * a.W + cx0 + ax;
                if (lane == 0) out[0] = self;
                for (int k = 1; k < K; ++k) {  // K-1 rounds of a warp arg-min on (distance, raster)
                    float bdv = dk[0];
                    int brv = rk[0];
#pragma unroll
                    for (int t = 1; t < PER; ++t)
                        if (dk[t] < bdv || (dk[t] == bdv && rk[t] < brv)) {
                            bdv = dk[t];
                            brv = rk[t];
                        }
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        const float od = __shfl_xor_sync(FULLM, bdv, o);
                        const int orr = __shfl_xor_sync(FULLM, brv, o);
                        if (od < bdv || (od == bdv && orr < brv)) {
                            bdv = od;
                            brv = orr;
                        }
                    }
                    if (lane == 0) out[k] = (brv == 0x7fffffff) ? self : brv;
#pragma unroll
                    for (int t = 0; t < PER; ++t)
                        if (rk[t] == brv) {
                            dk[t] = __builtin_huge_valf();
                            rk[t] = 0x7fffffff;
                        }
                }
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
}

template <int K>
hts_status launch_tc(const TcArgs &a, cudaStream_t s) {
    const TcLayout L = tc_layout<K>(a.hc_max, a.wc_max);
    const hts_status st0 = allow_smem(reinterpret_cast<const void *>(k_match_tc<K>), L.total);
    if (st0 != HTS_OK) return st0;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(a.ntiles, nsm));
    {
        KTimer kt("k_match_tc", s);
        k_match_tc<K><<<grid, NT, L.total, s>>>(a);
    }
    return check_launch("k_match_tc");
}

}  // namespace

hts_status launch_match_tc(const float *img, const Geom &g, int32_t *idx, const uint8_t *green, DevState *st,
                           cudaStream_t s) {
    TcArgs a;
    a.img = img;
    a.H = g.H;
    a.W = g.W;
    a.C = g.C;
    a.step = g.step;
    a.R = g.R;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nref = g.nref;
    a.idx = idx;
    a.green = green;
    a.st = st;
    a.nty = (g.ny + TTY - 1) / TTY;
    a.ntx = (g.nx + TTX - 1) / TTX;
    a.ntiles = a.nty * a.ntx;
    a.hc_max = std::min(g.H - PS + 1, (TTY - 1) * g.step + 1 + 2 * g.R);
    a.wc_max = std::min(g.W - PS + 1, (TTX - 1) * g.step + 1 + 2 * g.R);
    switch (g.K) {
        case 2: return launch_tc<2>(a, s);
        case 4: return launch_tc<4>(a, s);
        case 8: return launch_tc<8>(a, s);
        case 16: return launch_tc<16>(a, s);
        case 32: return launch_tc<32>(a, s);
        default: return HTS_EUNSUPPORTED;
    }
}

}  // namespace hts
