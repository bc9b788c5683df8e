// Block matching of the precision form (Alg. 1 step 1 with Eq. 9 planes) on
// the sm_103a tensor cores.
//
// For a reference a and a candidate b of the same matching plane,
//   ||a - b||^2 = ||a||^2 + ||b||^2 - 2 a.b,
// and the cross terms of a tile of 128 references (16 x 8 grid positions)
// against every candidate position of the tile's search region form one
// BF16 GEMM with FP32 accumulation (tcgen05.mma, accumulator in TMEM):
//   D[r][p] = sum_{u<8, v<8} A[r][8u+v] * plane[y_p + u][x_p + v].
// No candidate matrix is materialised: the region is staged once as
// "row-8 vectors" Q[p] = plane[y_p][x_p .. x_p+7] (16 bytes, one core-matrix
// row), candidates are numbered p = y * Wc + x in the region, and the K slice
// of patch rows (u, u+1) of the N = 256 candidates p0 .. p0+255 is the
// shared-memory matrix starting at Q[p0 + u Wc] with core matrices 8 rows
// (128 bytes) apart along N and Wc rows (16 Wc bytes) apart along K.
// Two TMEM accumulators of 256 columns alternate: the MMAs of chunk c+1 run
// while the four warps read chunk c.  Each thread owns one reference (TMEM
// lane), forms the approximate distance of every candidate inside its
// search window from the accumulator and the BF16 squared norms, and keeps
// the 2K smallest (48 for K = 32); those are re-ranked with FP32 distances of
// the FP32 plane, and the K-1 smallest (ties to the lower raster index)
// follow the reference in its group.  Eq. 9 picks the plane per reference: a colour
// tile runs once per plane that one of its references uses.
//
// Every mbarrier wait is bounded; a wait that gives up records error code 2
// in the call's state, and the block waits (bounded) for the MMAs it has
// issued, releases its tensor memory and leaves.
#include <cuda_bf16.h>

#include <algorithm>

#include "hts_internal.h"

namespace hts {
namespace {

constexpr int TTY = 16, TTX = 8;  // reference tile (grid rows x grid columns) = 128 = MMA M
constexpr int NCH = 256;          // candidates per MMA (N) and per TMEM accumulator
constexpr uint32_t TMEM_COLS = 512;
constexpr long long SPIN = 1ll << 24;
constexpr unsigned FULLM = 0xffffffffu;

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

struct TcLayout {
    size_t r0, a, e, ps, rn, bd, bp, bar, total;
};

__host__ __device__ inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Candidates kept per reference (the "2K" of the re-rank; 48 for K = 32 to
// fit on chip) and the list capacity: a 32-candidate group is appended
// without checks and the list is cut back to BUF when it might overflow.
template <int K>
struct ListCfg {
    static constexpr int BUF = (2 * K < 8) ? 8 : (2 * K > 48 ? 48 : 2 * K);
    static constexpr int CAP = BUF + 32;
    static constexpr bool KEEP_PLANE = K <= 16;  // FP32 plane stays on chip for the re-rank
};

// Shared memory: Q (row-8 vectors), A, E (squared norms), the FP32 plane Ps,
// then the lists, which overlay the row norms rn (only needed before the
// MMAs) -- and, for K = 32, Ps too (the re-rank then reads global memory).
template <int K>
__host__ __device__ inline TcLayout tc_layout(int hc_max, int wc_max) {
    TcLayout L;
    const size_t nch = ((size_t)hc_max * wc_max + NCH - 1) / NCH;
    const size_t nr0 = nch * NCH + 7 * (size_t)wc_max;
    L.r0 = 0;
    L.a = up(L.r0 + nr0 * 16, 1024);
    L.e = L.a + 128 * 64 * 2;
    L.ps = up(L.e + nch * NCH * 4, 16);
    L.rn = up(L.ps + (size_t)(hc_max + 7) * (wc_max + 7) * 4, 16);  // row norms, after the plane
    L.bd = ListCfg<K>::KEEP_PLANE ? L.rn : L.ps;
    L.bp = L.bd + (size_t)ListCfg<K>::CAP * 128 * 4;
    const size_t lists_end = L.bp + (size_t)ListCfg<K>::CAP * 128 * 4;
    const size_t ps_end = L.rn + nr0 * 4;
    L.bar = up(lists_end > ps_end ? lists_end : ps_end, 16);
    L.total = L.bar + 64;
    if (L.total < 120 * 1024) L.total = 120 * 1024;  // one block per SM: it holds all 512 TMEM columns
    return L;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: lbo = bytes between core
// matrices along K, sbo = bytes between core matrices along M / N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)));
}

__device__ __forceinline__ void bar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(su32(bar)));
}

// Bounded wait (non-blocking polls) for the completion of the phase with this
// parity; false on giving up.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    for (long long it = 0; it < SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Cuts this thread's list (slots i * 128 + tid, i < cnt) back to `keep`
// entries that include every entry below the returned value T (T is the
// smallest value, to a bisection of 24 steps, with at least `keep` entries
// <= T); later candidates are kept only if below T.  Every lane runs the same
// instruction sequence (loops over CAP slots with predicates), so lanes of a
// warp that cut together do not serialise.
template <int CAP>
__device__ float cut_list(float *bd, int *bp, int tid, int &cnt, int keep) {
    float lo = __builtin_huge_valf(), hi = -__builtin_huge_valf();
#pragma unroll 4
    for (int i = 0; i < CAP; ++i) {
        const float d = bd[i * 128 + tid];
        if (i < cnt) {
            lo = fminf(lo, d);
            hi = fmaxf(hi, d);
        }
    }
    for (int it = 0; it < 24; ++it) {  // invariant: count(<= hi) >= keep
        const float mid = 0.5f * (lo + hi);
        int c = 0;
#pragma unroll 8
        for (int i = 0; i < CAP; ++i) c += (i < cnt && bd[i * 128 + tid] <= mid) ? 1 : 0;
        if (c >= keep) hi = mid;
        else lo = mid;
    }
    int w = 0;
    for (int i = 0; i < CAP; ++i) {  // stable compaction: entries < hi, then entries == hi up to `keep`
        const float d = bd[i * 128 + tid];
        const int pv = bp[i * 128 + tid];
        if (i < cnt && d <= hi && w < keep) {
            bd[w * 128 + tid] = d;
            bp[w * 128 + tid] = pv;
            ++w;
        }
    }
    cnt = w;
    return hi;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

template <int K>
__global__ void __launch_bounds__(128, 1) k_match_tc(TcArgs a) {
    constexpr int BUF = ListCfg<K>::BUF, CAP = ListCfg<K>::CAP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const TcLayout L = tc_layout<K>(a.hc_max, a.wc_max);
    uint4 *Q = reinterpret_cast<uint4 *>(smem_raw + L.r0);
    unsigned char *Abuf = smem_raw + L.a;
    float *E = reinterpret_cast<float *>(smem_raw + L.e);
    float *Ps = reinterpret_cast<float *>(smem_raw + L.ps);
    float *rn = reinterpret_cast<float *>(smem_raw + L.rn);
    float *bd = reinterpret_cast<float *>(smem_raw + L.bd);
    int *bp = reinterpret_cast<int *>(smem_raw + L.bp);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L.bar);  // [2]
    uint64_t *empty = full + 2;                                         // [2]
    long long *issued_hi = reinterpret_cast<long long *>(empty + 2);  // one past the last chunk issued
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(issued_hi + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t HW = (size_t)a.H * a.W;
    if (tid == 0) {
        bar_init(&full[0], 1);
        bar_init(&full[1], 1);
        bar_init(&empty[0], 4);
        bar_init(&empty[1], 4);
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
    const uint32_t idesc = idesc_bf16(128, NCH);
    long long gc = 0;  // chunks issued by this block so far (buffer = gc & 1, use = gc >> 1)
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
        const int nch = (ncand + NCH - 1) / NCH;
        const int nq = nch * NCH + 7 * Wc;
        // this thread's reference
        const int ry = gy0 + warp * 4 + (lane >> 3), rx = gx0 + (lane & 7);
        const bool rvalid = ry <= gy1 && rx <= gx1;
        const int r = rvalid ? ry * a.nx + rx : 0;
        const int yr = grid_pos(ry, a.H, a.step), xr = grid_pos(rx, a.W, a.step);
        const int wy0 = max(0, yr - a.R) - cy0, wy1 = min(a.H - PS, yr + a.R) - cy0;  // window, region coords
        const int wx0 = max(0, xr - a.R) - cx0, wx1 = min(a.W - PS, xr + a.R) - cx0;
        const int pself = (yr - cy0) * Wc + (xr - cx0);

        for (int pass = 0; pass < (a.C == 3 ? 2 : 1) && ok; ++pass) {
            const bool mine = rvalid && (a.C == 1 || (int)a.green[r] == (pass == 0 ? 1 : 0));
            if (!__syncthreads_or(mine)) continue;
            // ---- stage the plane (FP32), then the row-8 vectors, A and the squared norms
            for (int e = tid; e < (Hc + 7) * PSW; e += 128) {
                const int y = e / PSW, x = e - y * PSW;
                const size_t o = (size_t)(cy0 + y) * a.W + cx0 + x;
                float v;
                if (a.C == 1) v = __ldg(a.img + o);
                else if (pass == 0) v = __ldg(a.img + HW + o);
                else v = (__ldg(a.img + o) + __ldg(a.img + HW + o)) + __ldg(a.img + 2 * HW + o);
                Ps[e] = v;
            }
            __syncthreads();
            for (int q = tid; q < nq; q += 128) {
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
            for (int p = tid; p < nch * NCH; p += 128) {
                float e2 = 0.f;
                if (p < ncand) {
#pragma unroll
                    for (int u = 0; u < PS; ++u) e2 += rn[p + u * Wc];
                }
                E[p] = e2;
            }
            // A: row t = this block's reference t, element 8u+v; core matrix (t/8, u) at (t/8)*1024 + u*128
            for (int e = tid; e < 128 * PS; e += 128) {
                const int t = e >> 3, u = e & 7;
                const int tw = t >> 5, tl = t & 31;
                const int ty_ = gy0 + tw * 4 + (tl >> 3), tx_ = gx0 + (tl & 7);
                uint4 w = make_uint4(0, 0, 0, 0);
                if (ty_ <= gy1 && tx_ <= gx1) {
                    const int py = grid_pos(ty_, a.H, a.step) - cy0 + u, px = grid_pos(tx_, a.W, a.step) - cx0;
                    const float *s = Ps + py * PSW + px;
                    w = make_uint4(pack_bf16(s[0], s[1]), pack_bf16(s[2], s[3]), pack_bf16(s[4], s[5]),
                                   pack_bf16(s[6], s[7]));
                }
                *reinterpret_cast<uint4 *>(Abuf + (t >> 3) * 1024 + u * 128 + (t & 7) * 16) = w;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            const float a2 = rvalid ? E[min(pself, nch * NCH - 1)] : 0.f;

            // ---- chunks: MMAs (warp 0, one elected lane) and the per-reference scan
            auto issue = [&](int c, long long g) {
                const uint32_t b = (uint32_t)(g & 1);
                const uint32_t d = tbase + b * NCH;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = sdesc(su32(Abuf) + kk * 256, 128, 1024);
                    const uint64_t bdsc = sdesc(su32(Q + (size_t)c * NCH + (size_t)2 * kk * Wc), 16u * Wc, 128);
                    mma_bf16(d, ad, bdsc, idesc, kk > 0 ? 1u : 0u);
                }
                mma_commit(&full[b]);
            };
            const long long g0 = gc;
            if (warp == 0 && lane == 0) {
                tc_fence_after();
                issue(0, g0);
                if (nch > 1) issue(1, g0 + 1);
                *issued_hi = g0 + (nch > 1 ? 2 : 1);
            }
            __syncwarp();
            // threshold seed: the (K-1)-th smallest BF16 distance from the reference to the
            // positions around it bounds the (K-1)-th nearest candidate from above, so every
            // candidate that can be among the K-1 nearest passes the filter below it, while
            // few others do (a factor 1.5 and an absolute margin cover the different FP32
            // rounding of the tensor-core form and keep, for the FP32 re-rank, the candidates
            // that BF16 rounding ranks slightly too far)
            int cnt = 0;
            float thr = __builtin_huge_valf();
            if (mine) {
                constexpr int NS = (K + 8 > 24) ? ((K + 8 > NSEED) ? NSEED : K + 8) : 24;
                const int ay = yr - cy0, ax = xr - cx0;
                float ab[64];
#pragma unroll
                for (int e = 0; e < 64; ++e) ab[e] = bf_round(Ps[(ay + (e >> 3)) * PSW + ax + (e & 7)]);
                float best[K - 1];
#pragma unroll
                for (int i = 0; i < K - 1; ++i) best[i] = __builtin_huge_valf();
                for (int sidx = 0; sidx < NS; ++sidx) {
                    const int y = yr + c_seed[sidx][0], x = xr + c_seed[sidx][1];
                    const bool in = y >= max(0, yr - a.R) && y <= min(a.H - PS, yr + a.R) &&
                                    x >= max(0, xr - a.R) && x <= min(a.W - PS, xr + a.R);
                    const float *q = Ps + (in ? (y - cy0) * PSW + (x - cx0) : ay * PSW + ax);
                    float d = 0.f;
#pragma unroll
                    for (int e = 0; e < 64; ++e) {
                        const float df = ab[e] - bf_round(q[(e >> 3) * PSW + (e & 7)]);
                        d = fmaf(df, df, d);
                    }
                    if (!in) d = __builtin_huge_valf();
#pragma unroll
                    for (int i = 0; i < K - 1; ++i) {  // branch-free insertion into the sorted seeds
                        const float lo = fminf(best[i], d);
                        d = fmaxf(best[i], d);
                        best[i] = lo;
                    }
                }
                const float t = best[K - 2];
                if (t < __builtin_huge_valf()) thr = t * 1.5f + 1e-6f * (4.f * a2 + 1.f);
            }
            long long consumed = g0;  // chunks whose accumulator this thread has waited for
            const int ylo = __reduce_min_sync(FULLM, mine ? wy0 : 1 << 30);
            const int yhi = __reduce_max_sync(FULLM, mine ? wy1 : -1);
            const int xlo = __reduce_min_sync(FULLM, mine ? wx0 : 1 << 30);
            const int xhi = __reduce_max_sync(FULLM, mine ? wx1 : -1);
            for (int c = 0; c < nch; ++c) {
                const long long g = g0 + c;
                const uint32_t b = (uint32_t)(g & 1);
                if (bar_wait(&full[b], (uint32_t)((g >> 1) & 1))) consumed = g + 1;
                else ok = false;
                ok = __all_sync(FULLM, ok);
                if (!ok) {
                    if (lane == 0) atomicExch(&a.st->error, 2);
                    break;
                }
                tc_fence_after();
                const int p0 = c * NCH;
#pragma unroll 1
                for (int grp = 0; grp < NCH / 32; ++grp) {
                    const int pg = p0 + grp * 32;
                    if (pg >= ncand) break;
                    // warp-uniform skip of 32-column groups outside every window of the warp
                    const int rlo = pg / Wc, rhi = min(pg + 31, ncand - 1) / Wc;
                    if (rhi < ylo || rlo > yhi) continue;
                    if (rlo == rhi && (pg - rlo * Wc > xhi || pg - rlo * Wc + 31 < xlo)) continue;
                    uint32_t v[32];
                    tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + b * NCH + grp * 32, v);
                    // candidates of this group inside this reference's window, as a bit mask
                    uint32_t mask = 0;
                    if (mine) {
                        int j = 0, row = rlo, col = pg - rlo * Wc;
                        while (j < 32) {
                            const int seg = min(32 - j, Wc - col);
                            if (row >= wy0 && row <= wy1) {
                                const int c0 = max(col, wx0), c1 = min(col + seg - 1, wx1);
                                if (c0 <= c1) {
                                    const int n = c1 - c0 + 1;
                                    mask |= (n == 32 ? 0xffffffffu : ((1u << n) - 1u)) << (j + c0 - col);
                                }
                            }
                            j += seg;
                            ++row;
                            col = 0;
                        }
                        if (ncand - pg < 32) mask &= (1u << (ncand - pg)) - 1u;
                        if (pself >= pg && pself < pg + 32) mask &= ~(1u << (pself - pg));
                    }
                    if (!__any_sync(FULLM, mask != 0)) continue;
                    const float4 *e4 = reinterpret_cast<const float4 *>(E + pg);
                    float dd[32];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 ev = e4[q];
                        dd[4 * q + 0] = ev.x + a2 - 2.f * __uint_as_float(v[4 * q + 0]);
                        dd[4 * q + 1] = ev.y + a2 - 2.f * __uint_as_float(v[4 * q + 1]);
                        dd[4 * q + 2] = ev.z + a2 - 2.f * __uint_as_float(v[4 * q + 2]);
                        dd[4 * q + 3] = ev.w + a2 - 2.f * __uint_as_float(v[4 * q + 3]);
                    }
                    uint32_t acc = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc |= (dd[j] < thr ? 1u : 0u) << j;
                    acc &= mask;
                    // lists are cut back together: when one lane must, every lane above BUF does
                    if (__any_sync(FULLM, cnt + __popc(acc) > CAP) && cnt > BUF) {
                        thr = fminf(thr, cut_list<CAP>(bd, bp, tid, cnt, BUF));
                        uint32_t a2m = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) a2m |= (dd[j] < thr ? 1u : 0u) << j;
                        acc &= a2m;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if ((acc >> j) & 1u) {
                            bd[cnt * 128 + tid] = dd[j];
                            bp[cnt * 128 + tid] = pg + j;  // region position; raster index at the re-rank
                            ++cnt;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&empty[b]);
                if (warp == 0 && c + 2 < nch) {
                    const bool got = __all_sync(FULLM, bar_wait(&empty[b], (uint32_t)((g >> 1) & 1)));
                    tc_fence_after();
                    if (lane == 0) {
                        if (got) {
                            issue(c + 2, g + 2);
                            *issued_hi = g + 3;
                        } else {
                            atomicExch(&a.st->error, 2);
                        }
                    }
                    __syncwarp();
                    if (!got) {
                        ok = false;
                        break;
                    }
                }
            }
            ok = !__syncthreads_or(!ok);
            if (!ok) {  // drain: wait (bounded) for the MMAs already issued before the memory is released
                for (long long g = consumed; g < *issued_hi; ++g) bar_wait(&full[g & 1], (uint32_t)((g >> 1) & 1));
                break;
            }
            gc = g0 + nch;

            // ---- FP32 re-rank of the kept candidates (plane read from global memory: the staging
            //      area now holds the lists), then the K-1 nearest (ties: lower raster index)
            if (mine) {
                if (cnt > BUF) cut_list<CAP>(bd, bp, tid, cnt, BUF);
                const float *c0 = a.img, *c1 = a.img + HW, *c2 = a.img + 2 * HW;
                // plane value at region row y, column x (on chip when kept, else from global memory)
                auto plane = [&](int y, int x) -> float {
                    if (ListCfg<K>::KEEP_PLANE) return Ps[y * PSW + x];
                    const size_t o = (size_t)(cy0 + y) * a.W + cx0 + x;
                    if (a.C == 1) return __ldg(c0 + o);
                    if (pass == 0) return __ldg(c1 + o);
                    return (__ldg(c0 + o) + __ldg(c1 + o)) + __ldg(c2 + o);
                };
                const int ay = yr - cy0, ax = xr - cx0;
                float ar[64];
#pragma unroll
                for (int e = 0; e < 64; ++e) ar[e] = plane(ay + (e >> 3), ax + (e & 7));
                for (int t = 0; t < cnt; ++t) {
                    const int pq = bp[t * 128 + tid];
                    const int by = pq / Wc, bx = pq - by * Wc;
                    bp[t * 128 + tid] = (cy0 + by) * a.W + cx0 + bx;
                    float d = 0.f;
#pragma unroll
                    for (int e = 0; e < 64; ++e) {
                        const float df = ar[e] - plane(by + (e >> 3), bx + (e & 7));
                        d = fmaf(df, df, d);
                    }
                    bd[t * 128 + tid] = d;
                }
                int32_t *out = a.idx + (size_t)r * K;
                out[0] = yr * a.W + xr;
                for (int k = 1; k < K; ++k) {
                    int best = -1;
                    float bdv = 0.f;
                    int bpv = 0;
                    for (int t = 0; t < cnt; ++t) {
                        const int pv = bp[t * 128 + tid];
                        if (pv < 0) continue;
                        const float dv = bd[t * 128 + tid];
                        if (best < 0 || dv < bdv || (dv == bdv && pv < bpv)) {
                            best = t;
                            bdv = dv;
                            bpv = pv;
                        }
                    }
                    out[k] = best >= 0 ? bpv : out[0];
                    if (best >= 0) bp[best * 128 + tid] = -1;
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
        k_match_tc<K><<<grid, 128, L.total, s>>>(a);
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
