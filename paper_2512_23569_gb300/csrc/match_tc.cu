// Block matching of the precision form (Alg. 1 step 1 with Eq. 9 planes) on
// the sm_103a tensor cores.
//
// For a reference a and a candidate b of the same matching plane,
//   ||a - b||^2 = ||a||^2 + ||b||^2 - 2 a.b,
// and the cross terms of a tile of 128 references (16 grid rows x 8 grid
// columns) against the candidate positions of the tile's search region form
// BF16 GEMMs with FP32 accumulation in tensor memory (tcgen05.mma kind::f16):
// the references are the MMA's M = 128 rows, so reference m's distances land
// in tensor-memory lane m.  No candidate matrix is materialised: the region is
// staged once as "row-8 vectors" Q[p] = plane[y_p][x_p .. x_p+7] (16 bytes,
// one core-matrix row), candidates are numbered p = y * Wq + x in the region
// (Wq >= Wc, the padding columns are never valid), and the K slice of patch
// rows (u, u+1) of the candidates p0 .. p0+63 is the shared-memory matrix
// starting at Q[p0 + u Wq], core matrices 8 rows (128 bytes) apart along N and
// Wq rows (16 Wq bytes) apart along K.
//
// Warp w reads lanes 32 (w % 4) .. + 31: the references of tile rows
// 4 (w % 4) .. + 3, whose search windows cover a band of the region's rows.
// Each run gives every lane quarter the next 64 candidates of its own band
// (four N = 64 MMAs into 256 tensor-memory columns), so all eight warps read
// 32 columns per run.  A thread turns its reference's 32 cross terms into
// keys (the distance's float bits with the low bits replaced by the
// candidate's index, so equal distances keep the lower index first; ~0 for a
// candidate outside the reference's window) and drops key i into bin i (K = 32:
// bin i mod 16), a sorted list of T slots, through a branch-free min / max network -- every
// lane and every warp does the same work in every run.  The smallest key a
// full bin pushed out is remembered.  A ninth warp issues the MMAs into two
// accumulators of 256 columns: a run goes into an accumulator once all eight
// warps have loaded the run before from it (mbarriers, no block-wide barrier
// per run), so the warps drift apart and the loads' latency hides.  At the end each
// thread keeps the LH smallest keys of its bins, the two threads of a
// reference (one per half of each run's columns) merge theirs, the LH
// smallest are re-ranked with FP32 distances of the FP32 plane, and the K-1
// smallest by (distance, raster index) follow the reference in its group.  If
// a pushed-out key lies below the (K+3)-th smallest kept one, the bins may
// have lost one of the nearest candidates: the reference goes to an
// exhaustive matcher with the re-rank's FP32 arithmetic, which rewrites its
// group (a few references in a thousand on natural-looking images; the row
// pitch of the candidate numbering is chosen so that the lines of equally
// good candidates along edges and stripes spread over the bins).  Eq. 9 picks the plane
// per reference: a colour tile runs once per plane that one of its
// references uses.
//
// Blocks take (tile, plane pass) items from a queue (an atomic counter), so
// the two passes of a colour tile run on two SMs.
//
// Every mbarrier wait is bounded; a wait that gives up records error code 2
// in the call's state, and the block waits (bounded) for the MMAs it has
// issued, gives the references of its item and of every item left in the
// queue their own position as their whole group (valid positions for the
// kernels that read the groups; the call reports HTS_ETIMEOUT where it reads
// the state back), releases its tensor memory and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "hts_internal.h"
#include "tc_ptx.h"

namespace hts {
namespace {

constexpr int TTY = 16, TTX = 8;  // reference tile (grid rows x grid columns)
constexpr int NR = TTY * TTX;     // references per tile = MMA M
constexpr int NQ = 4;             // lane quarters (tile rows 4q .. 4q+3)
constexpr int CH = 64;            // candidates per quarter and run = MMA N
constexpr int RUNC = NQ * CH;     // tensor-memory columns per run
constexpr int NBUF = 2;           // accumulators
constexpr uint32_t TMEM_COLS = NBUF * RUNC;
constexpr long long SPIN = 1ll << 24;
constexpr long long INJECT_SPIN = 1ll << 12;  // polls of the injected wait (hts_fault_inject "wait")
constexpr unsigned FULLM = 0xffffffffu;
constexpr int NWC = 8;               // reading warps: warp w takes lanes 32 (w % 4) .. + 31, columns 32 (w / 4) ..
constexpr int NT = (NWC + 1) * 32;   // + one warp that issues the MMAs

struct TcArgs {
    CUtensorMap tmap;  // the image as [C][H][W] FP32, box (tma_bw, tma_bh, 1): one channel's candidate region
    const float *img;
    int H, W, C, step, R, nx, ny, nref;
    int32_t *idx;
    const uint8_t *green;
    int32_t *fb;  // references for the exhaustive matcher (count in st->match_fallback)
    DevState *st;
    int ntx, nty, ntiles;
    int hc_max, wc_max;  // bounds of the candidate region over all tiles
    int inject_wait;     // 1: the issuing thread first waits, briefly, on a barrier nothing arrives on
    int use_tma;         // 1: the candidate region is staged by TMA (else by loads)
    int tma_bw, tma_bh;  // the TMA box: columns (a multiple of 4, from a column multiple of 4) and rows
};

// A launch over the images of a batch: jobs (device array of every image's arguments, staged by loads)
// and one work queue of (job, tile, plane pass) items; job j owns items item_start[j] .. item_start[j+1]-1.
struct TcBatch {
    const TcArgs *jobs;
    const int *item_start;
    int njobs, nitems;
    int *queue;          // the queue's counter (zero at the launch)
    int hc_max, wc_max;  // bounds of the candidate regions over the jobs
};

// LH: keys each thread keeps and the number re-ranked in FP32 per reference: the top 2K (at least K + 8);
// T: slots per bin; KC: the nearest keys that must all have been kept.
template <int K>
struct ListCfg {
    static constexpr int LH = 2 * K > K + 8 ? 2 * K : K + 8;
    static constexpr int NBIN = K <= 16 ? 32 : 16;  // key i goes into bin i mod NBIN
    static constexpr int T = K <= 16 ? 3 : 6;
    static constexpr int KC = K + 3;
    static_assert(KC <= LH, "the complete keys are re-ranked");
};

struct TcLayout {
    size_t q, a, e, ps, scr, ref, qr, bar, job, total;
};

__host__ __device__ inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-reference record in shared memory.
struct RefRec {
    int wy0, wy1, wx0, wx1;  // search window, region coordinates
    int pself, mine, pad0, pad1;
};

// Shared memory: Q (row-8 vectors), A (references), E (candidates' squared
// norms), the FP32 plane Ps, the row norms (only while E is formed),
// per-reference records, the quarters' candidate bands, barriers.  After the
// runs the final lists, re-rank keys and pushed-out minima overlay Q / A / E.
template <int K>
__host__ __device__ inline TcLayout tc_layout(int hc_max, int wc_max) {
    constexpr int LH = ListCfg<K>::LH;
    TcLayout L;
    const size_t wq_max = (size_t)wc_max + 7;  // largest row pitch of the candidate numbering
    const size_t ncand = (size_t)hc_max * wq_max;
    const size_t nq = ncand + CH + 7 * wq_max;
    L.q = 0;
    L.a = up(L.q + nq * 16, 1024);
    L.e = L.a + (size_t)NR * 64 * 2;
    L.ps = up(L.e + (ncand + CH) * 4, 16);
    const size_t fin_end = (size_t)LH * NR * 16 + (size_t)2 * NR * 4;  // [2][LH][NR] keys, [LH][NR] re-rank keys, [2][NR]
    if (L.ps < fin_end) L.ps = up(fin_end, 16);
    L.scr = up(L.ps + (size_t)(hc_max + 7) * (wc_max + 7) * 4, 16);
    L.ref = up(L.scr + nq * 4, 16);
    L.qr = L.ref + (size_t)NR * sizeof(RefRec);
    L.bar = up(L.qr + NQ * sizeof(int2), 16);
    L.job = up(L.bar + (2 * NBUF + 2) * 8 + 16, 64);  // the current job's arguments (batched launches)
    L.total = L.job + sizeof(TcArgs);
    // one block per SM, and never beside a block of the other tensor-core kernels (whose tensor
    // memory would not fit beside this block's 512 columns)
    if (L.total < 160 * 1024) L.total = 160 * 1024;
    return L;
}

using tc::sdesc;
using tc::su32;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half)
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Compare-exchange into ascending order.
__device__ __forceinline__ void cmpx(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
// Bitonic sequence v[B .. B + N) into ascending order.
template <int B, int N, int NP>
__device__ __forceinline__ void bitonic_clean(uint32_t (&v)[NP]) {
    constexpr int LN = ilog2c(N);
#pragma unroll
    for (int e = LN - 1; e >= 0; --e)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & (1 << e)) == 0) cmpx(v[B + i], v[B + i + (1 << e)]);
}
// One merge level: the ascending runs of length 2^L of v merged pairwise (the second reversed against the
// first makes both halves bitonic, then both are cleaned) into runs of length 2^(L+1).
template <int NP, int L>
__device__ __forceinline__ void merge_level(uint32_t (&v)[NP]) {
#pragma unroll
    for (int base = 0; base < NP; base += 2 << L) {
#pragma unroll
        for (int i = 0; i < (1 << L); ++i) cmpx(v[base + i], v[base + (2 << L) - 1 - i]);
#pragma unroll
        for (int e = L - 1; e >= 0; --e)
#pragma unroll
            for (int i = 0; i < (2 << L); ++i)
                if ((i & (1 << e)) == 0) cmpx(v[base + i], v[base + i + (1 << e)]);
    }
}
template <int NP, int L, int LE>
struct MergeLevels {
    static __device__ __forceinline__ void run(uint32_t (&v)[NP]) {
        merge_level<NP, L>(v);
        MergeLevels<NP, L + 1, LE>::run(v);
    }
};
template <int NP, int LE>
struct MergeLevels<NP, LE, LE> {
    static __device__ __forceinline__ void run(uint32_t (&)[NP]) {}
};
// The S smallest of v[NP] (NP / R ascending runs of length R, powers of two, S >= R) into v[0 .. S),
// ascending: runs merged up to length S, then the chunks of S folded into the first (element i against
// element S - 1 - i of the next chunk keeps the S smallest, as a bitonic sequence).  Only compile-time
// indices: the array stays in registers.
template <int NP, int R, int S>
__device__ __forceinline__ void smallest_sorted(uint32_t (&v)[NP]) {
    MergeLevels<NP, ilog2c(R), ilog2c(S)>::run(v);
#pragma unroll
    for (int c = 1; c < NP / S; ++c) {
#pragma unroll
        for (int i = 0; i < S; ++i) v[i] = min(v[i], v[c * S + S - 1 - i]);
        bitonic_clean<0, S, NP>(v);
    }
}

// Row pitch of the candidate numbering p = y * Wq + x: the value in [Wc, Wc + 7]
// whose key columns p mod 64 (bin and half of a thread's run) spread the
// points of the short lattice directions (dy <= 4, |dx| <= 4) over the most
// cells, weighted by the direction's length -- equally good candidates along
// an edge or a stripe must not crowd into one bin.  Lanes 0..7 of every warp
// score one pitch each.
__device__ __forceinline__ int pick_pitch(int Wc, int lane) {
    const int w = Wc + (lane & 7);
    unsigned sc = 0xffffffffu;
    for (int dy = 0; dy <= 4; ++dy)
        for (int dx = -4; dx <= 4; ++dx) {
            if (dy == 0 && dx <= 0) continue;
            const int d = (dy * w + dx) & 63;
            const int cells = d ? (64 >> (__ffs(d) - 1)) : 1;
            sc = min(sc, (unsigned)(cells * cells) * (unsigned)(dy * dy + dx * dx));
        }
    unsigned key = (sc << 3) | (unsigned)(7 - (lane & 7));  // the highest score, then the smallest pitch
#pragma unroll
    for (int o = 16; o; o >>= 1) key = max(key, __shfl_xor_sync(FULLM, key, o));
    return Wc + 7 - (int)(key & 7u);
}

// Group of reference r made of its own position `self` only (the failure path: valid positions for the
// kernels that read the groups).
template <int K>
__device__ __forceinline__ void self_group(const TcArgs &a, int r, int self) {
    int32_t *out = a.idx + (size_t)r * K;
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = self;
}

// BATCH: the items of every job of `bt` (a0 unused); else the items of the one image a0 (bt unused).
template <int K, bool BATCH>
__global__ void __launch_bounds__(NT, 1) k_match_tc(const __grid_constant__ TcArgs a0,
                                                    const __grid_constant__ TcBatch bt) {
    constexpr int LH = ListCfg<K>::LH, T = ListCfg<K>::T, KC = ListCfg<K>::KC, NBIN = ListCfg<K>::NBIN;
    constexpr int TP = T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : 8;                   // slots per bin, padded
    constexpr int LS = LH <= 8 ? 8 : LH <= 16 ? 16 : LH <= 32 ? 32 : 64;           // sorted list length >= LH
    static_assert(T <= 8 && LH <= 64 && LS >= TP && (NBIN * TP) % LS == 0, "top-list network shape");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const TcLayout L = tc_layout<K>(BATCH ? bt.hc_max : a0.hc_max, BATCH ? bt.wc_max : a0.wc_max);
    TcArgs *sjob = reinterpret_cast<TcArgs *>(smem_raw + L.job);
    uint4 *Q = reinterpret_cast<uint4 *>(smem_raw + L.q);
    unsigned char *Abuf = smem_raw + L.a;
    float *E = reinterpret_cast<float *>(smem_raw + L.e);
    float *Ps = reinterpret_cast<float *>(smem_raw + L.ps);
    float *rn = reinterpret_cast<float *>(smem_raw + L.scr);  // row norms (E formation)
    uint32_t *fk = reinterpret_cast<uint32_t *>(smem_raw);     // final lists [2][LH][NR]
    unsigned long long *fr = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)2 * LH * NR * 4);
    uint32_t *fe = reinterpret_cast<uint32_t *>(smem_raw + (size_t)LH * NR * 16);  // pushed-out minima [2][NR]
    RefRec *rec = reinterpret_cast<RefRec *>(smem_raw + L.ref);
    int2 *qr = reinterpret_cast<int2 *>(smem_raw + L.qr);  // per quarter: first candidate, count
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L.bar);  // [NBUF]: the run's MMAs completed
    uint64_t *empty = full + NBUF;                                    // [NBUF]: every warp loaded the run
    uint64_t *never = empty + NBUF;  // no thread arrives on it (the injected wait)
    uint64_t *tbar = never + 1;      // the TMA copies of an item's region landed
    int *abort_flag = reinterpret_cast<int *>(tbar + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(abort_flag + 1);
    int *item_slot = reinterpret_cast<int *>(tmem_slot + 1);  // the block's current work item

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool cw = warp < NWC;              // a reading warp
    const int q = warp & 3, hh = (warp >> 2) & 1;  // lane quarter, half of the quarter's 64 columns
    const int m = 32 * q + lane;            // this thread's reference slot (A row, tensor-memory lane)
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            tc::bar_init(&full[b], 1);
            tc::bar_init(&empty[b], NWC);
        }
        tc::bar_init(never, 1);
        tc::bar_init(tbar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tmem_slot;
    const uint32_t idesc = tc::idesc_f16(NR, CH, true);
    long long gc = 0;  // runs issued by this block so far (accumulator gc % NBUF, use gc / NBUF)
    uint32_t tphase = 0;  // TMA stagings so far (the parity of tbar's next phase)
    volatile int *abortp = abort_flag;
    bool ok = true;

    int cur_job = -1;
    while (true) {
        // next item of the work queue: (tile, plane pass), so that the two passes of a colour tile run
        // on two SMs and blocks that drew passes without references move on at once.  The fence orders this
        // thread's earlier shared-memory accesses before the next item's TMA writes into the same area.
        tc::fence_async_smem();
        if (tid == 0) *item_slot = atomicAdd(BATCH ? bt.queue : &a0.st->mtc_next, 1);
        __syncthreads();
        int item = *item_slot;
        __syncthreads();
        if (BATCH) {
            if (item >= bt.nitems) break;
            int lo = 0, hi = bt.njobs - 1;  // the job owning the item: the last j with item_start[j] <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bt.item_start[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            item -= bt.item_start[lo];
            if (lo != cur_job) {  // the job's arguments into shared memory (every thread reads them below)
                const int *src = reinterpret_cast<const int *>(bt.jobs + lo);
                int *dst = reinterpret_cast<int *>(sjob);
                for (int w = tid; w < (int)(sizeof(TcArgs) / 4); w += NT) dst[w] = src[w];
                cur_job = lo;
                __syncthreads();
            }
        }
        const TcArgs &a = BATCH ? *sjob : a0;
        const int npass = (a.C == 3) ? 2 : 1;
        const size_t HW = (size_t)a.H * a.W;
        if (!BATCH && item >= a.ntiles * npass) break;
        const int tile = item / npass;
        const int tyi = tile / a.ntx, txi = tile - tyi * a.ntx;
        const int gy0 = tyi * TTY, gx0 = txi * TTX;
        const int gy1 = min(a.ny, gy0 + TTY) - 1, gx1 = min(a.nx, gx0 + TTX) - 1;
        const int cy0 = max(0, grid_pos(gy0, a.H, a.step) - a.R);
        const int cy1 = min(a.H - PS, grid_pos(gy1, a.H, a.step) + a.R);
        const int cx0 = max(0, grid_pos(gx0, a.W, a.step) - a.R);
        const int cx1 = min(a.W - PS, grid_pos(gx1, a.W, a.step) + a.R);
        const int Hc = cy1 - cy0 + 1, Wc = cx1 - cx0 + 1, PSW = Wc + 7;
        const int Wq = pick_pitch(Wc, lane);  // row pitch of the candidate numbering
        const int ncand = Hc * Wq;
        const int nq = ncand + CH + 7 * Wq;
        const uint32_t lowm = (1u << (32 - __clz(ncand))) - 1u;  // candidate index bits of a key
        const uint32_t him = ~lowm;

        {
            const int pass = item - tile * npass;
            // ---- per-reference records (thread j < NR: reference j = tile row j / 8, column j % 8),
            //      and each quarter's band of candidate rows
            bool any = false;
            if (tid < NR) {
                const int ry = gy0 + (tid >> 3), rx = gx0 + (tid & 7);
                const bool valid = ry <= gy1 && rx <= gx1;
                const int r = valid ? ry * a.nx + rx : 0;
                const bool mine = valid && (a.C == 1 || (int)a.green[r] == (pass == 0 ? 1 : 0));
                const int yr = grid_pos(min(ry, gy1), a.H, a.step), xr = grid_pos(min(rx, gx1), a.W, a.step);
                RefRec rq;
                rq.wy0 = max(0, yr - a.R) - cy0;
                rq.wy1 = min(a.H - PS, yr + a.R) - cy0;
                rq.wx0 = max(0, xr - a.R) - cx0;
                rq.wx1 = min(a.W - PS, xr + a.R) - cx0;
                rq.pself = (yr - cy0) * Wq + (xr - cx0);
                rq.mine = mine ? 1 : 0;
                rq.pad0 = rq.pad1 = 0;
                rec[tid] = rq;
                any = mine;
                int lo = mine ? rq.wy0 : 0x3fffffff, hi = mine ? rq.wy1 : -1;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(FULLM, lo, o));
                    hi = max(hi, __shfl_xor_sync(FULLM, hi, o));
                }
                if (lane == 0) {
                    const int s0 = (hi < 0) ? 0 : ((lo * Wq) & ~31);
                    qr[warp] = make_int2(s0, (hi < 0) ? 0 : (hi + 1) * Wq - s0);
                }
            }
            if (!__syncthreads_or(any)) continue;
            // the failure path: the references of this item and of every item left in the queue get the
            // group of the reference alone, so that the kernels after this one read valid positions only
            auto self_groups = [&]() {
                if (tid < NR && rec[tid].mine) {
                    const int py = rec[tid].pself / Wq, px = rec[tid].pself - py * Wq;
                    self_group<K>(a, (gy0 + (tid >> 3)) * a.nx + gx0 + (tid & 7), (cy0 + py) * a.W + cx0 + px);
                }
            };
            if (!ok) {
                self_groups();
                continue;
            }
            // ---- stage the plane (FP32), the row-8 vectors and their norms, E, A
            if (a.use_tma) {
                // the channels the plane needs, each a box of the image from column cx0 rounded down to a
                // multiple of 4 (16 bytes), into the free area of Q; zero outside the image
                const int nch = (a.C == 3 && pass == 1) ? 3 : 1;  // pass 1: R + G + B
                const int ch0 = (a.C == 3 && pass == 0) ? 1 : 0;
                const int xs = cx0 & 3, bsz = (a.tma_bw * a.tma_bh + 31) & ~31;  // 128-byte aligned boxes
                float *stg = reinterpret_cast<float *>(smem_raw + L.q);
                if (tid == 0) {
                    tc::bar_arrive_expect_tx(tbar, (uint32_t)(nch * a.tma_bw * a.tma_bh * 4));  // the boxes' bytes
                    for (int c = 0; c < nch; ++c)
                        tc::tma_load_3d(stg + c * bsz, &a.tmap, tbar, cx0 - xs, cy0, ch0 + c);
                }
                const bool landed = tc::bar_wait_or_abort(tbar, (uint32_t)(tphase & 1), SPIN, abortp);
                ++tphase;
                if (!__all_sync(FULLM, landed)) {
                    // the copy must land before the area is used again; the item fails as a bounded wait does
                    if (tid == 0) tc::bar_wait(tbar, (uint32_t)((tphase - 1) & 1), SPIN);
                }
                if (__syncthreads_or(*abortp)) {
                    if (tid == 0) atomicExch(&a.st->error, 2);
                    ok = false;
                    self_groups();
                    continue;
                }
#pragma unroll 4
                for (int e = tid; e < (Hc + 7) * PSW; e += NT) {
                    const int y = e / PSW, x = e - y * PSW;
                    const int o = y * a.tma_bw + x + xs;
                    Ps[e] = (nch == 1) ? stg[o] : (stg[o] + stg[bsz + o]) + stg[2 * bsz + o];
                }
            } else {
#pragma unroll 4
                for (int e = tid; e < (Hc + 7) * PSW; e += NT) {
                    const int y = e / PSW, x = e - y * PSW;
                    const size_t o = (size_t)(cy0 + y) * a.W + cx0 + x;
                    float v;
                    if (a.C == 1) v = __ldg(a.img + o);
                    else if (pass == 0) v = __ldg(a.img + HW + o);
                    else v = (__ldg(a.img + o) + __ldg(a.img + HW + o)) + __ldg(a.img + 2 * HW + o);
                    Ps[e] = v;
                }
            }
            __syncthreads();
            for (int qi = tid; qi < nq; qi += NT) {
                const int y = qi / Wq, x = qi - y * Wq;
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                float n2 = 0.f;
                if (y < Hc + 7 && x < Wc) {
                    const float *s = Ps + y * PSW + x;
#pragma unroll
                    for (int v = 0; v < PS; ++v) {
                        const float b = bf_round(s[v]);
                        n2 = fmaf(b, b, n2);
                    }
                    w = make_uint4(pack_bf16(s[0], s[1]), pack_bf16(s[2], s[3]), pack_bf16(s[4], s[5]),
                                   pack_bf16(s[6], s[7]));
                }
                Q[qi] = w;
                rn[qi] = n2;  // squared norm of the BF16 row-8 vector
            }
            __syncthreads();
            for (int p = tid; p < ncand + CH; p += NT) {
                float e2 = 0.f;
                if (p < ncand) {
#pragma unroll
                    for (int u = 0; u < PS; ++u) e2 += rn[p + u * Wq];
                }
                E[p] = e2;
            }
            // A: row j = reference j, element 8u+v; core matrix (j/8, u) at (j/8)*1024 + u*128
            for (int e = tid; e < NR * PS; e += NT) {
                const int j = e >> 3, u = e & 7;
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                if ((gy0 + (j >> 3)) <= gy1 && (gx0 + (j & 7)) <= gx1 &&
                    HTS_IN_BOUNDS(rec[j].pself + u * Wq < nq, &a.st->error))
                    w = Q[rec[j].pself + u * Wq];
                *reinterpret_cast<uint4 *>(Abuf + (j >> 3) * 1024 + u * 128 + (j & 7) * 16) = w;
            }
            tc::fence_async_smem();
            __syncthreads();

            // ---- this thread's reference
            const RefRec rq = rec[m];
            const bool mine = cw && rq.mine != 0;
            const int ay = rq.pself / Wq, ax = rq.pself - ay * Wq;
            const float a2 = E[rq.pself];

            // ---- runs: quarter qq's next CH candidates into columns qq*CH of the accumulator
            int2 band[NQ];
            int nrun = 0;
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                band[qq] = qr[qq];
                nrun = max(nrun, (band[qq].y + CH - 1) / CH);
            }
            const long long g0 = gc;
            auto issue = [&](int c) {
                const uint32_t b = (uint32_t)((g0 + c) % NBUF);
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) {
                    if (c * CH >= band[qq].y) continue;
                    const uint4 *qb = Q + band[qq].x + c * CH;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = sdesc(su32(Abuf) + kk * 256, 128, 1024);
                        const uint64_t bd = sdesc(su32(qb + (size_t)2 * kk * Wq), 16u * Wq, 128);
                        tc::mma_f16(tbase + b * RUNC + qq * CH, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                }
                tc::mma_commit(&full[b]);
            };
            uint32_t bn[NBIN][T];  // bin g: the T smallest keys of the columns g mod NBIN of this thread's half-runs
#pragma unroll
            for (int g = 0; g < NBIN; ++g)
#pragma unroll
                for (int t = 0; t < T; ++t) bn[g][t] = 0xffffffffu;
            uint32_t ev = 0xffffffffu;  // smallest key a full bin pushed out
            if (!cw) {  // the issuing warp: run c goes into its accumulator once run c - NBUF was loaded by all
                if (lane == 0) {
                    int issued = 0;
                    // fault injection: before issuing anything the thread waits on a barrier nothing
                    // arrives on; the bounded wait gives up and sets the abort flag (no MMA in flight)
                    const bool injected =
                        a.inject_wait && g0 == 0 && !tc::bar_wait_or_abort(never, 0u, INJECT_SPIN, abortp);
                    for (int c = 0; c < nrun && !injected; ++c) {
                        const long long g = g0 + c;
                        const uint32_t b = (uint32_t)(g % NBUF);
                        if (g >= NBUF &&
                            !tc::bar_wait_or_abort(&empty[b], (uint32_t)(((g / NBUF) - 1) & 1), SPIN, abortp))
                            break;
                        tc::fence_after();
                        issue(c);
                        ++issued;
                    }
                    if (*abortp && issued > 0) {  // drain: the last issued run completes after every earlier one
                        const long long gl = g0 + issued - 1;
                        tc::bar_wait(&full[gl % NBUF], (uint32_t)((gl / NBUF) & 1), SPIN);
                    }
                }
                __syncwarp();
            } else {
                const int start = band[q].x, len = band[q].y;
                int ry = (start + 32 * hh) / Wq, rx = start + 32 * hh - ry * Wq;  // region row / column of pb
                for (int c = 0; c < nrun; ++c) {
                    const long long g = g0 + c;
                    const uint32_t b = (uint32_t)(g % NBUF);
                    const bool got = tc::bar_wait_or_abort(&full[b], (uint32_t)((g / NBUF) & 1), SPIN, abortp);
                    if (!__all_sync(FULLM, got)) break;
                    const int off = c * CH + 32 * hh;
                    const bool act = off < len;
                    const int pb = start + off;  // a multiple of 32
                    uint32_t v[32];
                    uint32_t vm = 0u;  // candidates pb .. pb+31 inside the window, without the reference
                    if (act) {
                        tc::fence_after();
                        tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + b * RUNC + q * CH + 32 * hh, v);
                        if (mine) {
                            for (int y = ry, rs = pb - rx; rs <= pb + 31 && y <= rq.wy1; ++y, rs += Wq) {
                                if (y < rq.wy0) continue;
                                const int lo = max(rs + rq.wx0, pb), hi = min(rs + rq.wx1, pb + 31);
                                if (lo <= hi) {
                                    const int n = hi - lo + 1;
                                    vm |= (n >= 32 ? FULLM : ((1u << n) - 1u)) << (lo - pb);
                                }
                            }
                            if ((unsigned)(rq.pself - pb) < 32u) vm &= ~(1u << (rq.pself - pb));
                        }
                        __syncwarp();
                        tc::tmem_wait_ld(v);
                    }
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::bar_arrive(&empty[b]);  // this warp is done with accumulator b
                    if (act && __any_sync(FULLM, vm != 0u)) {
                        const float4 *E4 = reinterpret_cast<const float4 *>(E + pb);
#pragma unroll
                        for (int i4 = 0; i4 < 8; ++i4) {
                            const float4 e4 = E4[i4];
                            const float evl[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                            for (int l = 0; l < 4; ++l) {
                                const int i = 4 * i4 + l;
                                const float d = fmaf(-2.f, __uint_as_float(v[i]), a2 + evl[l]);
                                uint32_t key = (__float_as_uint(fmaxf(d, 0.f)) & him) | (uint32_t)(pb + i);
                                key = (vm & (1u << i)) ? key : 0xffffffffu;
                                uint32_t *bb = bn[i % NBIN];
                                ev = min(ev, max(bb[T - 1], key));
                                // every slot from the old bin alone: no dependent chain
#pragma unroll
                                for (int t = T - 1; t > 0; --t) bb[t] = max(bb[t - 1], min(bb[t], key));
                                bb[0] = min(bb[0], key);
                            }
                        }
                    }
                    rx += CH;
                    while (rx >= Wq) {
                        rx -= Wq;
                        ++ry;
                    }
                }
            }
            __syncthreads();  // every run was loaded (or the block gave up): Q, A, E are free
            if (*abortp) {
                if (tid == 0) atomicExch(&a.st->error, 2);
                ok = false;
                self_groups();
                continue;
            }
            gc = g0 + nrun;

            // ---- the LH smallest keys of this thread's bins, both threads' lists and pushed-out minima to
            //      shared memory (every MMA has completed: Q, A, E are free)
            if (cw) {
                uint32_t v[NBIN * TP];  // bin g's slots ascending at g * TP, padded with ~0
#pragma unroll
                for (int g = 0; g < NBIN; ++g)
#pragma unroll
                    for (int s = 0; s < TP; ++s) v[g * TP + s] = s < T ? bn[g][s] : 0xffffffffu;
                smallest_sorted<NBIN * TP, TP, LS>(v);
#pragma unroll
                for (int t = 0; t < LH; ++t) fk[(hh * LH + t) * NR + m] = v[t];
                fe[hh * NR + m] = ev;
            }
            __syncthreads();
            // ---- merged LH smallest keys, FP32 distances of the FP32 plane in the definition's (u, v)
            //      order (the two threads take alternate entries); the reference goes to the exhaustive
            //      matcher if a pushed-out key lies below the KC-th smallest kept key
            bool lost = false;
            if (mine) {
                float ra[PS * PS];
#pragma unroll
                for (int u = 0; u < PS; ++u)
#pragma unroll
                    for (int v = 0; v < PS; ++v) ra[u * PS + v] = Ps[(ay + u) * PSW + ax + v];
                const uint32_t evm = min(fe[m], fe[NR + m]);
                int i0 = 0, i1 = 0;
                for (int t = 0; t < LH; ++t) {
                    const uint32_t k0 = i0 < LH ? fk[i0 * NR + m] : 0xffffffffu;
                    const uint32_t k1 = i1 < LH ? fk[(LH + i1) * NR + m] : 0xffffffffu;
                    uint32_t k;
                    if (k0 <= k1) {
                        k = k0;
                        ++i0;
                    } else {
                        k = k1;
                        ++i1;
                    }
                    if (t == KC - 1) lost = evm < k;
                    if ((t & 1) != hh) continue;
                    unsigned long long rk = ~0ull;
                    if (k != 0xffffffffu) {
                        const int p = (int)(k & lowm);
                        const int by = p / Wq, bx = p - by * Wq;
                        if (!HTS_IN_BOUNDS(by < Hc && bx < Wc, &a.st->error)) continue;
                        const float *pbv = Ps + by * PSW + bx;
                        float d = 0.f;
#pragma unroll
                        for (int u = 0; u < PS; ++u)
#pragma unroll
                            for (int v = 0; v < PS; ++v) {
                                const float df = ra[u * PS + v] - pbv[u * PSW + v];
                                d = fmaf(df, df, d);
                            }
                        rk = ((unsigned long long)__float_as_uint(d) << 32) |
                             (uint32_t)((cy0 + by) * a.W + cx0 + bx);
                    }
                    fr[(size_t)t * NR + m] = rk;
                }
            }
            __syncthreads();
            // ---- the K-1 smallest by (distance, raster index)
            if (hh == 0 && mine) {
                unsigned long long sel[K - 1];
#pragma unroll
                for (int i = 0; i < K - 1; ++i) sel[i] = ~0ull;
                for (int t = 0; t < LH; ++t) {
                    const unsigned long long k = fr[(size_t)t * NR + m];
#pragma unroll
                    for (int i = K - 2; i > 0; --i) {
                        const unsigned long long lo = k < sel[i] ? k : sel[i];
                        sel[i] = sel[i - 1] > lo ? sel[i - 1] : lo;
                    }
                    sel[0] = k < sel[0] ? k : sel[0];
                }
                const int r = (gy0 + (m >> 3)) * a.nx + gx0 + (m & 7);
                const int self = (cy0 + ay) * a.W + cx0 + ax;
                int32_t *out = a.idx + (size_t)r * K;
                out[0] = self;
#pragma unroll
                for (int i = 0; i < K - 1; ++i) out[i + 1] = (sel[i] == ~0ull) ? self : (int)(uint32_t)sel[i];
                if (lost) a.fb[atomicAdd(&a.st->match_fallback, 1)] = r;
            }
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

template <int K>
hts_status launch_tc(const TcArgs &a, cudaStream_t s) {
    const TcLayout L = tc_layout<K>(a.hc_max, a.wc_max);
    const hts_status st0 = allow_smem(reinterpret_cast<const void *>(k_match_tc<K, false>), L.total);
    if (st0 != HTS_OK) return st0;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int items = a.ntiles * (a.C == 3 ? 2 : 1);
    const int grid = std::max(1, std::min(items, nsm));
    if (cudaMemsetAsync(&a.st->mtc_next, 0, sizeof(int), s) != cudaSuccess) return check_launch("cudaMemsetAsync");
    TcBatch none{};
    {
        KTimer kt("k_match_tc", s);
        k_match_tc<K, false><<<grid, NT, L.total, s>>>(a, none);
    }
    return check_launch("k_match_tc");
}

template <int K>
hts_status launch_tc_batch(const TcBatch &bt, int grid, cudaStream_t s) {
    const TcLayout L = tc_layout<K>(bt.hc_max, bt.wc_max);
    const hts_status st0 = allow_smem(reinterpret_cast<const void *>(k_match_tc<K, true>), L.total);
    if (st0 != HTS_OK) return st0;
    if (cudaMemsetAsync(bt.queue, 0, sizeof(int), s) != cudaSuccess) return check_launch("cudaMemsetAsync");
    TcArgs none{};
    {
        KTimer kt("k_match_tc", s);
        k_match_tc<K, true><<<grid, NT, L.total, s>>>(none, bt);
    }
    return check_launch("k_match_tc");
}

}  // namespace

size_t match_tc_job_size() { return sizeof(TcArgs); }

int match_tc_job(const float *img, const Geom &g, int32_t *idx, const uint8_t *green, int32_t *fallback_list,
                 DevState *st, void *job) {
    TcArgs a{};
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
    a.fb = fallback_list;
    a.st = st;
    a.nty = (g.ny + TTY - 1) / TTY;
    a.ntx = (g.nx + TTX - 1) / TTX;
    a.ntiles = a.nty * a.ntx;
    a.hc_max = std::min(g.H - PS + 1, (TTY - 1) * g.step + 1 + 2 * g.R);
    a.wc_max = std::min(g.W - PS + 1, (TTX - 1) * g.step + 1 + 2 * g.R);
    a.use_tma = 0;  // the job table lives in global memory: regions staged by loads
    std::memcpy(job, &a, sizeof(TcArgs));
    return a.ntiles * (g.C == 3 ? 2 : 1);
}

hts_status launch_match_tc_batch(int K, const void *jobs_host, const void *jobs_dev, const int *item_start_dev,
                                 int njobs, int nitems, int *queue_dev, int grid, cudaStream_t s) {
    TcBatch bt{};
    bt.jobs = static_cast<const TcArgs *>(jobs_dev);
    bt.item_start = item_start_dev;
    bt.njobs = njobs;
    bt.nitems = nitems;
    bt.queue = queue_dev;
    const TcArgs *jh = static_cast<const TcArgs *>(jobs_host);
    for (int j = 0; j < njobs; ++j) {
        bt.hc_max = std::max(bt.hc_max, jh[j].hc_max);
        bt.wc_max = std::max(bt.wc_max, jh[j].wc_max);
    }
    grid = std::max(1, std::min(grid, nitems));
    switch (K) {
        case 2: return launch_tc_batch<2>(bt, grid, s);
        case 4: return launch_tc_batch<4>(bt, grid, s);
        case 8: return launch_tc_batch<8>(bt, grid, s);
        case 16: return launch_tc_batch<16>(bt, grid, s);
        case 32: return launch_tc_batch<32>(bt, grid, s);
        default: return HTS_EUNSUPPORTED;
    }
}

hts_status launch_match_tc(const float *img, const Geom &g, double gamma_gcp, int32_t *idx, const uint8_t *green,
                           int32_t *fallback_list, DevState *st, cudaStream_t s) {
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
    a.fb = fallback_list;
    a.st = st;
    a.nty = (g.ny + TTY - 1) / TTY;
    a.ntx = (g.nx + TTX - 1) / TTX;
    a.ntiles = a.nty * a.ntx;
    a.hc_max = std::min(g.H - PS + 1, (TTY - 1) * g.step + 1 + 2 * g.R);
    a.wc_max = std::min(g.W - PS + 1, (TTX - 1) * g.step + 1 + 2 * g.R);
    a.inject_wait = (!stream_capturing(s) && fault_take(FAULT_WAIT)) ? 1 : 0;
    // TMA staging of the candidate regions: one channel's region is a box of the image tensor [C][H][W]
    // starting at a column multiple of 4 (16 bytes), so the box is 3 columns wider than the widest region;
    // used where the rows are 16-byte multiples and the boxes of all channels fit in the area of Q
    a.use_tma = 0;
    a.tma_bw = ((a.wc_max + 7 + 3) + 3) & ~3;
    a.tma_bh = a.hc_max + 7;
    std::memset(&a.tmap, 0, sizeof(a.tmap));
    {
        size_t qarea = 0;
        switch (g.K) {
            case 2: qarea = tc_layout<2>(a.hc_max, a.wc_max).a; break;
            case 4: qarea = tc_layout<4>(a.hc_max, a.wc_max).a; break;
            case 8: qarea = tc_layout<8>(a.hc_max, a.wc_max).a; break;
            case 16: qarea = tc_layout<16>(a.hc_max, a.wc_max).a; break;
            default: qarea = tc_layout<32>(a.hc_max, a.wc_max).a; break;
        }
        const size_t box = (size_t)((a.tma_bw * a.tma_bh + 31) & ~31) * 4;
        const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
        if (enc && g.W % 4 == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0 && a.tma_bw <= 256 &&
            a.tma_bh <= 256 && (size_t)g.C * box <= qarea) {
            const cuuint64_t dims[3] = {(cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.C};
            const cuuint64_t strides[2] = {(cuuint64_t)g.W * 4, (cuuint64_t)g.H * g.W * 4};
            const cuuint32_t boxd[3] = {(cuuint32_t)a.tma_bw, (cuuint32_t)a.tma_bh, 1};
            const cuuint32_t estr[3] = {1, 1, 1};
            if (enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(img), dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
                a.use_tma = 1;
        }
    }
    hts_status st0 = HTS_EUNSUPPORTED;
    switch (g.K) {
        case 2: st0 = launch_tc<2>(a, s); break;
        case 4: st0 = launch_tc<4>(a, s); break;
        case 8: st0 = launch_tc<8>(a, s); break;
        case 16: st0 = launch_tc<16>(a, s); break;
        case 32: st0 = launch_tc<32>(a, s); break;
        default: break;
    }
    if (st0 != HTS_OK) return st0;
    return launch_match_rescue(img, g, idx, green, fallback_list, st, s);
}

}  // namespace hts
