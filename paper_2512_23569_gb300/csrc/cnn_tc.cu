// Tensor-core forward pass of the learned noise-level network (the
// convolutional estimate of the adaptive variant, Sec. III-C), used when
// denoising.
//
// A 3x3 convolution with zero padding is an implicit GEMM: for every tap
// (ky, kx), out[p][n] += sum_c in[p + (ky - 1, kx - 1)][c] w[n][c][ky][kx].
// A block takes a strip of 16 x 64 output pixels and stages its input with a
// one-pixel halo in shared memory as planes of 8 channels: entry (g, py, px)
// is the 16-byte vector of channels 8g .. 8g + 7 of one pixel.  Eight 16 x 8
// pixel tiles of the strip are the MMA's M = 128 rows (tile row i = 8
// consecutive pixels of output row i, one core matrix), so the A operand of
// tap (ky, kx) is the staged region itself, its descriptor starting ky rows
// and kx pixels further on: core matrices one staged row apart along M and
// one channel plane apart along K.  No im2col copy is made.  B holds the
// layer's FP16 weights per tap (N = 32 output channels, or 16 of which one
// is used for the last layer); each tile accumulates 9 taps x (input
// channels / 16) MMAs of kind::f16 in its own 32 (16) tensor-memory columns.
// The epilogue reads a tile row per thread (tcgen05.ld), adds the bias,
// applies ReLU and writes FP16 planes for the next layer, or the FP32 log
// sigma map after the last layer.
//
// Layers: 0: image / 255 (rounded to FP16, channels padded to 16) -> 32;
// 1..3: 32 -> 32; 4: 32 -> 1.  Every mbarrier wait is bounded; a wait that
// gives up sets the network's error flag, the block waits (bounded) for its
// MMAs and releases its tensor memory, and the map is then filled with NaN
// so that the learned-map check falls back to the estimate.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cnn_internal.h"
#include "hts_internal.h"
#include "tc_ptx.h"

namespace hts {
namespace {

constexpr int SY = 16;                   // output rows of a strip
constexpr int MT = 8;                    // 16 x 8 pixel tiles (MMA M = 128) per strip
constexpr int SX = 8 * MT;               // output columns of a strip
constexpr int PY = SY + 2, PX = SX + 2;  // staged rows and columns (halo of one pixel)
constexpr int NTH = 256;                 // 8 warps; warp w reads tensor-memory lanes 32 (w % 4) .. + 31
constexpr long long SPIN = 1ll << 22;
// At least this much shared memory per block: at most two blocks per SM, so
// their tensor memory (at most 2 x 256 columns) is always free to allocate.
constexpr size_t MIN_SMEM = 80 * 1024;

template <int CING, int NOUT>
struct ConvTcLayout {
    static constexpr size_t a_bytes = (size_t)CING * PY * PX * 16;  // staged input planes
    static constexpr size_t b_off = a_bytes;
    static constexpr size_t b_bytes = (size_t)9 * CING * NOUT * 16;  // weights [tap][plane][n][8]
    static constexpr size_t bias_off = b_off + b_bytes;
    static constexpr size_t bar_off = bias_off + (size_t)NOUT * 4;
    static constexpr size_t slot_off = bar_off + 16;
    static constexpr size_t used = slot_off + 16;
    static constexpr size_t total = used > MIN_SMEM ? used : MIN_SMEM;
    static constexpr uint32_t tcols = MT * NOUT;  // 256 or 128
};

// CING: input planes of 8 channels (2 for layer 0, whose C <= 3 channels
// occupy plane 0 and plane 1 is zero; 4 otherwise).  NOUT: MMA N.
// IN_F32: the input is the FP32 image (planar C x H x W, scaled by 1/255);
// otherwise FP16 planes hin[g][y][x][8].  OUT_MAP: write column 0 plus bias
// to the FP32 map; otherwise ReLU, FP16 planes hout[g][y][x][8].
template <int CING, int NOUT, bool IN_F32, bool OUT_MAP>
__global__ void __launch_bounds__(NTH, 1)
    k_conv_tc(const float *__restrict__ img, int C, const __half *__restrict__ hin, int H, int W,
              const __half *__restrict__ wt, int cin, int cout, __half *__restrict__ hout, float *__restrict__ map,
              int *err) {
    using L = ConvTcLayout<CING, NOUT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *sA = reinterpret_cast<uint4 *>(smem);
    __half *sB = reinterpret_cast<__half *>(smem + L::b_off);
    float *sBias = reinterpret_cast<float *>(smem + L::bias_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + L::slot_off);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights B[tap][g][n][k] = w[n][8 g + k][tap], zero outside the layer's channels
    for (int e = tid; e < 9 * CING * NOUT * 8; e += NTH) {
        const int k = e & 7, rest = e >> 3;
        const int n = rest % NOUT, g = (rest / NOUT) % CING, tap = rest / (NOUT * CING);
        const int ci = g * 8 + k;
        sB[e] = (n < cout && ci < cin) ? wt[(n * cin + ci) * 9 + tap] : __float2half_rn(0.f);
    }
    for (int n = tid; n < NOUT; n += NTH) sBias[n] = n < cout ? __half2float(wt[cout * cin * 9 + n]) : 0.f;
    if (tid == 0) {
        tc::bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(slot, L::tcols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idesc = tc::idesc_f16(128, NOUT, false);
    const int nsx = (W + SX - 1) / SX, nstrip = ((H + SY - 1) / SY) * nsx;
    const size_t HW = (size_t)H * W;
    uint32_t phase = 0;

    for (int strip = blockIdx.x; strip < nstrip; strip += gridDim.x) {
        const int y0 = (strip / nsx) * SY, x0 = (strip % nsx) * SX;
        // ---- stage the input planes with the halo (zero outside the image)
        for (int e = tid; e < CING * PY * PX; e += NTH) {
            const int g = e / (PY * PX), r = e - g * (PY * PX), py = r / PX, px = r - py * PX;
            const int y = y0 - 1 + py, x = x0 - 1 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (y >= 0 && y < H && x >= 0 && x < W) {
                if (IN_F32) {
                    if (g == 0) {
                        __align__(16) __half h[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            h[c] = __float2half_rn(c < C ? img[c * HW + (size_t)y * W + x] * (1.f / 255.f) : 0.f);
                        v = *reinterpret_cast<const uint4 *>(h);
                    }
                } else {
                    v = reinterpret_cast<const uint4 *>(hin)[((size_t)g * H + y) * W + x];
                }
            }
            sA[e] = v;
        }
        tc::fence_async_smem();
        __syncthreads();
        // ---- MMAs (one thread): tile j, tap (ky, kx), K step s = planes 2s, 2s + 1
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::su32(sA), b0 = tc::su32(sB);
            for (int j = 0; j < MT; ++j)
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int s = 0; s < CING / 2; ++s) {
                        const uint32_t aoff = (uint32_t)((((2 * s) * PY + ky) * PX + 8 * j + kx) * 16);
                        const uint32_t boff = (uint32_t)((tap * CING + 2 * s) * NOUT * 16);
                        const uint64_t ad = tc::sdesc(a0 + aoff, PY * PX * 16, PX * 16);
                        const uint64_t bd = tc::sdesc(b0 + boff, NOUT * 16, 128);
                        tc::mma_f16(tbase + j * NOUT, ad, bd, idesc, (tap | s) ? 1u : 0u);
                    }
                }
            tc::mma_commit(bar);
        }
        const bool done = tc::bar_wait(bar, phase, SPIN);
        if (__syncthreads_or(!done)) {
            if (tid == 0) {
                tc::bar_wait(bar, phase, SPIN);  // the MMAs must end before the memory is released
                atomicExch(err, 1);
            }
            break;
        }
        phase ^= 1u;
        tc::fence_after();
        // ---- epilogue: thread = pixel (row m of the tile), warps 0-3 even tiles, 4-7 odd tiles
        const int q = warp & 3, m = 32 * q + lane;
        const int oy = y0 + (m >> 3);
        for (int j = warp >> 2; j < MT; j += 2) {
            const int ox = x0 + 8 * j + (m & 7);
            const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * NOUT);
            if (OUT_MAP) {
                const float v = __uint_as_float(tc::tmem_ld1(taddr));
                tc::tmem_wait_ld();
                if (oy < H && ox < W) map[(size_t)oy * W + ox] = v + sBias[0];
            } else {
                uint32_t r[32];
                tc::tmem_ld32(taddr, r);
                tc::tmem_wait_ld();
                if (oy < H && ox < W) {
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        __align__(16) __half h[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            h[c] = __float2half_rn(fmaxf(__uint_as_float(r[8 * g + c]) + sBias[8 * g + c], 0.f));
                        reinterpret_cast<uint4 *>(hout)[((size_t)g * H + oy) * W + ox] =
                            *reinterpret_cast<const uint4 *>(h);
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();  // tensor memory and the staged planes are free for the next strip
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

// Hidden layers (1..4: four planes of 8 FP16 channels in), with the input staged by TMA: a block runs
// its strips in turn with two staging buffers; while strip i's MMAs and epilogue run, the tensor-memory
// accumulators being read and the outputs written, the TMA copy of strip i + 1's input (the same
// 4 x 18 x 66 box of 16-byte pixel vectors, zero outside the image) lands in the other buffer.  One
// block per SM (two 76 KB buffers).  Waits bounded as in k_conv_tc; a block that gives up waits
// (bounded) for its copy in flight and its MMAs before it releases its tensor memory.
constexpr int CING_H = 4;
constexpr size_t TMA_BOX_BYTES = (size_t)CING_H * PY * PX * 16;
constexpr size_t TMA_BUF = (TMA_BOX_BYTES + 1023) / 1024 * 1024;

template <int NOUT>
struct ConvTmaLayout {
    static constexpr size_t buf0 = 0, buf1 = TMA_BUF;
    static constexpr size_t b_off = 2 * TMA_BUF;
    static constexpr size_t b_bytes = (size_t)9 * CING_H * NOUT * 16;
    static constexpr size_t bias_off = b_off + b_bytes;
    static constexpr size_t bar_off = (bias_off + (size_t)NOUT * 4 + 15) / 16 * 16;
    static constexpr size_t total = bar_off + 4 * 8 + 16;
    static constexpr uint32_t tcols = MT * NOUT;
};

template <int NOUT, bool OUT_MAP>
__global__ void __launch_bounds__(NTH, 1)
    k_conv_tma(const __grid_constant__ CUtensorMap tmap, int H, int W, const __half *__restrict__ wt, int cin, int cout,
               __half *__restrict__ hout, float *__restrict__ map, int *err) {
    using L = ConvTmaLayout<NOUT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __half *sB = reinterpret_cast<__half *>(smem + L::b_off);
    float *sBias = reinterpret_cast<float *>(smem + L::bias_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::bar_off);  // [2]: a staging buffer's copy landed
    uint64_t *mbar = full + 2;                                         // the strip's MMAs completed
    uint32_t *slot = reinterpret_cast<uint32_t *>(full + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < 9 * CING_H * NOUT * 8; e += NTH) {
        const int k = e & 7, rest = e >> 3;
        const int n = rest % NOUT, g = (rest / NOUT) % CING_H, tap = rest / (NOUT * CING_H);
        const int ci = g * 8 + k;
        sB[e] = (n < cout && ci < cin) ? wt[(n * cin + ci) * 9 + tap] : __float2half_rn(0.f);
    }
    for (int n = tid; n < NOUT; n += NTH) sBias[n] = n < cout ? __half2float(wt[cout * cin * 9 + n]) : 0.f;
    const int nsx = (W + SX - 1) / SX, nstrip = ((H + SY - 1) / SY) * nsx;
    if (tid == 0) {
        tc::bar_init(&full[0], 1);
        tc::bar_init(&full[1], 1);
        tc::bar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(slot, L::tcols);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idesc = tc::idesc_f16(128, NOUT, false);
    auto issue_copy = [&](int strip, int b) {  // thread 0: the strip's input box into buffer b
        const int y0 = (strip / nsx) * SY, x0 = (strip % nsx) * SX;
        tc::bar_arrive_expect_tx(&full[b], (uint32_t)TMA_BOX_BYTES);
        tc::tma_load_3d(smem + (b ? L::buf1 : L::buf0), &tmap, &full[b], 2 * (x0 - 1), y0 - 1, 0);
    };
    // copies issued into / waited for from each buffer (the same on every thread: the decisions are uniform)
    int issued[2] = {0, 0}, waited[2] = {0, 0};
    if ((int)blockIdx.x < nstrip) {
        if (tid == 0) issue_copy(blockIdx.x, 0);
        issued[0] = 1;
    }
    bool failed = false;
    int i = 0;
    for (int strip = blockIdx.x; strip < nstrip; strip += gridDim.x, ++i) {
        const int b = i & 1;
        const int y0 = (strip / nsx) * SY, x0 = (strip % nsx) * SX;
        // the next strip's copy goes out now (its buffer's last reader, strip i - 1's MMAs, has completed)
        const int next = strip + gridDim.x;
        if (next < nstrip) {
            if (tid == 0) issue_copy(next, b ^ 1);
            ++issued[b ^ 1];
        }
        const bool landed = tc::bar_wait(&full[b], (uint32_t)(waited[b] & 1), SPIN);
        if (__syncthreads_or(!landed)) {
            failed = true;
            break;
        }
        ++waited[b];
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::su32(smem + (b ? L::buf1 : L::buf0)), b0 = tc::su32(sB);
            for (int j = 0; j < MT; ++j)
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int ss = 0; ss < CING_H / 2; ++ss) {
                        const uint32_t aoff = (uint32_t)((((2 * ss) * PY + ky) * PX + 8 * j + kx) * 16);
                        const uint32_t boff = (uint32_t)((tap * CING_H + 2 * ss) * NOUT * 16);
                        const uint64_t ad = tc::sdesc(a0 + aoff, PY * PX * 16, PX * 16);
                        const uint64_t bd = tc::sdesc(b0 + boff, NOUT * 16, 128);
                        tc::mma_f16(tbase + j * NOUT, ad, bd, idesc, (tap | ss) ? 1u : 0u);
                    }
                }
            tc::mma_commit(mbar);
        }
        const bool done = tc::bar_wait(mbar, (uint32_t)(i & 1), SPIN);
        if (__syncthreads_or(!done)) {
            if (tid == 0) tc::bar_wait(mbar, (uint32_t)(i & 1), SPIN);  // the MMAs end before the memory is released
            failed = true;
            break;
        }
        tc::fence_after();
        const int q = warp & 3, m = 32 * q + lane;
        const int oy = y0 + (m >> 3);
        for (int j = warp >> 2; j < MT; j += 2) {
            const int ox = x0 + 8 * j + (m & 7);
            const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * NOUT);
            if (OUT_MAP) {
                const float v = __uint_as_float(tc::tmem_ld1(taddr));
                tc::tmem_wait_ld();
                if (oy < H && ox < W) map[(size_t)oy * W + ox] = v + sBias[0];
            } else {
                uint32_t r[32];
                tc::tmem_ld32(taddr, r);
                tc::tmem_wait_ld();
                if (oy < H && ox < W) {
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        __align__(16) __half h[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            h[c] = __float2half_rn(fmaxf(__uint_as_float(r[8 * g + c]) + sBias[8 * g + c], 0.f));
                        reinterpret_cast<uint4 *>(hout)[((size_t)g * H + oy) * W + ox] =
                            *reinterpret_cast<const uint4 *>(h);
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();  // tensor memory is free for the next strip
    }
    if (failed && tid == 0) {
        atomicExch(err, 1);
        // copies still in flight must land before the block's shared memory is released
        for (int pb = 0; pb < 2; ++pb)
            for (int w = waited[pb]; w < issued[pb]; ++w) tc::bar_wait(&full[pb], (uint32_t)(w & 1), SPIN);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

// After a forward whose wait gave up: the whole map becomes NaN.
__global__ void k_map_poison(float *map, size_t n, const int *err) {
    if (*err == 0) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        map[i] = __int_as_float(0x7fc00000);
}

template <int CING, int NOUT, bool IN_F32, bool OUT_MAP>
hts_status conv_tc(const hts_cnn *n, int l, const float *img, const __half *hin, int H, int W, __half *hout,
                   float *map, int nsm, cudaStream_t s) {
    using L = ConvTcLayout<CING, NOUT>;
    const void *k = reinterpret_cast<const void *>(k_conv_tc<CING, NOUT, IN_F32, OUT_MAP>);
    const hts_status st = allow_smem(k, L::total);
    if (st != HTS_OK) return st;
    const int nstrip = ((H + SY - 1) / SY) * ((W + SX - 1) / SX);
    const int grid = std::max(1, std::min(nstrip, 2 * nsm));
    {
        KTimer kt("k_conv_tc", s);
        k_conv_tc<CING, NOUT, IN_F32, OUT_MAP><<<grid, NTH, L::total, s>>>(
            img, n->C, hin, H, W, n->w16 + n->off[l], n->cin[l], n->cout[l], hout, map, n->err);
    }
    return check_launch("k_conv_tc");
}

// A hidden layer with the TMA-staged input: the tensor map describes hin as [plane][y][x][8 halves], read
// as 8-byte elements (3-D, innermost first: 2 W, H, 4 planes) with the box of one strip's staged input.
template <int NOUT, bool OUT_MAP>
hts_status conv_tma(const hts_cnn *n, int l, const __half *hin, int H, int W, __half *hout, float *map, int nsm,
                    cudaStream_t s) {
    using L = ConvTmaLayout<NOUT>;
    const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return report(HTS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    // 8-byte elements, two per pixel vector: each box row is one contiguous run of 2 PX elements
    CUtensorMap tmap;
    const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)CING_H};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * PX), (cuuint32_t)PY, (cuuint32_t)CING_H};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<__half *>(hin), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return report(HTS_ECUDA, "cuTensorMapEncodeTiled failed for a network layer");
    const void *k = reinterpret_cast<const void *>(k_conv_tma<NOUT, OUT_MAP>);
    const hts_status st = allow_smem(k, L::total);
    if (st != HTS_OK) return st;
    const int nstrip = ((H + SY - 1) / SY) * ((W + SX - 1) / SX);
    const int grid = std::max(1, std::min(nstrip, nsm));
    {
        KTimer kt("k_conv_tma", s);
        k_conv_tma<NOUT, OUT_MAP><<<grid, NTH, L::total, s>>>(tmap, H, W, n->w16 + n->off[l], n->cin[l], n->cout[l],
                                                               hout, map, n->err);
    }
    return check_launch("k_conv_tma");
}

}  // namespace

template <typename T>
hts_status grow_buf(T *&p, size_t &cap, size_t need) {
    if (need <= cap && p) return HTS_OK;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    if (dev_malloc(&p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return report(HTS_ENOMEM, "cudaMalloc(cnn inference buffers)");
    }
    cap = need;
    return HTS_OK;
}

hts_status cnn_ensure_infer(hts_cnn *n, int H, int W, int nx) {
    const size_t px = (size_t)H * W;
    if (px * 32 > n->cap_h16 || !n->h16[1]) {
        size_t c0 = 0;
        hts_status st = grow_buf(n->h16[0], c0, px * 32);
        size_t c1 = 0;
        if (st == HTS_OK) st = grow_buf(n->h16[1], c1, px * 32);
        n->cap_h16 = st == HTS_OK ? px * 32 : 0;
        if (st != HTS_OK) return st;
    }
    const hts_status st = grow_buf(n->map, n->cap_map, px);
    if (st != HTS_OK) return st;
    return grow_buf(n->rows, n->cap_rows, (size_t)H * nx);
}

hts_status cnn_forward_tc(hts_cnn *n, const float *img, int H, int W, cudaStream_t s) {
    return cnn_forward_tc_into(n, img, H, W, n->h16[0], n->h16[1], n->map, s);
}

hts_status cnn_forward_tc_into(hts_cnn *n, const float *img, int H, int W, __half *h0, __half *h1, float *map,
                               cudaStream_t s) {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMemsetAsync(n->err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return report(HTS_ECUDA, "cudaMemsetAsync(cnn error flag)");
    }
    hts_status st = conv_tc<2, 32, true, false>(n, 0, img, nullptr, H, W, h0, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, false>(n, 1, h0, H, W, h1, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, false>(n, 2, h1, H, W, h0, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, false>(n, 3, h0, H, W, h1, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<16, true>(n, 4, h1, H, W, nullptr, map, nsm, s);
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_map_poison", s);
        k_map_poison<<<nsm, 256, 0, s>>>(map, (size_t)H * W, n->err);
    }
    return check_launch("k_map_poison");
}

}  // namespace hts
