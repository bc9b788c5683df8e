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

// Epilogues: bias and ReLU to FP16 planes (forward, hidden layers), column 0 plus bias to the FP32 map
// (forward, last layer), or the accumulated value times the ReLU mask of a stored activation to FP16 planes
// (backward: the gradient of a layer's input, zero where the activation is zero).
constexpr int EPI_RELU = 0, EPI_MAP = 1, EPI_MASK = 2;

// One tile row of the epilogue: thread m of lane quarter q holds output pixel (oy, ox); r: its NOUT
// accumulator columns (read by the caller).
template <int NOUT, int EPI>
__device__ __forceinline__ void epilogue_store(const uint32_t *r, const float *sBias, int H, int W, int oy, int ox,
                                               __half *hout, float *map, const __half *hmask) {
    if (oy >= H || ox >= W) return;
    const size_t HW = (size_t)H * W;
    if constexpr (EPI == EPI_MAP) {
        map[(size_t)oy * W + ox] = __uint_as_float(r[0]) + sBias[0];
    } else {
#pragma unroll
        for (int g = 0; g < NOUT / 8; ++g) {
            const size_t pix = (size_t)g * HW + (size_t)oy * W + ox;
            __align__(16) __half h[8];
            if (EPI == EPI_RELU) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    h[c] = __float2half_rn(fmaxf(__uint_as_float(r[8 * g + c]) + sBias[8 * g + c], 0.f));
            } else {
                const uint4 mv = reinterpret_cast<const uint4 *>(hmask)[pix];
                const __half *mk = reinterpret_cast<const __half *>(&mv);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    h[c] = __float2half_rn(__hgt(mk[c], __float2half_rn(0.f)) ? __uint_as_float(r[8 * g + c]) : 0.f);
            }
            reinterpret_cast<uint4 *>(hout)[pix] = *reinterpret_cast<const uint4 *>(h);
        }
    }
}

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
// IN_F32: the input is an FP32 planar C x H x W array (the image) times
// in_scale (1/255); otherwise FP16 planes hin[g][y][x][8].  EPI: the
// epilogue (EPI_RELU, EPI_MAP, EPI_MASK with the activation planes hmask).
template <int CING, int NOUT, bool IN_F32, int EPI>
__global__ void __launch_bounds__(NTH, 2)
    k_conv_tc(const float *__restrict__ img, int C, float in_scale, const __half *__restrict__ hin, int H, int W,
              const __half *__restrict__ wt, int cin, int cout, __half *__restrict__ hout, float *__restrict__ map,
              const __half *__restrict__ hmask, int *err) {
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
        if constexpr (IN_F32) {
            // plane 0 only (the others stay zero from the first strip): every load of the thread's pixels
            // issued before the first conversion
            constexpr int NE = (PY * PX + NTH - 1) / NTH;
            float v[NE][3];
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const int e = tid + i * NTH, py = e / PX, px = e - py * PX;
                const int y = y0 - 1 + py, x = x0 - 1 + px;
                const bool in = e < PY * PX && y >= 0 && y < H && x >= 0 && x < W;
#pragma unroll
                for (int c = 0; c < 3; ++c) v[i][c] = (in && c < C) ? __ldg(img + c * HW + (size_t)y * W + x) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const int e = tid + i * NTH;
                if (e < PY * PX) {
                    __align__(16) __half h[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) h[c] = __float2half_rn(c < 3 ? v[i][c] * in_scale : 0.f);
                    sA[e] = *reinterpret_cast<const uint4 *>(h);
                }
            }
            if (strip == (int)blockIdx.x)
                for (int e = PY * PX + tid; e < CING * PY * PX; e += NTH) sA[e] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            for (int e = tid; e < CING * PY * PX; e += NTH) {
                const int g = e / (PY * PX), r = e - g * (PY * PX), py = r / PX, px = r - py * PX;
                const int y = y0 - 1 + py, x = x0 - 1 + px;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (y >= 0 && y < H && x >= 0 && x < W) v = reinterpret_cast<const uint4 *>(hin)[((size_t)g * H + y) * W + x];
                sA[e] = v;
            }
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
            uint32_t r[32];
            if (EPI == EPI_MAP) {
                r[0] = tc::tmem_ld1(taddr);
            } else {
                tc::tmem_ld32(taddr, r);
            }
            tc::tmem_wait_ld();
            epilogue_store<NOUT, EPI>(r, sBias, H, W, oy, ox, hout, map, hmask);
        }
        tc::fence_before();
        __syncthreads();  // tensor memory and the staged planes are free for the next strip
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

// Hidden layers (1..4: four planes of 8 FP16 channels in), with the input staged by TMA: a block runs
// its strips (16 x 16 output pixels: two 16 x 8 tiles) in turn through a ring of NBH staging buffers.  The
// copies of the block's next NBH - 1 strips (4 x 18 x 18 boxes of 16-byte pixel vectors, zero outside the
// image) are in flight while a strip's MMAs and epilogue run; once a strip's MMAs have completed its buffer
// takes the copy of the strip NBH ahead.  Two blocks per SM (four 21 KB buffers each, 64 tensor-memory
// columns, at most 128 registers a thread): six input boxes in flight per SM keep enough reads outstanding
// for the memory's latency.  Waits bounded as in k_conv_tc; a block that gives up waits (bounded) for its
// copies in flight and its MMAs before it releases its shared and tensor memory.
constexpr int CING_H = 4;
constexpr int MTH = 2;                 // tiles per strip of the hidden layers
constexpr int NBH = 4;                 // staging buffers (ring)
constexpr int SXH = 8 * MTH, PXH = SXH + 2;
constexpr size_t TMA_BOX_BYTES = (size_t)CING_H * PY * PXH * 16;
constexpr size_t TMA_BUF = (TMA_BOX_BYTES + 1023) / 1024 * 1024;

template <int NOUT>
struct ConvTmaLayout {
    static constexpr size_t b_off = NBH * TMA_BUF;  // buffer k at k * TMA_BUF
    static constexpr size_t b_bytes = (size_t)9 * CING_H * NOUT * 16;
    static constexpr size_t bias_off = b_off + b_bytes;
    static constexpr size_t bar_off = (bias_off + (size_t)NOUT * 4 + 15) / 16 * 16;
    static constexpr size_t total = bar_off + (NBH + 1) * 8 + 16;  // NBH copy barriers, the MMA barrier, slot
    static constexpr uint32_t tcols = MTH * NOUT < 32 ? 32 : MTH * NOUT;
};

template <int NOUT, int EPI>
__global__ void __launch_bounds__(NTH, 2)
    k_conv_tma(const __grid_constant__ CUtensorMap tmap, int H, int W, const __half *__restrict__ wt, int cin, int cout,
               __half *__restrict__ hout, float *__restrict__ map, const __half *__restrict__ hmask, int *err) {
    using L = ConvTmaLayout<NOUT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __half *sB = reinterpret_cast<__half *>(smem + L::b_off);
    float *sBias = reinterpret_cast<float *>(smem + L::bias_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::bar_off);  // [NBH]: a staging buffer's copy landed
    uint64_t *mbar = full + NBH;                                       // the strip's MMAs completed
    uint32_t *slot = reinterpret_cast<uint32_t *>(full + NBH + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < 9 * CING_H * NOUT * 8; e += NTH) {
        const int k = e & 7, rest = e >> 3;
        const int n = rest % NOUT, g = (rest / NOUT) % CING_H, tap = rest / (NOUT * CING_H);
        const int ci = g * 8 + k;
        sB[e] = (n < cout && ci < cin) ? wt[(n * cin + ci) * 9 + tap] : __float2half_rn(0.f);
    }
    for (int n = tid; n < NOUT; n += NTH) sBias[n] = n < cout ? __half2float(wt[cout * cin * 9 + n]) : 0.f;
    const int nsx = (W + SXH - 1) / SXH, nstrip = ((H + SY - 1) / SY) * nsx;
    if (tid == 0) {
        for (int k = 0; k <= NBH; ++k) tc::bar_init(&full[k], 1);
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
        const int y0 = (strip / nsx) * SY, x0 = (strip % nsx) * SXH;
        tc::bar_arrive_expect_tx(&full[b], (uint32_t)TMA_BOX_BYTES);
        tc::tma_load_3d(smem + (size_t)b * TMA_BUF, &tmap, &full[b], 2 * (x0 - 1), y0 - 1, 0);
    };
    // The block's k-th strip goes through buffer k % NBH; copies issued (and waited for) in order, so copy k
    // lands on the (k / NBH)-th phase of its buffer's barrier.  The counts are the same on every thread.
    int issued = 0, waited = 0;
    for (int k = 0; k < NBH && (int)blockIdx.x + k * (int)gridDim.x < nstrip; ++k) {
        if (tid == 0) issue_copy(blockIdx.x + k * gridDim.x, k);
        ++issued;
    }
    bool failed = false;
    int i = 0;
    for (int strip = blockIdx.x; strip < nstrip; strip += gridDim.x, ++i) {
        const int b = i % NBH;
        const int y0 = (strip / nsx) * SY, x0 = (strip % nsx) * SXH;
        const bool landed = tc::bar_wait(&full[b], (uint32_t)((i / NBH) & 1), SPIN);
        if (__syncthreads_or(!landed)) {
            failed = true;
            break;
        }
        ++waited;
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::su32(smem + (size_t)b * TMA_BUF), b0 = tc::su32(sB);
            for (int j = 0; j < MTH; ++j)
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int ss = 0; ss < CING_H / 2; ++ss) {
                        const uint32_t aoff = (uint32_t)((((2 * ss) * PY + ky) * PXH + 8 * j + kx) * 16);
                        const uint32_t boff = (uint32_t)((tap * CING_H + 2 * ss) * NOUT * 16);
                        const uint64_t ad = tc::sdesc(a0 + aoff, PY * PXH * 16, PXH * 16);
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
        // buffer b is free (this strip's MMAs have read it): the copy of the strip NBH ahead
        const int ahead = strip + NBH * (int)gridDim.x;
        if (ahead < nstrip) {
            if (tid == 0) issue_copy(ahead, b);
            ++issued;
        }
        const int q = warp & 3, m = 32 * q + lane;
        const int oy = y0 + (m >> 3);
        for (int j = warp >> 2; j < MTH; j += 2) {
            const int ox = x0 + 8 * j + (m & 7);
            const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * NOUT);
            uint32_t r[32];
            if (EPI == EPI_MAP) {
                r[0] = tc::tmem_ld1(taddr);
            } else {
                tc::tmem_ld32(taddr, r);
            }
            tc::tmem_wait_ld();
            epilogue_store<NOUT, EPI>(r, sBias, H, W, oy, ox, hout, map, hmask);
        }
        tc::fence_before();
        __syncthreads();  // tensor memory is free for the next strip
    }
    if (failed && tid == 0) {
        atomicExch(err, 1);
        // copies still in flight must land before the block's shared memory is released
        for (int w = waited; w < issued; ++w) tc::bar_wait(&full[w % NBH], (uint32_t)((w / NBH) & 1), SPIN);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

// The network's FP16 weights of layer l with its channel counts, as conv_tc / conv_tma take them.
#define LW(n, l) (n)->w16 + (n)->off[l], (n)->cin[l], (n)->cout[l]

// After a forward whose wait gave up: the whole map becomes NaN.
__global__ void k_map_poison(float *map, size_t n, const int *err) {
    if (*err == 0) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        map[i] = __int_as_float(0x7fc00000);
}

// wt: FP16 weights [cout][cin][3][3] then cout biases (the network's, or the flipped ones of a backward pass).
template <int CING, int NOUT, bool IN_F32, int EPI>
hts_status conv_tc(const hts_cnn *n, const __half *wt, int cin, int cout, const float *img, int C, float in_scale,
                   const __half *hin, int H, int W, __half *hout, float *map, const __half *hmask, int nsm,
                   cudaStream_t s) {
    using L = ConvTcLayout<CING, NOUT>;
    const void *k = reinterpret_cast<const void *>(k_conv_tc<CING, NOUT, IN_F32, EPI>);
    const hts_status st = allow_smem(k, L::total);
    if (st != HTS_OK) return st;
    const int nstrip = ((H + SY - 1) / SY) * ((W + SX - 1) / SX);
    const int grid = std::max(1, std::min(nstrip, 2 * nsm));
    {
        KTimer kt("k_conv_tc", s);
        k_conv_tc<CING, NOUT, IN_F32, EPI><<<grid, NTH, L::total, s>>>(img, C, in_scale, hin, H, W, wt, cin, cout,
                                                                      hout, map, hmask, n->err);
    }
    return check_launch("k_conv_tc");
}

// A hidden layer with the TMA-staged input: the tensor map describes hin as [plane][y][x][8 halves], read
// as 8-byte elements (3-D, innermost first: 2 W, H, 4 planes) with the box of one strip's staged input.
template <int NOUT, int EPI>
hts_status conv_tma(const hts_cnn *n, const __half *wt, int cin, int cout, const __half *hin, int H, int W,
                    __half *hout, float *map, const __half *hmask, int nsm, cudaStream_t s) {
    using L = ConvTmaLayout<NOUT>;
    const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return report(HTS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    // 8-byte elements, two per pixel vector: each box row is one contiguous run of 2 PXH elements
    CUtensorMap tmap;
    const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)CING_H};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * PXH), (cuuint32_t)PY, (cuuint32_t)CING_H};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<__half *>(hin), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return report(HTS_ECUDA, "cuTensorMapEncodeTiled failed for a network layer");
    const void *k = reinterpret_cast<const void *>(k_conv_tma<NOUT, EPI>);
    const hts_status st = allow_smem(k, L::total);
    if (st != HTS_OK) return st;
    const int nstrip = ((H + SY - 1) / SY) * ((W + SXH - 1) / SXH);
    const int grid = std::max(1, std::min(nstrip, 2 * nsm));
    {
        KTimer kt("k_conv_tma", s);
        k_conv_tma<NOUT, EPI><<<grid, NTH, L::total, s>>>(tmap, H, W, wt, cin, cout, hout, map, hmask, n->err);
    }
    return check_launch("k_conv_tma");
}

// ------------------------------------------------------------------ training (backward) on the tensor cores

// Weight and bias gradient of one 3x3 layer: dW[co][ci][ky][kx] = sum_p dY[co](p) X[ci](p + (ky - 1, kx - 1)),
// db[co] = sum_p dY[co](p), a contraction over the pixels: D[(tap, ci)][co] = sum_p A[(tap, ci)][p] B[co][p]
// with the pixels as the MMA's K.  A block takes strips of 8 x 64 pixels, stages X with a one-pixel halo and
// dY as planes of 8 FP16 channels, and per strip row (64 pixels, four K steps) copies the 64 pixel vectors of
// every (tap, plane) into a 1 KB group of a chunk buffer, so that the 8-row groups of A (8 channels of one
// plane at one tap) lie 1 KB apart: A is MN-major (8 channels per 16-byte pixel vector), M = 128 rows = 16
// groups per tile; one extra group holds ones (its rows give the bias gradient).  B is the staged dY row,
// MN-major as well (core matrices of 8 pixels, planes 8 KB apart).  The block accumulates every strip it
// takes in tensor memory and writes its sums once; k_wgrad_reduce adds the blocks' sums in block order.
constexpr int WSY = 8;            // strip rows
constexpr int WPY = WSY + 2;      // staged X rows
constexpr int WCH = SX;           // pixels per chunk (one strip row)

template <int CINX, int NPLY>
struct WgradLayout {
    static constexpr int NG = 9 * CINX + 1;        // (tap, plane) groups and the ones group
    static constexpr int NTILE = (NG + 15) / 16;   // M tiles of 16 groups
    static constexpr int N = NPLY * 8;             // MMA N: the output channels
    static constexpr int ROWS = 9 * CINX * 8 + 1;  // rows written per block: (tap, ci), then the bias row
    static constexpr size_t x_bytes = (size_t)CINX * WPY * PX * 16;
    static constexpr size_t y_off = (x_bytes + 1023) / 1024 * 1024;
    static constexpr size_t y_plane = (size_t)WSY * WCH * 16;
    static constexpr size_t i_off = y_off + (size_t)NPLY * y_plane;
    static constexpr size_t bar_off = i_off + (size_t)NTILE * 16 * 1024;
    static constexpr size_t used = bar_off + 32;
    static constexpr size_t total = used > MIN_SMEM ? used : MIN_SMEM;
    static constexpr uint32_t tcols = NTILE * N <= 32 ? 32 : NTILE * N <= 64 ? 64 : NTILE * N <= 128 ? 128 : 256;
};

// X_F32: X is the FP32 image (planar, C channels) times 1/255, else FP16 planes xin[CINX][H][W][8].
// Y_F32: dY is the FP32 gradient map (one channel) times y_scale, else FP16 planes yin[NPLY][H][W][8].
template <int CINX, int NPLY, bool X_F32, bool Y_F32>
__global__ void __launch_bounds__(NTH, 1)
    k_conv_wgrad(const float *__restrict__ img, int C, const __half *__restrict__ xin, const float *__restrict__ ymap,
                 float y_scale, const __half *__restrict__ yin, int H, int W, float *__restrict__ part,
                 int *err) {
    using L = WgradLayout<CINX, NPLY>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint4 *sX = reinterpret_cast<uint4 *>(smem);
    uint4 *sY = reinterpret_cast<uint4 *>(smem + L::y_off);
    uint4 *sI = reinterpret_cast<uint4 *>(smem + L::i_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t HW = (size_t)H * W;
    // chunk buffer: groups past the (tap, plane) ones: the ones group, then zeros
    for (int e = tid; e < (L::NTILE * 16 - 9 * CINX) * WCH; e += NTH) {
        const int gr = 9 * CINX + e / WCH;
        const __half one = __float2half_rn(gr == 9 * CINX ? 1.f : 0.f);
        const __half2 h2 = __halves2half2(one, one);
        uint4 v;
        v.x = v.y = v.z = v.w = *reinterpret_cast<const uint32_t *>(&h2);
        sI[gr * WCH + (e % WCH)] = v;
    }
    if (tid == 0) {
        tc::bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) tc::tmem_alloc(slot, L::tcols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t idesc = tc::idesc_f16(128, L::N, false) | (1u << 15) | (1u << 16);  // A and B MN-major
    const int nsx = (W + WCH - 1) / WCH, nstrip = ((H + WSY - 1) / WSY) * nsx;
    uint32_t phase = 0;
    bool first = true, failed = false;
    for (int strip = blockIdx.x; strip < nstrip && !failed; strip += gridDim.x) {
        const int y0 = (strip / nsx) * WSY, x0 = (strip % nsx) * WCH;
        // ---- stage X (halo, zero outside the image) and dY (zero outside)
        for (int e = tid; e < CINX * WPY * PX; e += NTH) {
            const int gp = e / (WPY * PX), r = e - gp * (WPY * PX), py = r / PX, px = r - py * PX;
            const int y = y0 - 1 + py, x = x0 - 1 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (y >= 0 && y < H && x >= 0 && x < W) {
                if (X_F32) {
                    __align__(16) __half h[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        h[c] = __float2half_rn(c < C ? img[c * HW + (size_t)y * W + x] * (1.f / 255.f) : 0.f);
                    v = *reinterpret_cast<const uint4 *>(h);
                } else {
                    v = reinterpret_cast<const uint4 *>(xin)[((size_t)gp * H + y) * W + x];
                }
            }
            sX[e] = v;
        }
        for (int e = tid; e < NPLY * WSY * WCH; e += NTH) {
            const int gp = e / (WSY * WCH), r = e - gp * (WSY * WCH), py = r / WCH, px = r - py * WCH;
            const int y = y0 + py, x = x0 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (y < H && x < W) {
                if (Y_F32) {
                    if (gp == 0) {
                        __align__(16) __half h[8];
                        h[0] = __float2half_rn(ymap[(size_t)y * W + x] * y_scale);
#pragma unroll
                        for (int c = 1; c < 8; ++c) h[c] = __float2half_rn(0.f);
                        v = *reinterpret_cast<const uint4 *>(h);
                    }
                } else {
                    v = reinterpret_cast<const uint4 *>(yin)[((size_t)gp * H + y) * W + x];
                }
            }
            sY[e] = v;
        }
        __syncthreads();
        for (int r = 0; r < WSY; ++r) {
            // ---- the chunk (strip row r): group (tap, plane) = the 64 staged X vectors of that tap's shift
            for (int e = tid; e < 9 * CINX * WCH; e += NTH) {
                const int gr = e / WCH, px = e - gr * WCH;
                const int tap = gr / CINX, gp = gr - tap * CINX, ky = tap / 3, kx = tap - 3 * ky;
                sI[gr * WCH + px] = sX[(gp * WPY + r + ky) * PX + px + kx];
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
                const uint32_t a0 = tc::su32(sI), b0 = tc::su32(sY) + (uint32_t)(r * WCH * 16);
#pragma unroll
                for (int t = 0; t < L::NTILE; ++t)
#pragma unroll
                    for (int kk = 0; kk < WCH / 16; ++kk) {
                        const uint64_t ad = tc::sdesc(a0 + t * 16 * 1024 + kk * 256, 128, 1024);
                        const uint64_t bd = tc::sdesc(b0 + kk * 256, 128, (uint32_t)L::y_plane);
                        tc::mma_f16(tbase + t * L::N, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
                    }
                tc::mma_commit(bar);
            }
            const bool done = tc::bar_wait(bar, phase, SPIN);
            if (__syncthreads_or(!done)) {
                if (tid == 0) {
                    tc::bar_wait(bar, phase, SPIN);  // the MMAs must end before the memory is released
                    atomicExch(err, 1);
                }
                failed = true;
                break;
            }
            phase ^= 1u;
            tc::fence_after();
            first = false;
        }
    }
    // ---- the block's sums: row (tap, ci) or the bias row, N output channels
    if (!failed && !first) {
        const int q = warp & 3;
        for (int t = warp >> 2; t < L::NTILE; t += NTH / 128) {
            const int row = t * 128 + 32 * q + lane, gr = row >> 3, ch = row & 7;
            uint32_t v[32];
            const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(t * L::N);
            if constexpr (L::N == 32) {
                tc::tmem_ld32(taddr, v);
            } else {
                tc::tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(v));
            }
            tc::tmem_wait_ld();
            int orow = -1;
            if (gr < 9 * CINX) orow = gr * 8 + ch;                  // (tap, plane, channel) = tap * 8 CINX + ci
            else if (gr == 9 * CINX && ch == 0) orow = L::ROWS - 1;  // the bias
            if (orow >= 0) {
                float *dst = part + ((size_t)blockIdx.x * L::ROWS + orow) * L::N;
#pragma unroll
                for (int n = 0; n < L::N; ++n) dst[n] = __uint_as_float(v[n]);
            }
        }
    } else if (!failed) {  // a block without strips adds zeros
        for (int e = tid; e < L::ROWS * L::N; e += NTH) part[(size_t)blockIdx.x * L::ROWS * L::N + e] = 0.f;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, L::tcols);
}

// grad[e] += (sum over the blocks, in block order, of their sums) / scale for every parameter of the layer
// (cout x cin x 9 weights, then cout biases); NaN everywhere after a wait that gave up.
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nblk, int rows, int N, int cin, int cout,
                               int cin_pad, float inv_scale, const int *err, float *__restrict__ grad) {
    const int ne = cout * cin * 9 + cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        int row, co;
        if (e < cout * cin * 9) {
            co = e / (cin * 9);
            const int rem = e - co * cin * 9, ci = rem / 9, tap = rem - ci * 9;
            row = tap * cin_pad + ci;
        } else {
            co = e - cout * cin * 9;
            row = rows - 1;
        }
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += part[((size_t)b * rows + row) * N + co];
        grad[e] = *err ? __int_as_float(0x7fc00000) : grad[e] + s * inv_scale;
    }
}

// The flipped, transposed weights of a backward pass through layer l: out channel n = the layer's input
// channel, input channel c = its output channel, tap 8 - t; biases zero.
__global__ void k_wflip(const __half *__restrict__ w, int cout, int cin, __half *__restrict__ wt) {
    const int ne = cin * cout * 9;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne + cin; e += gridDim.x * blockDim.x) {
        if (e >= ne) {
            wt[e] = __float2half_rn(0.f);
            continue;
        }
        const int n = e / (cout * 9), rem = e - n * cout * 9, c = rem / 9, tap = rem - c * 9;
        wt[e] = w[(c * cin + n) * 9 + (8 - tap)];
    }
}

// y_scale: the loss scale dY carries (applied here when dY is the FP32 map, by the caller otherwise); the
// reduction divides it out.
template <int CINX, int NPLY, bool X_F32, bool Y_F32>
hts_status conv_wgrad(hts_cnn *n, int l, const float *img, const __half *xin, const float *ymap, float y_scale,
                      const __half *yin, int H, int W, int nsm, cudaStream_t s) {
    using L = WgradLayout<CINX, NPLY>;
    const void *k = reinterpret_cast<const void *>(k_conv_wgrad<CINX, NPLY, X_F32, Y_F32>);
    hts_status st = allow_smem(k, L::total);
    if (st != HTS_OK) return st;
    const int nstrip = ((H + WSY - 1) / WSY) * ((W + WCH - 1) / WCH);
    const int grid = std::max(1, std::min(nstrip, nsm));
    {
        KTimer kt("k_conv_wgrad", s);
        k_conv_wgrad<CINX, NPLY, X_F32, Y_F32><<<grid, NTH, L::total, s>>>(img, n->C, xin, ymap, y_scale, yin, H, W,
                                                                          n->tr_part, n->err);
    }
    st = check_launch("k_conv_wgrad");
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_wgrad_reduce", s);
        k_wgrad_reduce<<<64, 256, 0, s>>>(n->tr_part, grid, L::ROWS, L::N, n->cin[l], n->cout[l], CINX * 8,
                                          1.f / y_scale, n->err, n->grad + n->off[l]);
    }
    return check_launch("k_wgrad_reduce");
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
    hts_status st = conv_tc<2, 32, true, EPI_RELU>(n, LW(n, 0), img, n->C, 1.f / 255.f, nullptr, H, W, h0, nullptr,
                                                   nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, EPI_RELU>(n, LW(n, 1), h0, H, W, h1, nullptr, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, EPI_RELU>(n, LW(n, 2), h1, H, W, h0, nullptr, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<32, EPI_RELU>(n, LW(n, 3), h0, H, W, h1, nullptr, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<16, EPI_MAP>(n, LW(n, 4), h1, H, W, nullptr, map, nullptr, nsm, s);
    if (st != HTS_OK) return st;
    {
        KTimer kt("k_map_poison", s);
        k_map_poison<<<nsm, 256, 0, s>>>(map, (size_t)H * W, n->err);
    }
    return check_launch("k_map_poison");
}


// ------------------------------------------------------------------ tensor-core training step

namespace {
constexpr int WG_ROWS_MAX = 9 * 4 * 8 + 1;
}  // namespace

hts_status cnn_train_ensure(hts_cnn *n, int H, int W, int nsm) {
    const size_t px = (size_t)H * W;
    if (px > n->tr_cap_px) {
        for (int i = 0; i < 4; ++i) {
            cudaFree(n->tr_act[i]);
            n->tr_act[i] = nullptr;
        }
        for (int i = 0; i < 2; ++i) {
            cudaFree(n->tr_dy[i]);
            n->tr_dy[i] = nullptr;
        }
        cudaFree(n->tr_map);
        cudaFree(n->tr_d0);
        n->tr_map = n->tr_d0 = nullptr;
        n->tr_cap_px = 0;
        size_t cap = 0;
        for (int i = 0; i < 4; ++i) {
            cap = 0;
            if (grow_buf(n->tr_act[i], cap, px * 32) != HTS_OK) return HTS_ENOMEM;
        }
        for (int i = 0; i < 2; ++i) {
            cap = 0;
            if (grow_buf(n->tr_dy[i], cap, px * 32) != HTS_OK) return HTS_ENOMEM;
        }
        cap = 0;
        if (grow_buf(n->tr_map, cap, px) != HTS_OK) return HTS_ENOMEM;
        cap = 0;
        if (grow_buf(n->tr_d0, cap, px) != HTS_OK) return HTS_ENOMEM;
        n->tr_cap_px = px;
    }
    hts_status st = grow_buf(n->tr_part, n->tr_cap_part, (size_t)nsm * WG_ROWS_MAX * 32);
    if (st != HTS_OK) return st;
    return grow_buf(n->tr_wt, n->tr_cap_wt, (size_t)n->nparams + 5 * 32);
}

// One image's loss and gradient on the tensor cores: the forward of cnn_forward_tc keeping every layer's
// FP16 activations, the loss gradient map 2 (out - target) / N_ref times the loss scale 2^(floor(log2 N_ref)
// + 2) (so (4, 8] times the error, well inside FP16's range) rounded to FP16, then per layer from the last:
// the weight and bias gradients (k_conv_wgrad, FP32 accumulation, the scale divided out) and the gradient of
// the layer input (the forward kernels with the flipped, transposed weights, times the ReLU mask of the
// stored activation, FP16).
hts_status cnn_grad_tc(hts_cnn *n, const float *img, int H, int W, const Geom &g, const float *target,
                       cudaStream_t s) {
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    hts_status st = cnn_train_ensure(n, H, W, nsm);
    if (st != HTS_OK) return st;
    if (cudaMemsetAsync(n->err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return report(HTS_ECUDA, "cudaMemsetAsync(cnn error flag)");
    }
    __half **a = n->tr_act;
    const float S = ldexpf(1.f, ilogb((double)g.nref) + 2);
    st = conv_tc<2, 32, true, EPI_RELU>(n, LW(n, 0), img, n->C, 1.f / 255.f, nullptr, H, W, a[0], nullptr, nullptr,
                                        nsm, s);
    for (int l = 1; l < 4 && st == HTS_OK; ++l)
        st = conv_tma<32, EPI_RELU>(n, LW(n, l), a[l - 1], H, W, a[l], nullptr, nullptr, nsm, s);
    if (st == HTS_OK) st = conv_tma<16, EPI_MAP>(n, LW(n, 4), a[3], H, W, nullptr, n->tr_map, nullptr, nsm, s);
    if (st == HTS_OK) st = cnn_loss(n->tr_map, H, W, g, target, n->tr_d0, n->loss, s);
    if (st != HTS_OK) return st;
    // flipped weights of layers 1..4 (layer l's at n->off[l] + 32 l: its cin biases follow its weights)
    for (int l = 1; l < 5; ++l) {
        {
            KTimer kt("k_wflip", s);
            k_wflip<<<64, 256, 0, s>>>(n->w16 + n->off[l], n->cout[l], n->cin[l], n->tr_wt + n->off[l] + 32 * l);
        }
        st = check_launch("k_wflip");
        if (st != HTS_OK) return st;
    }
    auto wf = [&](int l) { return n->tr_wt + n->off[l] + 32 * l; };
    // layer 4 (linear): its gradients from the loss map, then the gradient of its input
    st = conv_wgrad<4, 2, false, true>(n, 4, nullptr, a[3], n->tr_d0, S, nullptr, H, W, nsm, s);
    if (st == HTS_OK)
        st = conv_tc<2, 32, true, EPI_MASK>(n, wf(4), n->cout[4], n->cin[4], n->tr_d0, 1, S, nullptr, H, W,
                                            n->tr_dy[0], nullptr, a[3], nsm, s);
    int cur = 0;
    for (int l = 3; l >= 1 && st == HTS_OK; --l) {
        st = conv_wgrad<4, 4, false, false>(n, l, nullptr, a[l - 1], nullptr, S, n->tr_dy[cur], H, W, nsm, s);
        if (st == HTS_OK)
            st = conv_tma<32, EPI_MASK>(n, wf(l), n->cout[l], n->cin[l], n->tr_dy[cur], H, W, n->tr_dy[cur ^ 1],
                                        nullptr, a[l - 1], nsm, s);
        cur ^= 1;
    }
    if (st == HTS_OK)
        st = conv_wgrad<1, 4, true, false>(n, 0, img, nullptr, nullptr, S, n->tr_dy[cur], H, W, nsm, s);
    return st;
}

}  // namespace hts
