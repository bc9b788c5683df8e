// The learned noise-level network's handle and the entry points shared by its
// two translation units: cnn.cu (FP32 forward and backward for training,
// Adam, readout, host interface) and cnn_tc.cu (the tensor-core forward pass
// used for denoising).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/hts.h"

struct hts_cnn {
    int C = 1, device = 0, nparams = 0, t = 0, window = 128;
    int off[5] = {}, cin[5] = {}, cout[5] = {};  // per layer: parameter offset, input / output channels
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;  // FP32 parameters, Adam state
    __half *w16 = nullptr;                                                  // FP16 copy used by the kernels
    size_t cap_px = 0;
    float *act[5] = {};                   // FP32 activations (planar CHW) of the training forward
    float *d0 = nullptr, *d1 = nullptr;   // gradient maps; d0 also holds the readout's row sums
    size_t cap_part = 0;
    float *part = nullptr;                // per-tile partial weight gradients
    double *loss = nullptr;
    size_t cap_h16 = 0, cap_map = 0, cap_rows = 0;
    __half *h16[2] = {};    // FP16 activations of the tensor-core forward, 4 planes of 8 channels
    float *map = nullptr;   // its log-sigma map (H x W)
    float *rows = nullptr;  // row sums of the readout window (H x reference columns)
    int *err = nullptr;     // set by a tensor-core forward whose wait gave up (the map is then NaN)
    // tensor-core training (cnn_tc.cu): per-layer FP16 activations, FP16 input gradients (ping-pong), the
    // map and its loss gradient, per-block weight-gradient sums, the flipped weights of the backward passes
    int train_tc = 1;  // 1: hts_cnn_accumulate_grad runs on the tensor cores (FP16); 0: the FP32 kernels
    size_t tr_cap_px = 0, tr_cap_part = 0, tr_cap_wt = 0;
    __half *tr_act[4] = {}, *tr_dy[2] = {}, *tr_wt = nullptr;
    float *tr_map = nullptr, *tr_d0 = nullptr, *tr_part = nullptr;
};

namespace hts {

// Tensor-core forward pass (cnn_tc.cu): the log-sigma map of img (device,
// planar C x H x W, [0, 255]) in net->map (H x W, FP32).  Hidden
// activations are rounded to FP16 (8-channel planes, net->h16), the network
// input x / 255 too; FP16 weights, FP32 accumulation in tensor memory.
// cnn_ensure_infer sizes net->h16, net->map and net->rows first.
hts_status cnn_forward_tc(hts_cnn *net, const float *img, int H, int W, cudaStream_t s);
hts_status cnn_ensure_infer(hts_cnn *net, int H, int W, int nx);
// The same forward into caller-owned buffers: h0, h1 (H * W * 32 halves each)
// and map (H * W floats); only the weights and the error flag are the net's.
hts_status cnn_forward_tc_into(hts_cnn *net, const float *img, int H, int W, __half *h0, __half *h1, float *map,
                               cudaStream_t s);
struct Geom;
// Training loss (added to *loss) and its gradient map (dout, zeroed first) over the reference patches.
hts_status cnn_loss(const float *map, int H, int W, const Geom &g, const float *target, float *dout, double *loss,
                    cudaStream_t s);
// One image's loss and gradient (added to net->grad) on the tensor cores: FP16 activations and input
// gradients (loss scale 2^(floor(log2 N_ref) + 2)), FP32 accumulation of the weight gradients.
hts_status cnn_grad_tc(hts_cnn *net, const float *img, int H, int W, const Geom &g, const float *target,
                       cudaStream_t s);
// Noise level of every reference patch (sigma_ref, device, N_ref) through the
// readout window, from a forward into caller-owned buffers (rows: H * nx floats).
hts_status cnn_sigma_refs_into(hts_cnn *net, const float *img, const Geom &g, __half *h0, __half *h1, float *map,
                               float *rows, float *sigma_ref, cudaStream_t s);

}  // namespace hts
