/*
 * hts.h -- C ABI of the GB300 (sm_103a) Haar-tSVD denoiser.
 *
 * Haar-tSVD ("Image Denoising Using Global and Local Circulant
 * Representation", Kong, Yang, Zhang, arXiv 2512.23569) is a one-step
 * patch-based denoiser: every reference patch is grouped with its K nearest
 * patches (Eq. 9, Alg. 1 step 1), the group is projected on a global t-SVD
 * basis combined with a Haar transform along the group axis (Eq. 19), hard
 * thresholded (Eq. 20), transformed back (Eq. 21) and averaged into the
 * output (Alg. 1 step 3).  The noise level can be estimated from the
 * eigenvalues of the circulant structures (Eq. 12, 22, 23).
 *
 * Conventions shared by every call:
 *   - Images are planar CHW float32, row-major, contiguous, C in {1, 3}
 *     (channel order R, G, B), values on any scale (the method's parameters
 *     assume [0, 255]).
 *   - Image pointers are DEVICE pointers unless the name says `host`.  The
 *     caller owns every buffer it passes; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it unless their comment says they synchronise.
 *   - Every call validates its arguments on the host first and returns
 *     HTS_EINVAL / HTS_EUNSUPPORTED before launching anything.  On any
 *     failure `hts_last_error()` returns a message (per host thread).
 *   - The library keeps a device workspace per (device, stream), grown on
 *     demand with cudaMalloc and released by hts_shutdown().  Two calls in
 *     flight on the same stream are ordered by the stream; calls on different
 *     streams use different workspaces.
 *   - There is no CPU fallback: every step runs in the library's kernels.
 */
#ifndef HTS_H
#define HTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HTS_OK = 0,
    HTS_EINVAL = 1,        /* bad argument (checked before any device work) */
    HTS_ENOMEM = 2,        /* device or host allocation failed */
    HTS_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    HTS_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    HTS_EUNSUPPORTED = 5,  /* valid for the method, not built here (e.g. ps != 8) */
    HTS_EINTERNAL = 6      /* a device-side consistency check failed */
} hts_status;

/* Method parameters.  Defaults (hts_params_default) follow Sec. IV-A of the
 * paper (ps = 8, gamma = 1.2 in Eq. 9, beta = 1.2 and gamma = 13 for K = 32
 * in Eq. 23, tau = sigma sqrt(2 ln(c K ps^2))) with K = 16, win = 21, step 4,
 * precision 0. */
typedef struct {
    int ps;            /* patch side; only 8 is built (else HTS_EUNSUPPORTED) */
    int K;             /* patches per group: 2, 4, 8, 16 or 32 (Haar needs 2^n, Eq. 8) */
    int win;           /* search window side: odd, 3..63, centred on the reference corner */
    int step;          /* reference grid step, 1..ps; the last row/column n-ps is always added */
    double gamma_gcp;  /* Eq. 9 green-channel weight (> 0) */
    double beta;       /* Eq. 23 divisor (> 0) */
    double gamma_rank; /* Eq. 23 rank threshold; <= 0 selects 13 K / 32 */
    double tau_mult;   /* multiplier on the universal threshold (>= 0) */
    int adjust_rank;   /* 1: apply the Eq. 22-23 vote when sigma is estimated */
    int mp_correct;    /* 1: divide the Eq. 12 floor by the Marchenko-Pastur edge (1-1/sqrt(N_ref))^2 */
    int precision;     /* arithmetic of the grouping and the filter.
                        * 0: FP32 distances certified against FP64 (the groups equal the FP64
                        *    definition's, ties to the lower index); FP32 transforms with FP64
                        *    threshold decisions inside the FP32 error band.
                        * 1: precision form: BF16 distances on the tensor cores (FP32
                        *    accumulation), the 2K nearest (at least K + 8) re-ranked with FP32
                        *    distances (groups may differ from the FP64 definition's where BF16
                        *    rounding reorders near neighbours; a reference whose candidate
                        *    bins may have dropped one of its K + 3 nearest is matched
                        *    exhaustively in FP32); FP16 projections on the tensor cores (FP32
                        *    accumulation) with FP32 threshold decisions.  Windows too large for
                        *    on-chip staging give HTS_EUNSUPPORTED.  The FP16 operands and the
                        *    filter's 32-bit tile sums assume pixel values of magnitude below
                        *    2^11 (the [0, 255] scale has ample room); estimates beyond 2^13 (of a
                        *    channel-DFT slice, summed before the inverse DFT) are clamped.
                        * 2: the groups of 0 with the filter of 1. */
} hts_params;

/* Fills *p with the defaults above.  HTS_EINVAL if p is NULL. */
hts_status hts_params_default(hts_params *p);

/* ---------------------------------------------------------------- basis */

/* Opaque global t-SVD basis (Eq. 11): for every stored Fourier slice j of
 * mode 3 (1 slice for C = 1, 2 for C = 3; slice 3 is the conjugate of slice
 * 2) the 8 x 8 pair (U^(j), V^(j)), kept on the device in FP64 and FP32, plus
 * the eigenvalues it was derived from. */
typedef struct hts_basis hts_basis;

/* Globally-learned basis (Sec. III-B2, Eq. 11): eigenvectors of the row and
 * column covariances of all reference patches of `img` (device, CHW),
 * accumulated and eigendecomposed in FP64 on the device.  *out receives a new
 * basis owned by the caller (free with hts_basis_free).  Synchronises on
 * `stream` before returning. */
hts_status hts_estimate_basis(const float *img, int H, int W, int C, const hts_params *p,
                              hts_basis **out, void *stream);

/* Builds a basis from host data (globally-reused variant, Sec. III-B2).
 * host_basis: float64 array [ns][2][8][8][2] with ns = C/2+1; [j][0] is
 * U^(j), [j][1] is V^(j), element [a][i] is row a of eigenvector i, last index
 * (re, im).  host_eigvals: optional float64 [ns][2][8] (may be NULL).
 * Slice 0 must be real (imaginary parts zero).  Matrices must be unitary to
 * 1e-6 (checked).  Synchronous. */
hts_status hts_basis_create(const double *host_basis, const double *host_eigvals, int C, hts_basis **out);

/* Copies a basis to host arrays laid out as in hts_basis_create (either
 * pointer may be NULL); *C_out (optional) receives the channel count. */
hts_status hts_basis_read(const hts_basis *b, double *host_basis, double *host_eigvals, int *C_out);

/* Releases a basis (NULL is a no-op). */
hts_status hts_basis_free(hts_basis *b);

/* Saves / loads a basis to / from a small binary file (magic "HTSB1"). */
hts_status hts_basis_save(const hts_basis *b, const char *path);
hts_status hts_basis_load(const char *path, hts_basis **out);

/* ---------------------------------------------------------- noise level */

typedef struct {
    double sigma_hat;   /* final estimate (Eq. 23 applied) */
    double sigma_est;   /* covariance floor (Eq. 12) before the vote */
    int votes;          /* groups whose rank position of lambda_hat is <= gamma_rank */
    int nref;           /* number of groups (reference patches) */
    int adjusted;       /* 1 if a strict majority voted and sigma_est was divided by beta */
    int uncertain;      /* groups whose FP32 rank test was re-evaluated in FP64 */
} hts_sigma_info;

/* Noise level of `img` (device, CHW): sigma_est from the smallest eigenvalue
 * of the global covariances (Eq. 12: the noise adds ps * N_ref * sigma^2),
 * then every group votes with the rank position of lambda_hat (Eq. 22) and a
 * strict majority divides by beta (Eq. 23).  basis: the covariances'
 * eigenvalues are taken from it when non-NULL (it must have been estimated,
 * not created without eigenvalues), else estimated.  Writes *sigma_out (host)
 * and *info (optional).  Synchronises on `stream`; HTS_ETIMEOUT / HTS_EINTERNAL
 * if a kernel recorded a failure (the outputs are then invalid). */
hts_status hts_estimate_sigma(const float *img, int H, int W, int C, const hts_basis *basis,
                              const hts_params *p, double *sigma_out, hts_sigma_info *info, void *stream);

/* ------------------------------------------------------------- denoise */

/* Haar-tSVD (Alg. 1) of `noisy` into `out` (device, CHW, may not alias).
 * sigma >= 0: known noise level; sigma < 0: estimated on the device as in
 * hts_estimate_sigma (nothing is copied to the host).  basis NULL: the
 * globally-learned basis of `noisy` is estimated on the device.  Output is
 * the plain average of all group estimates, not clipped.  Asynchronous. */
hts_status hts_denoise(const float *noisy, float *out, int H, int W, int C, float sigma,
                       const hts_basis *basis, const hts_params *p, void *stream);

/* hts_denoise without any device allocation, for callers that may not
 * allocate device memory once they are running: for example a plugin inside
 * a host application that owns the whole device memory budget and forbids
 * cudaMalloc after start-up, or a latency-critical loop that cannot afford
 * the implicit device synchronisation of cudaMalloc / cudaFree.  The paper
 * has no counterpart; this is a deployment variant of hts_denoise.
 * All intermediate buffers live in one static device array of the library
 * (about 21 MB).  A GPU holds it from the first call on that GPU (CUDA may
 * load the library's device code, and the array with it, only then) until
 * the process exits, so make the first call at start-up.  That bounds the
 * image: H*W <= 262144 pixels, at most 65536 reference patches and
 * N_ref*K <= 1048576; larger images return HTS_EINVAL before any device work.
 * The caller still passes `noisy` and `out` (device); every other argument
 * (a caller's basis must live on the current device and match C) is as for
 * hts_denoise, and the result equals hts_denoise's within 1e-3 on the
 * [0, 255] scale.  Unlike hts_denoise, the basis estimate runs in series with
 * the grouping on `stream` (no second stream), so a call takes a little
 * longer.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it: make that first call before any
 * stream capture, and do not call this entry point again after resetting the
 * device.  All calls share the one array and each overwrites what the
 * previous call left there, so calls that overlap on the GPU (other streams,
 * or host threads without ordering) race and corrupt each other's results;
 * serialise them.  Asynchronous. */
hts_status hts_denoise_noalloc(const float *noisy, float *out, int H, int W, int C, float sigma,
                               const hts_basis *basis, const hts_params *p, void *stream);

/* hts_denoise on HOST buffers: copies noisy_host to the device, denoises and
 * copies the result back into out_host, all on `stream`, then synchronises.
 * Pinned host memory is fastest but not required.  HTS_ETIMEOUT /
 * HTS_EINTERNAL if a kernel recorded a failure (out_host is then invalid). */
hts_status hts_denoise_host(const float *noisy_host, float *out_host, int H, int W, int C, float sigma,
                            const hts_basis *basis, const hts_params *p, void *stream);

/* One image of a batch. */
typedef struct {
    const float *noisy;       /* device, CHW */
    float *out;               /* device, CHW */
    int H, W, C;
    float sigma;              /* < 0: estimate (ignored where sigma_map is given) */
    const hts_params *params; /* NULL: the batch's parameters (read at the call, not kept) */
    const float *sigma_map;   /* NULL, or a noise level per reference patch (device, N_ref floats,
                               * raster order of the reference grid): the image is denoised as by
                               * hts_denoise_sigma_map (Eq. 20 with a local sigma) */
} hts_image;

/* Denoises n independent images (mixed sizes and channel counts, sigma known
 * or estimated per image), each with its own globally-learned basis, as ONE
 * CUDA-graph launch on `stream`: every image's whole pipeline is captured into
 * a graph whose branches run concurrently on several internal streams, with
 * all buffers in one device arena per batch signature (the list of H, W, C,
 * sigma-estimated flags and parameters of every image).  The first call of a signature
 * allocates the arena, autotunes (times every valid filter tile shape per
 * image geometry not tuned before, and the graph on 1, 2, 4 and 8 concurrent
 * streams) and synchronises; later calls with the same signature reuse the
 * graph (updating it in place when pointers or sigma values change) and are
 * asynchronous.  The output equals hts_denoise's on each image, bit for bit,
 * whatever the tuning chose.  Up to 4 signatures are kept per process (least
 * recently used dropped, hts_shutdown frees all).  Calls are serialised
 * across host threads. */
hts_status hts_denoise_batch(const hts_image *imgs, int n, const hts_params *p, void *stream);

/* Schedule of the last hts_denoise_batch on a stream. */
typedef struct {
    int images;    /* images in the batch */
    int lanes;     /* concurrent streams the autotuner chose */
    int kernels;   /* kernel launches per graph launch */
    int captures;  /* graph captures made for this signature so far */
    int updates;   /* in-place graph updates (new pointers / sigma) so far */
    int phased;    /* 1: every image is in a tensor-core form (precision 1 or 2), and the tensor-core
                    * matcher and filter each run as one persistent launch per group of images (same K;
                    * filter: same C and K) over a device work queue of (image, tile) items, between
                    * the per-image steps on the lanes; 0: one pipeline per image on the lanes */
} hts_batch_info;

/* Filter tile shape chosen by the autotuner for this geometry (*ty x *tx
 * reference positions per tile; 0 x 0 = the non-local mode) or -1 x -1 if the
 * geometry has not been tuned in this process. */
hts_status hts_tuned_tile(int H, int W, int C, const hts_params *p, int *ty, int *tx);

/* ------------------------------------------- spatially varying noise */

/* hts_denoise with a noise level per reference patch: group r is thresholded
 * at tau_mult * sigma_ref[r] * sqrt(2 ln(c K ps^2)) (Eq. 20 with a local
 * sigma).  sigma_ref: device float array of N_ref values (hts_num_refs),
 * raster order of the reference grid.  Asynchronous. */
hts_status hts_denoise_sigma_map(const float *noisy, float *out, int H, int W, int C, const float *sigma_ref,
                                 const hts_basis *basis, const hts_params *p, void *stream);

/* Learned noise-level map: the convolutional estimate that the adaptive
 * variant of the paper (Sec. III-C) uses in place of one global level.  Five
 * 3x3 convolutions (C -> 32 -> 32 -> 32 -> 32 -> 1, ReLU between, zero
 * padding) map the image / 255 to a dense log(sigma) map.  Training reads
 * the map at the centre (y + 4, x + 4) of reference patch (y, x); denoising
 * gives the patch exp(mean of the map over the window of S x S pixels
 * starting S/2 rows and columns before that centre, cut to the image) --
 * the paper estimates one level per sub-image, the window is that sub-image
 * moved with the patch (S = 128 by default, S = 1 is the centre alone).
 * FP16 weights, FP32 accumulation, trained by the library's own kernels
 * (mean squared error of log sigma over the reference patches, Adam).  A
 * network is not thread-safe. */
typedef struct hts_cnn hts_cnn;
int hts_cnn_num_params(int C); /* 0 for C not in {1, 3} */
int hts_cnn_channels(const hts_cnn *net); /* C of the network, 0 for NULL */
/* New network for C channels, He-initialised from `seed`; synchronous. */
hts_status hts_cnn_create(int C, uint64_t seed, hts_cnn **out);
hts_status hts_cnn_free(hts_cnn *net);
/* FP32 master parameters, per layer W[co][ci][3][3] then b[co] (host arrays of
 * hts_cnn_num_params(C) floats); set also resets the optimiser state.  Synchronous. */
hts_status hts_cnn_get_params(const hts_cnn *net, float *host_params);
hts_status hts_cnn_set_params(hts_cnn *net, const float *host_params);
/* Forward pass used for denoising: log-sigma map (device, H x W) of a device
 * CHW image, on the tensor cores with the network input and the hidden
 * activations rounded to FP16 (the same forward as tensor-core training). */
hts_status hts_cnn_log_sigma_map(hts_cnn *net, const float *img, int H, int W, float *map_out, void *stream);
/* Readout window S (1 <= S <= 4096) of hts_cnn_sigma_refs / hts_denoise_learned. */
hts_status hts_cnn_set_window(hts_cnn *net, int S);
int hts_cnn_window(const hts_cnn *net); /* 0 for NULL */
/* sigma at every reference patch through the readout window (device, N_ref). */
hts_status hts_cnn_sigma_refs(hts_cnn *net, const float *img, int H, int W, const hts_params *p,
                              float *sigma_ref, void *stream);
/* Training: gradients accumulate over images until hts_cnn_zero_grad; the
 * loss (mean squared error of log sigma against target_log_sigma, device,
 * N_ref) accumulates until hts_cnn_take_loss (synchronises).  By default a
 * training step runs on the tensor cores: the forward of
 * hts_cnn_log_sigma_map keeping every layer's FP16 activations, the
 * gradients of the layer inputs in FP16 (the loss gradient scaled by
 * 2^(floor(log2 N_ref) + 2), the scale divided out of the weight
 * gradients), the weight and bias
 * gradients accumulated in FP32.  hts_cnn_set_train_fp16(net, 0) selects
 * the FP32 kernels instead (FP32 activations and gradients); either setting
 * keeps FP32 master parameters and FP32 Adam state.  If a bounded wait of a
 * training kernel gives up, the layer's gradient becomes NaN. */
hts_status hts_cnn_set_train_fp16(hts_cnn *net, int on);
int hts_cnn_train_fp16(const hts_cnn *net); /* 1: tensor-core training (default), 0: FP32, -1 for NULL */
hts_status hts_cnn_zero_grad(hts_cnn *net, void *stream);
hts_status hts_cnn_accumulate_grad(hts_cnn *net, const float *img, int H, int W, const hts_params *p,
                                   const float *target_log_sigma, void *stream);
hts_status hts_cnn_take_loss(hts_cnn *net, double *loss_sum, void *stream);
hts_status hts_cnn_get_grad(const hts_cnn *net, float *host_grad, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the accumulated gradient. */
hts_status hts_cnn_adam_step(hts_cnn *net, float lr, void *stream);
/* Parameters and readout window to / from a small binary file (magic "HTSCNN2"). */
hts_status hts_cnn_save(const hts_cnn *net, const char *path);
hts_status hts_cnn_load(const char *path, hts_cnn **out);

/* Denoising with the learned map checked against the eigenvalue estimate of
 * hts_estimate_sigma: if the geometric mean of learned / estimated sigma lies
 * outside [1/fallback_factor, fallback_factor] (or the map is not finite and
 * positive), every group falls back to the estimate; hts_last_stats reports
 * which was used and the ratio.  fallback_factor > 1.  Asynchronous. */
hts_status hts_denoise_learned(const float *noisy, float *out, int H, int W, int C, hts_cnn *net,
                               const hts_basis *basis, const hts_params *p, double fallback_factor, void *stream);

/* hts_denoise_learned on HOST buffers (the host-to-device copy, the call and
 * the device-to-host copy on `stream`, then a synchronisation), as
 * hts_denoise_host is to hts_denoise.  HTS_ETIMEOUT / HTS_EINTERNAL if a
 * kernel recorded a failure (out_host is then invalid). */
hts_status hts_denoise_learned_host(const float *noisy_host, float *out_host, int H, int W, int C, hts_cnn *net,
                                    const hts_basis *basis, const hts_params *p, double fallback_factor,
                                    void *stream);

/* The batched learned form: hts_denoise_batch in which every image's noise
 * level per reference patch comes from the network `net` (as in
 * hts_denoise_learned, Sec. III-C), checked against the image's eigenvalue
 * estimate (Eq. 12, 22-23) with `fallback_factor` (> 1).  The networks'
 * forward passes run inside the same graph launch, one image after another
 * (largest first) on a stream of their own, into buffers the batch's plan
 * owns; each image's filter waits only for its own map.  Every image must have
 * net's channel count and no sigma_map; sigma is ignored.  The plan keeps
 * `net` (its weights are read at every launch, so training between calls is
 * seen); hts_cnn_free drops the plans that use it.  Output equals
 * hts_denoise_learned's on each image, bit for bit.  hts_last_batch_stats
 * reports each image's learned / learned_ratio. */
hts_status hts_denoise_batch_learned(const hts_image *imgs, int n, hts_cnn *net, double fallback_factor,
                                     const hts_params *p, void *stream);

/* -------------------------------------- enhancement strategy (RA-Haar-tSVD) */

/* RA-Haar-tSVD (Eq. 24-25): the first Haar row of every group -- sqrt(K)
 * times its mean patch in the transform domain -- is replaced by sqrt(K)
 * times the transform of the mean patch refined by a plain fully connected
 * network, and kept whole (not thresholded); the other rows are filtered as
 * usual.  The network sees the mean patch c in the image's transform
 * coordinates (hts_mean_coefs; pixels channel-major, t * 64 + u * 8 + v) in
 * units of its noise level s = sigma / sqrt(K): input g(c / s), g(x) = x /
 * (1 + |x| / 16), then sigma / 255, zero-padded to a multiple of 16; two
 * hidden layers of 128 ReLU units; linear output r of C x 64 values;
 * refined = c + s r (residual learning).  FP32 weights and arithmetic,
 * trained by the library's own kernels (mean squared error of r against
 * (clean - noisy) / s, Adam).  Not thread-safe. */
typedef struct hts_fcn hts_fcn;
int hts_fcn_num_params(int C); /* 0 for C not in {1, 3} */
int hts_fcn_channels(const hts_fcn *fcn);
int hts_fcn_group_size(const hts_fcn *fcn); /* K of the network, 0 for NULL */
/* New network for C channels and groups of K patches (He initialisation from
 * `seed`, output layer scaled by 0.1, zero biases); synchronous. */
hts_status hts_fcn_create(int C, int K, uint64_t seed, hts_fcn **out);
hts_status hts_fcn_free(hts_fcn *fcn);
/* Parameters, per layer W[out][in] then b[out] (host, hts_fcn_num_params(C)
 * floats); set resets the optimiser state.  Synchronous. */
hts_status hts_fcn_get_params(const hts_fcn *fcn, float *host_params);
hts_status hts_fcn_set_params(hts_fcn *fcn, const float *host_params);
/* Mean patch of every group (device: idx N_ref x K from hts_match, means out
 * N_ref x C x 64). */
hts_status hts_group_means(const float *img, int H, int W, int C, const hts_params *p, const int32_t *idx,
                           float *means, void *stream);
/* The image transform of n patches (Eq. 19 without the Haar factor; device,
 * n x C x 64 in and out): [S^(1), sqrt 2 Re S^(2), sqrt 2 Im S^(2)] (C = 3,
 * orthonormal) or S^(1) (C = 1), with the given basis; inverse != 0 maps
 * coordinates back to pixels.  The network reads and refines these. */
hts_status hts_mean_coefs(const float *in, int n, int C, const hts_basis *basis, int inverse, float *out,
                          void *stream);
/* Refined coordinates of n mean patches (device: coords n x C x 64, sigma n
 * values, refined out n x C x 64). */
hts_status hts_fcn_refine(hts_fcn *fcn, const float *means, const float *sigma, int n, float *refined, void *stream);
/* Training on n pairs (device: noisy and clean mean-patch coordinates
 * n x C x 64, the noise level of each); gradients add up until
 * hts_fcn_zero_grad, the loss (mean over the n x C x 64 values) until
 * hts_fcn_take_loss (synchronises). */
hts_status hts_fcn_zero_grad(hts_fcn *fcn, void *stream);
hts_status hts_fcn_accumulate_grad(hts_fcn *fcn, const float *noisy_means, const float *clean_means,
                                   const float *sigma, int n, void *stream);
hts_status hts_fcn_take_loss(hts_fcn *fcn, double *loss_sum, void *stream);
hts_status hts_fcn_get_grad(const hts_fcn *fcn, float *host_grad, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected). */
hts_status hts_fcn_adam_step(hts_fcn *fcn, float lr, void *stream);
/* hts_denoise with the enhancement strategy; the network sees the call's
 * sigma (given, or estimated as in hts_denoise).  Needs the tensor-core
 * filter: p->precision 1 or 2 (else HTS_EUNSUPPORTED).  Asynchronous. */
hts_status hts_denoise_ra(const float *noisy, float *out, int H, int W, int C, float sigma, hts_fcn *fcn,
                          const hts_basis *basis, const hts_params *p, void *stream);

/* ------------------------------------------------- inspection / tests */

/* Grouping step alone (Eq. 9, Alg. 1 step 1): idx_out (device, int32,
 * N_ref x K) receives raster indices y*W+x of the group members' top-left
 * corners; slot 0 is the reference, then the K-1 nearest other candidates
 * in ascending (squared distance, raster index).  green_out (device,
 * uint8 N_ref, may be NULL) receives the Eq. 9 flag.  N_ref = ny * nx with
 * ny = number of grid positions 0, step, ... plus H-8.  Asynchronous. */
hts_status hts_match(const float *img, int H, int W, int C, const hts_params *p,
                     int32_t *idx_out, uint8_t *green_out, void *stream);

/* Number of reference patches for an H x W image (0 on bad input). */
int hts_num_refs(int H, int W, const hts_params *p);

/* Counters of the last hts_denoise / hts_match / hts_estimate_sigma call on
 * `stream` (synchronises on it). */
typedef struct {
    int nref;
    int match_reranked;    /* references whose order was settled by the FP64 re-rank */
    int match_fallback;    /* references matched by the exhaustive FP64 path */
    int filter_redo;       /* groups recomputed by the FP64 exact pass (in-band list full) */
    int filter_exact;      /* coefficients whose threshold decision was taken in FP64 */
    int vote_uncertain;    /* groups whose rank test was taken in FP64 */
    double sigma;          /* noise level used */
    double tau;            /* threshold used */
    int filter_fixed;      /* FP64 decisions that overturned the FP32 one (contribution corrected) */
    int learned;           /* hts_denoise_learned: 1 = learned noise map used, 0 = fell back */
    double learned_ratio;  /* hts_denoise_learned: geometric mean of learned / estimated sigma */
    int device_error;      /* failure the kernels recorded: 0 none, 2 a bounded wait gave up, 1 a
                            * consistency check failed */
} hts_stats;
/* Fills *out and returns HTS_OK, or HTS_ETIMEOUT (device_error 2) / HTS_EINTERNAL
 * (device_error 1) when a kernel of that call recorded a failure: its result is
 * then invalid.  This is how the asynchronous calls report device-side failures. */
hts_status hts_last_stats(hts_stats *out, void *stream);

/* Per-image counters (out[0..n-1], as hts_last_stats) and, if info is not
 * NULL, the schedule of the last hts_denoise_batch on `stream`.  HTS_EINVAL if
 * no batch ran there; HTS_ETIMEOUT / HTS_EINTERNAL if a kernel recorded a
 * failure for one of the images (its device_error says which).  Synchronises. */
hts_status hts_last_batch_stats(hts_stats *out, int n, hts_batch_info *info, void *stream);

/* Kernel timing: between hts_profile_begin() and hts_profile_end() every
 * kernel launch of the library is bracketed by CUDA events recorded on its
 * launch stream.  hts_profile_end synchronises on those events and writes up
 * to `max` entries (one per kernel name: summed milliseconds and number of
 * launches); *n_out receives the number written.  Process-wide. */
typedef struct {
    char name[48];
    double total_ms;
    int launches;
} hts_kernel_time;
hts_status hts_profile_begin(void);
hts_status hts_profile_end(hts_kernel_time *out, int max, int *n_out);

/* Host-side fault injection, for tests of the failure paths (nothing is made
 * to fault on the GPU).  spec: comma-separated "kind:N" items, N >= 1, each arming a
 * one-shot countdown: the N-th event of that kind from now on fails; NULL or ""
 * disarms all.  Kinds:
 *   alloc:N   the N-th device allocation of the library fails as out of memory
 *             (the call returns HTS_ENOMEM; nothing is allocated);
 *   launch:N  the N-th kernel launch is reported as failed (the call returns
 *             HTS_ECUDA; the library stays usable);
 *   wait:N    in the N-th launch of the tensor-core matcher (precision 1) the
 *             thread that issues the MMAs first waits on a barrier that nothing
 *             arrives on; the bounded wait gives up after a few thousand polls, the
 *             kernel records the failure and gives every reference its own position
 *             as its group (HTS_ETIMEOUT where the state is read back:
 *             hts_last_stats, hts_denoise_host, hts_estimate_sigma).
 * Launches inside a stream capture are never counted.  The environment variable
 * HTS_FAULT (same syntax) arms the countdowns at the library's first event.
 * Process-wide.  HTS_EINVAL on a malformed spec (nothing changes). */
hts_status hts_fault_inject(const char *spec);

/* Thread-local message for the last failing call on this host thread. */
const char *hts_last_error(void);

/* Number of kernels this library has launched since it was loaded. */
uint64_t hts_launch_count(void);

/* Library version string. */
const char *hts_version(void);

/* Frees every workspace on every device.  No call may be in flight. */
hts_status hts_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* HTS_H */
