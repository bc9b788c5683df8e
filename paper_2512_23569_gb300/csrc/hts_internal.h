// Internal declarations of the Haar-tSVD CUDA library (sm_103a).
// Not part of the public ABI (include/hts.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hts.h"

namespace hts {

constexpr int PS = 8;          // patch side (the only one built)
constexpr int NPIX = PS * PS;  // pixels per patch
constexpr int MAX_WIN = 63;    // largest search window side
constexpr double FIX_SCALE = 65536.0;  // 2^16: fixed-point scale of the aggregation sums

constexpr int LEARNED_PARTS = 160;  // blocks of the learned-map check

// Device-resident state of one call: noise level, threshold and counters.
// Bounds checks of the check build (compiled with -DHTS_CHECK, library libhts_check.so): a failed check
// records error code 3 in *errp and the guarded access is skipped; in the normal build the condition is not
// evaluated and the access always runs.
#ifdef HTS_CHECK
#define HTS_IN_BOUNDS(cond, errp) ((cond) ? true : (atomicExch((errp), 3), false))
#else
#define HTS_IN_BOUNDS(cond, errp) true
#endif

struct DevState {
    double sigma_est;
    double sigma_hat;
    double tau;
    float tau32;
    int votes;
    int vote_uncertain;
    int adjusted;
    int nref;
    int match_reranked;
    int match_fallback;   // length of the fallback list
    int filter_redo;      // length of the redo list
    int filter_exact;     // FP64 threshold decisions taken
    int filter_fixed;     // of which disagreed with FP32 and were corrected
    int xcount;           // in-band coefficients recorded by the main pass
    int error;
    int mtc_next;         // next (tile, plane pass) item of the tensor-core matcher's work queue
    int learned;          // 1: the learned noise map was used, 0: fell back to the estimate
    double learned_ratio; // geometric mean of (learned sigma / estimated sigma)
    double learned_part[LEARNED_PARTS];  // per-block sums of log(learned sigma)
};

// Basis on the device: [ns][2][8][8][2] (U then V, element [a][i], re/im).
struct hts_basis_dev {
    int C;
    int ns;
    int has_eig;
    int device;
    double *b64;  // ns*2*64*2 doubles
    float *b32;   // ns*2*64*2 floats
    double *eig;  // ns*2*8 doubles (ascending)
};

// Geometry of one call.
struct Geom {
    int H, W, C;
    int step, R, K;
    int ny, nx, nref;
};

inline int grid_count(int n, int step) {
    if (n < PS || step < 1) return 0;
    int c = (n - PS) / step + 1;
    if ((n - PS) % step != 0) c += 1;
    return c;
}

__host__ __device__ __forceinline__ int grid_pos(int i, int n, int step) {
    int p = i * step;
    return p < n - PS ? p : n - PS;
}

// Argument checks and error reporting shared by the entry points (api.cu).
hts_status validate(int H, int W, int C, const hts_params *p, Geom *g);
hts_status report(hts_status s, const char *msg);
// HTS_OK for DevState.error == 0, else the status of the failure it records
// (2: HTS_ETIMEOUT, a bounded wait gave up; 1: HTS_EINTERNAL).
hts_status device_status(int err);

// Launch bookkeeping (defined in api.cu).  Every kernel launch sits inside a
// KTimer scope: it counts the launch, opens an NVTX range named after the
// kernel (seen by profilers; a no-op without one) and, while profiling is on,
// records a CUDA event before and after it on the launch stream.
void count_launch();
void count_launches(unsigned long long n);
hts_status check_launch(const char *what);
// Launches recorded by this host thread into stream captures since the last
// reset (a captured launch is counted when its graph is launched).
unsigned long long captured_launches();
void reset_captured_launches();

// Host-side fault injection (test support, include/hts.h: hts_fault_inject).
// fault_take(k) is true for exactly the event of kind k that the armed
// countdown names (and disarms it); false otherwise.
enum FaultKind { FAULT_ALLOC = 0, FAULT_LAUNCH = 1, FAULT_WAIT = 2, FAULT_KINDS = 3 };
bool fault_take(FaultKind k);
// cudaMalloc through the allocation fault point.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}
// True while `s` is capturing into a CUDA graph.
bool stream_capturing(cudaStream_t s);
// cuTensorMapEncodeTiled of the driver (the library links only the runtime), as a
// PFN_cuTensorMapEncodeTiled_v12000; nullptr if the driver does not provide it.
void *tensor_map_encoder();

// Largest shared memory a block may opt in to on the current device.
int smem_optin();
// Sets, once per kernel and device, the kernel's dynamic shared memory
// attribute to the largest allowed value, and checks `need` against it.
hts_status allow_smem(const void *func, size_t need);
struct KTimer {
    int slot;
    bool range;  // an NVTX range was opened (launches outside stream captures)
    cudaStream_t stream;
    KTimer(const char *name, cudaStream_t s);
    ~KTimer();
};

// ---- matching (match.cu)
hts_status launch_match(const float *img, const Geom &g, double gamma_gcp, int32_t *idx, uint8_t *green,
                        int32_t *fallback_list, DevState *st, cudaStream_t s);

// Eq. 9 flag per reference (colour images; match.cu).
hts_status launch_gcp_flags(const float *img, const Geom &g, double gamma_gcp, uint8_t *green, cudaStream_t s);
// Precision form of the grouping (match_tc.cu): BF16 distances on the tensor
// cores, top-2K per reference, FP32 re-rank.  `green` must hold the Eq. 9
// flags (colour).  HTS_EUNSUPPORTED when the window does not fit on chip.
hts_status launch_match_tc(const float *img, const Geom &g, double gamma_gcp, int32_t *idx, const uint8_t *green,
                           int32_t *fallback_list, DevState *st, cudaStream_t s);
hts_status launch_match_rescue(const float *img, const Geom &g, int32_t *idx, const uint8_t *green,
                               int32_t *fallback_list, DevState *st, cudaStream_t s);

// The grouping step in the arithmetic p.precision selects (api.cu).
hts_status launch_grouping(const float *img, const Geom &g, const hts_params &p, int32_t *idx, uint8_t *green,
                           int32_t *fb, DevState *st, cudaStream_t s, bool flags_done = false);

// ---- global basis (basis.cu)
size_t cov_partial_count(const Geom &g);  // doubles needed for partial sums
hts_status launch_basis(const float *img, const Geom &g, double *partials, double *b64, float *b32, double *eig,
                        cudaStream_t s);

// ---- noise level (sigma.cu)
// `list`: N_ref int32 scratch for the groups whose rank test is taken in FP64
hts_status launch_sigma(const float *img, const Geom &g, const hts_params &p, const double *eig, const int32_t *idx,
                        int32_t *list, DevState *st, cudaStream_t s);
hts_status launch_set_sigma(double sigma, const Geom &g, const hts_params &p, DevState *st, cudaStream_t s);
// the three parts of launch_sigma, for callers that overlap them with other work
hts_status launch_sigma_floor(const Geom &g, const hts_params &p, const double *eig, DevState *st, cudaStream_t s);
hts_status launch_sigma_vote(const float *img, const Geom &g, const hts_params &p, const int32_t *idx,
                             int32_t *list, DevState *st, cudaStream_t s);
hts_status launch_sigma_final(const Geom &g, const hts_params &p, DevState *st, cudaStream_t s);

// ---- filtering and aggregation (filter.cu)
// xlist: XLIST_PER_REF * N_ref int4 entries for the in-band coefficients; xskip: N_ref
// bytes (see filter.cu).  exact = 0 (precision form): threshold decisions in FP32 only.
// sigma_ref (device, N_ref, may be nullptr): a noise level per group, threshold
// tau_scale * sigma_ref[r]; nullptr: the threshold in the call's state.  With
// map_judged = 1 the map is used only if DevState.learned is set (else the
// state's threshold).
constexpr int XLIST_PER_REF = 4;
// mean_est (device, N_ref x C x 64, may be nullptr; tensor-core filter only): the
// enhancement strategy's refined mean patch of every group, which replaces the
// group's first Haar row (Eq. 24-25).
hts_status launch_filter(const float *img, const Geom &g, const int32_t *idx, const double *b64, const float *b32,
                         long long *acc, int *wcount, int32_t *redo_list, int4 *xlist, uint8_t *xskip,
                         DevState *st, float *out, int exact, const float *sigma_ref, int map_judged,
                         double tau_scale, cudaStream_t s, const float *mean_est = nullptr);
double tau_scale(const Geom &g, const hts_params &p);  // sigma -> tau factor (sigma.cu)
// Tensor-core filter of the precision form (filter_tc.cu): FP16 projections of
// each Fourier slice on tcgen05, FP32 decisions, tile aggregation into acc /
// wcount (per slice for colour; no normalisation: normalize_box forms the
// weights and turns the slice sums into R, G, B).  *used = false (and nothing launched) where the group
// size or the window does not fit it.
hts_status launch_filter_tc(const float *img, const Geom &g, const int32_t *idx, const float *b32, long long *acc,
                            int *wcount, DevState *st, const float *sigma_ref, int map_judged, double tau_scale,
                            const float *mean_est, cudaStream_t s, bool *used);
// Enhancement strategy (fcn.cu): mean patch of every group (N_ref x C x 64,
// channel-major) and its refinement by the network with the state's sigma in
// the basis b32's coordinates (buf is overwritten; the refined patch in
// pixels lands in out).
hts_status launch_group_means(const float *img, const Geom &g, const int32_t *idx, float *means, cudaStream_t s);
hts_status fcn_refine_state(hts_fcn *f, float *buf, int n, const DevState *st, const float *b32, float *out,
                            cudaStream_t s);

// Filter tile shape (k_filter_tile): ty x tx reference positions per tile,
// ty = 0 for the non-local mode (no tile accumulators).  The launch uses, in
// this order: the thread's forced shape (set while autotuning), the tuned
// shape of the geometry, the largest listed shape that fits.
struct TileChoice {
    int ty, tx;
};
int tile_candidates(const Geom &g, TileChoice *out, int max);  // shapes valid for g, largest first
void force_tile(const TileChoice *c);                          // nullptr: off (per host thread)
bool tuned_tile(const Geom &g, TileChoice *out);
void set_tuned_tile(const Geom &g, TileChoice c);

// Device buffers of one image's pipeline: a stream's workspace, or one slot
// of a batch arena.  aux / ev_fork / ev_join: the second stream and the two
// events of the basis chain's fork and join.
struct Bufs {
    int32_t *idx = nullptr;
    uint8_t *green = nullptr;
    int32_t *fb = nullptr;
    int32_t *redo = nullptr;
    int4 *xlist = nullptr;
    uint8_t *xskip = nullptr;
    long long *acc = nullptr;
    int *wcount = nullptr;
    double *cov = nullptr;
    double *b64 = nullptr;
    float *b32 = nullptr;
    double *eig = nullptr;
    DevState *st = nullptr;
    float *sref = nullptr;  // a noise level per reference patch (batched learned form)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};
size_t bufs_bytes(const Geom &g);                              // arena bytes of one image
void bufs_carve(const Geom &g, unsigned char *base, Bufs *b);  // device pointers (not aux / events)
// Learned noise map check (cnn.cu): geometric mean of sigma_ref / the
// estimated sigma_hat; sets DevState.learned (1 if inside [1/factor, factor]
// and the map is finite and positive) and learned_ratio.
hts_status launch_learned_check(const float *sigma_ref, int nref, double factor, DevState *st, cudaStream_t s);
// Noise level of every reference patch from the learned network (device, N_ref; cnn.cu).
hts_status cnn_sigma_refs(hts_cnn *n, const float *img, const Geom &g, float *sigma_ref, cudaStream_t s);
// Batched launches of the tensor-core kernels over the images of a batch (match_tc.cu, filter_tc.cu):
// *_job writes an image's arguments (job_size bytes, host memory) and returns its work items (matcher:
// tiles x plane passes; filter: tiles, -1 if the tensor-core filter does not take the geometry); the
// launches read the job table and the prefix sums of the items from device memory.
size_t match_tc_job_size();
int match_tc_job(const float *img, const Geom &g, int32_t *idx, const uint8_t *green, int32_t *fallback_list,
                 DevState *st, void *job);
hts_status launch_match_tc_batch(int K, const void *jobs_host, const void *jobs_dev, const int *item_start_dev,
                                 int njobs, int nitems, int *queue_dev, int grid, cudaStream_t s);
size_t filter_tc_job_size();
// force_shape >= 0: the filter's tile shape number force_shape (8x8, 4x8, 4x4, 2x4, ...) where it fits.
int filter_tc_job(const float *img, const Geom &g, const int32_t *idx, const float *b32, long long *acc, int *wcount,
                  DevState *st, const float *sigma_ref, int map_judged, double tau_scale, int nsm, void *job,
                  int force_shape = -1);
hts_status launch_filter_tc_batch(int C, int K, const void *jobs_host, const void *jobs_dev, const int *tile_start_dev,
                                  int njobs, int ntiles, int grid, cudaStream_t s);
// Pixel weights from the tensor-core filter's patch-origin counts, and the normalisation (filter.cu).
hts_status launch_normalize_box(const long long *acc, const int *cnt, float *out, int H, int W, int C, cudaStream_t s);

// Releases every batch plan (batch.cu).
void batch_shutdown();
// The whole method for one image on stream s with the buffers of b (api.cu).
// sigma_ref (device, N_ref, may be nullptr): a noise level per reference
// patch; with a fallback factor > 0 it is checked against the estimated
// level (launch_learned_check) and the estimate is used if it fails.
// fcn (may be nullptr) with ra_buf (2 N_ref C 64 floats): the enhancement strategy.
// map_ready (may be nullptr): an event s waits for before the first use of sigma_ref.
hts_status denoise_run(const float *noisy, float *out, const Geom &g, float sigma, const hts_basis *basis,
                       const hts_params &p, const Bufs &b, cudaStream_t s, float *sigma_ref = nullptr,
                       double fallback_factor = 0.0, hts_fcn *fcn = nullptr, float *ra_buf = nullptr,
                       cudaEvent_t map_ready = nullptr);
// Destroys the batch plans that use this network (batch.cu; hts_cnn_free calls it).
void batch_drop_net(const hts_cnn *net);

}  // namespace hts

// The opaque handle of the public header.
struct hts_basis : hts::hts_basis_dev {};

namespace hts {
hts_status check_basis(const hts_basis *basis, int C);
}  // namespace hts
