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

// Device-resident state of one call: noise level, threshold and counters.
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

// Launch bookkeeping (defined in api.cu).  Every kernel launch sits inside a
// KTimer scope: it counts the launch and, while profiling is on, records a
// CUDA event before and after it on the launch stream.
void count_launch();
hts_status check_launch(const char *what);
struct KTimer {
    int slot;
    cudaStream_t stream;
    KTimer(const char *name, cudaStream_t s);
    ~KTimer();
};

// ---- matching (match.cu)
hts_status launch_match(const float *img, const Geom &g, double gamma_gcp, int32_t *idx, uint8_t *green,
                        int32_t *fallback_list, DevState *st, cudaStream_t s);

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
// xlist: N_ref int4 entries for the in-band coefficients; xskip: N_ref bytes (see filter.cu)
hts_status launch_filter(const float *img, const Geom &g, const int32_t *idx, const double *b64, const float *b32,
                         long long *acc, int *wcount, int32_t *redo_list, int4 *xlist, uint8_t *xskip,
                         DevState *st, float *out, cudaStream_t s);

}  // namespace hts

// The opaque handle of the public header.
struct hts_basis : hts::hts_basis_dev {};

namespace hts {
hts_status check_basis(const hts_basis *basis, int C);
}  // namespace hts
