// hts_denoise_noalloc: the same Haar-tSVD pipeline as hts_denoise, for
// callers that may not allocate device memory once they are running -- for
// example a plugin inside a host application that owns the whole device
// memory budget and forbids cudaMalloc after start-up, or a latency-critical
// loop where the implicit device synchronisation of cudaMalloc / cudaFree is
// not acceptable.  All intermediate buffers of the call live in one static
// device array of this file, sized for images of at most 512 x 512 pixels
// (any channel count the library supports), at most 65536 reference patches
// and at most 2^20 group slots (N_ref * K).  A GPU holds this array (about
// 21 MB) from the first call on it (with CUDA's lazy module loading the
// library's module, and the array with it, may be loaded only then) until the
// process exits.  The basis and noise-floor chain runs in series with the
// grouping on the caller's stream (hts_denoise overlaps them on a second
// stream), so a call takes somewhat longer; the result equals hts_denoise's
// up to 1e-3 on the [0, 255] scale (the same kernels run).
#include <mutex>

#include "hts_internal.h"

namespace hts {
namespace {

constexpr size_t NA_MAX_PIXELS = 512 * 512;  // H * W
constexpr int NA_MAX_NREF = 65536;           // reference patches
constexpr size_t NA_MAX_SLOTS = 1u << 20;    // N_ref * K
constexpr int NA_MAX_DEVICES = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte offsets of the carved buffers.
constexpr size_t OFF_STATE = 0;
constexpr size_t OFF_B64 = OFF_STATE + align256(sizeof(DevState));
constexpr size_t OFF_B32 = OFF_B64 + align256(2 * 256 * sizeof(double));
constexpr size_t OFF_EIG = OFF_B32 + align256(2 * 256 * sizeof(float));
constexpr size_t OFF_COV = OFF_EIG + align256(32 * sizeof(double));
// covariance sums (at most 2 x 608 blocks of 300 channel-pair entries, then the 600 totals; the
// launch checks cov_partial_count against this)
constexpr size_t COV_DOUBLES = (size_t)((NA_MAX_NREF + 63) / 64) * 600 + 600;
constexpr size_t OFF_IDX = OFF_COV + align256(COV_DOUBLES * sizeof(double));
constexpr size_t OFF_GREEN = OFF_IDX + align256(NA_MAX_SLOTS * sizeof(int32_t));
constexpr size_t OFF_FB = OFF_GREEN + align256(NA_MAX_NREF);
constexpr size_t OFF_REDO = OFF_FB + align256(NA_MAX_NREF * sizeof(int32_t));
constexpr size_t OFF_XLIST = OFF_REDO + align256(NA_MAX_NREF * sizeof(int32_t));
constexpr size_t OFF_XSKIP = OFF_XLIST + align256((size_t)NA_MAX_NREF * XLIST_PER_REF * 16);
constexpr size_t OFF_ACC = OFF_XSKIP + align256(NA_MAX_NREF);
constexpr size_t OFF_W = OFF_ACC + align256(3 * NA_MAX_PIXELS * sizeof(long long));
constexpr size_t NA_BYTES = OFF_W + align256(NA_MAX_PIXELS * sizeof(int));

}  // namespace

// The scratch of hts_denoise_noalloc.  Host code may not use its name as a
// device address: the address is obtained once per device with
// cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char hts_noalloc_scratch[NA_BYTES];

namespace {

std::mutex g_na_mu;
unsigned char *g_na_base[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch on the current device (looked up on the
// first call on that device and kept: after a reset of the device, e.g.
// cudaDeviceReset, the kept address is stale and the entry point must not be
// called again in this process).
hts_status scratch_base(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return report(HTS_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return report(HTS_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_base[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, hts_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return report(HTS_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_na_base[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_na_base[dev];
    return HTS_OK;
}

}  // namespace
}  // namespace hts

using namespace hts;

extern "C" hts_status hts_denoise_noalloc(const float *noisy, float *out, int H, int W, int C, float sigma,
                                          const hts_basis *basis, const hts_params *p, void *stream) {
    Geom g;
    hts_status st = validate(H, W, C, p, &g);
    if (st != HTS_OK) return st;
    if (!noisy || !out) return report(HTS_EINVAL, "NULL pointer");
    if (noisy == out) return report(HTS_EINVAL, "out may not alias noisy");
    if (sigma != sigma || sigma == __builtin_inff() || sigma == -__builtin_inff())
        return report(HTS_EINVAL, "sigma must be finite");
    if ((size_t)H * W > NA_MAX_PIXELS || g.nref > NA_MAX_NREF || (size_t)g.nref * g.K > NA_MAX_SLOTS)
        return report(HTS_EINVAL,
                      "image exceeds the static scratch of hts_denoise_noalloc (H*W <= 262144, N_ref <= 65536, "
                      "N_ref*K <= 1048576)");
    if (cov_partial_count(g) > COV_DOUBLES) return report(HTS_EINTERNAL, "covariance scratch too small");
    st = check_basis(basis, C);
    if (st != HTS_OK) return st;
    unsigned char *base = nullptr;
    st = scratch_base(&base);
    if (st != HTS_OK) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevState *ds = reinterpret_cast<DevState *>(base + OFF_STATE);
    double *b64 = reinterpret_cast<double *>(base + OFF_B64);
    float *b32 = reinterpret_cast<float *>(base + OFF_B32);
    double *eig = reinterpret_cast<double *>(base + OFF_EIG);
    double *cov = reinterpret_cast<double *>(base + OFF_COV);
    int32_t *idx = reinterpret_cast<int32_t *>(base + OFF_IDX);
    uint8_t *green = reinterpret_cast<uint8_t *>(base + OFF_GREEN);
    int32_t *fb = reinterpret_cast<int32_t *>(base + OFF_FB);
    int32_t *redo = reinterpret_cast<int32_t *>(base + OFF_REDO);
    int4 *xlist = reinterpret_cast<int4 *>(base + OFF_XLIST);
    uint8_t *xskip = reinterpret_cast<uint8_t *>(base + OFF_XSKIP);
    long long *acc = reinterpret_cast<long long *>(base + OFF_ACC);
    int *wcount = reinterpret_cast<int *>(base + OFF_W);
    const size_t hw = (size_t)H * W;

    // the scratch keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(ds, 0, sizeof(DevState), s) != cudaSuccess ||
        cudaMemsetAsync(acc, 0, hw * C * sizeof(long long), s) != cudaSuccess ||
        cudaMemsetAsync(wcount, 0, hw * sizeof(int), s) != cudaSuccess)
        return report(HTS_ECUDA, "cudaMemsetAsync of the static scratch failed");
    const bool est = (basis == nullptr) || (sigma < 0 && !basis->has_eig);
    if (est) {
        st = launch_basis(noisy, g, cov, b64, b32, eig, s);
        if (st != HTS_OK) return st;
    }
    const double *ub64 = basis ? basis->b64 : b64;
    const float *ub32 = basis ? basis->b32 : b32;
    const double *ueig = (basis && basis->has_eig) ? basis->eig : eig;
    st = launch_grouping(noisy, g, *p, idx, green, fb, ds, s);
    if (st != HTS_OK) return st;
    if (sigma < 0) st = launch_sigma(noisy, g, *p, ueig, idx, redo, ds, s);
    else st = launch_set_sigma(sigma > 0 ? (double)sigma : 0.0, g, *p, ds, s);
    if (st != HTS_OK) return st;
    return launch_filter(noisy, g, idx, ub64, ub32, acc, wcount, redo, xlist, xskip, ds, out,
                         p->precision == 0 ? 1 : 0, nullptr, 0, tau_scale(g, *p), s);
}
