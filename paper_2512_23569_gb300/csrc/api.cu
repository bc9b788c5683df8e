// C ABI of the Haar-tSVD library (include/hts.h): argument validation,
// per-(device, stream) workspaces and the order of the kernel launches.
// Every step of the method runs in the kernels of match.cu, basis.cu,
// sigma.cu and filter.cu; the host only validates and launches.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hts_internal.h"


namespace hts {

static std::atomic<unsigned long long> g_launches{0};
static thread_local std::string g_err;
static thread_local unsigned long long g_captured = 0;
static thread_local bool g_launch_fault = false;  // an injected launch failure awaits its check_launch

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long captured_launches() { return g_captured; }
void reset_captured_launches() { g_captured = 0; }

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

bool stream_capturing(cudaStream_t s) { return capturing(s); }

void *tensor_map_encoder() {
    static void *fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = p;
        else
            cudaGetLastError();
    });
    return fn;
}

// ------------------------------------------------------- fault injection

// One-shot countdowns per kind (0 = disarmed): the N-th event of the kind
// after arming fails.  Armed by hts_fault_inject, or once, at the library's
// first event, from the environment variable HTS_FAULT (same syntax).
static std::atomic<long long> g_fault[FAULT_KINDS];
static std::once_flag g_fault_env;

static bool parse_fault(const char *spec, long long out[FAULT_KINDS]) {
    for (int k = 0; k < FAULT_KINDS; ++k) out[k] = 0;
    if (!spec) return true;
    std::string s(spec);
    size_t i = 0;
    while (i < s.size()) {
        size_t j = s.find_first_of(",|", i);
        if (j == std::string::npos) j = s.size();
        const std::string item = s.substr(i, j - i);
        i = j + 1;
        if (item.empty()) continue;
        const size_t c = item.find(':');
        if (c == std::string::npos) return false;
        const std::string kind = item.substr(0, c), num = item.substr(c + 1);
        if (num.empty() || num.size() > 12 || num.find_first_not_of("0123456789") != std::string::npos) return false;
        const long long n = std::stoll(num);
        if (n < 1) return false;
        if (kind == "alloc") out[FAULT_ALLOC] = n;
        else if (kind == "launch") out[FAULT_LAUNCH] = n;
        else if (kind == "wait") out[FAULT_WAIT] = n;
        else return false;
    }
    return true;
}

static void fault_env() {
    std::call_once(g_fault_env, [] {
        long long v[FAULT_KINDS];
        if (parse_fault(std::getenv("HTS_FAULT"), v))
            for (int k = 0; k < FAULT_KINDS; ++k)
                if (v[k] > 0) g_fault[k].store(v[k]);
    });
}

bool fault_take(FaultKind k) {
    fault_env();
    long long v = g_fault[k].load();
    while (v > 0) {
        if (g_fault[k].compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}

cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
    if (fault_take(FAULT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

hts_status allow_smem(const void *func, size_t need) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> lim;
    int dev = 0;
    cudaGetDevice(&dev);
    const int optin = smem_optin();
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(func, dev);
    auto it = lim.find(key);
    int L = 0;
    if (it == lim.end()) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return check_launch("cudaFuncGetAttributes");
        L = optin - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, L) != cudaSuccess)
            return check_launch("cudaFuncSetAttribute");
        lim[key] = L;
    } else {
        L = it->second;
    }
    if (need > (size_t)L) return report(HTS_EUNSUPPORTED, "kernel shared memory exceeds the device limit");
    return HTS_OK;
}

int smem_optin() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
        v = 48 * 1024;
    cache[dev] = v;
    return v;
}

// ------------------------------------------------------------ profiling

struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
};
static std::mutex g_pmu;
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

KTimer::KTimer(const char *name, cudaStream_t s) : slot(-1), range(false), stream(s) {
    if (capturing(s)) {  // counted when the graph launches; no profiling events in graphs
        ++g_captured;
        return;
    }
    count_launch();
    nvtxRangePushA(name);
    range = true;
    if (fault_take(FAULT_LAUNCH)) g_launch_fault = true;
    std::lock_guard<std::mutex> lk(g_pmu);
    if (!g_prof) return;
    ProfRec r;
    r.name = name;
    r.e0 = take_event();
    r.e1 = take_event();
    if (!r.e0 || !r.e1) return;
    cudaEventRecord(r.e0, s);
    slot = (int)g_recs.size();
    g_recs.push_back(r);
}

KTimer::~KTimer() {
    if (range) nvtxRangePop();
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    cudaEventRecord(g_recs[slot].e1, stream);
}

static hts_status fail(hts_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

hts_status report(hts_status s, const char *msg) { return fail(s, msg); }

hts_status check_launch(const char *what) {
    if (g_launch_fault) {
        g_launch_fault = false;
        cudaGetLastError();
        return fail(HTS_ECUDA, std::string(what) + ": launch failure (injected by hts_fault_inject)");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HTS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return HTS_OK;
}

static hts_status cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HTS_OK;
    if (e == cudaErrorMemoryAllocation) return fail(HTS_ENOMEM, std::string(what) + ": out of device memory");
    return fail(HTS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Status of a failure the kernels recorded in DevState.error (2: a bounded
// wait gave up; 1: a consistency check failed; 3: a bounds check of the check
// build failed).
hts_status device_status(int err) {
    if (err == 2) return fail(HTS_ETIMEOUT, "a bounded device-side wait gave up; the call's result is invalid");
    if (err == 3) return fail(HTS_EINTERNAL, "a device-side bounds check failed; the call's result is invalid");
    if (err != 0) return fail(HTS_EINTERNAL, "a device-side consistency check failed; the call's result is invalid");
    return HTS_OK;
}

#define HTS_TRY(expr)                       \
    do {                                    \
        hts_status _s = (expr);             \
        if (_s != HTS_OK) return _s;        \
    } while (0)

// ----------------------------------------------------------- workspace

// Buffers grown on demand; aux is the second stream on which the basis and
// the noise floor overlap the grouping.
struct Workspace : Bufs {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t cap_idx = 0, cap_fb = 0, cap_redo = 0, cap_green = 0, cap_hw = 0, cap_chw = 0, cap_cov = 0;
    size_t cap_x = 0, cap_xskip = 0;
    size_t cap_in = 0, cap_out = 0, cap_sref = 0, cap_ra = 0;
    float *io_in = nullptr, *io_out = nullptr;
    float *sref = nullptr;  // learned noise level per reference patch
    float *ra = nullptr;    // enhancement strategy: mean patches and refined ones
};

static std::mutex g_mu;
static std::map<std::pair<int, cudaStream_t>, Workspace *> g_ws;

template <typename T>
static hts_status grow(T *&ptr, size_t &cap, size_t need, const char *what) {
    if (need <= cap && ptr) return HTS_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    const size_t n = need + need / 4 + 64;
    HTS_TRY(cuda_ok(dev_malloc(reinterpret_cast<void **>(&ptr), n * sizeof(T)), what));
    cap = n;
    return HTS_OK;
}

static hts_status get_ws(cudaStream_t s, Workspace **out) {
    int dev = 0;
    HTS_TRY(cuda_ok(cudaGetDevice(&dev), "cudaGetDevice"));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) {
        *out = it->second;
        return HTS_OK;
    }
    Workspace *w = new Workspace();
    w->device = dev;
    w->stream = s;
    hts_status st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&w->st), sizeof(DevState)), "cudaMalloc(state)");
    if (st == HTS_OK) st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&w->b64), 2 * 256 * sizeof(double)), "cudaMalloc");
    if (st == HTS_OK) st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&w->b32), 2 * 256 * sizeof(float)), "cudaMalloc");
    if (st == HTS_OK) st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&w->eig), 4 * 8 * sizeof(double)), "cudaMalloc");
    // The basis chain ends in a few-block eigensolver that the threshold waits
    // for: its stream gets the highest priority so that its blocks are not
    // queued behind the grouping's.
    int prio_lo = 0, prio_hi = 0;
    if (st == HTS_OK) st = cuda_ok(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi), "cudaDeviceGetStreamPriorityRange");
    if (st == HTS_OK)
        st = cuda_ok(cudaStreamCreateWithPriority(&w->aux, cudaStreamNonBlocking, prio_hi), "cudaStreamCreate");
    if (st == HTS_OK) st = cuda_ok(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    if (st == HTS_OK) st = cuda_ok(cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    if (st != HTS_OK) {  // release what was made before the failure
        cudaFree(w->st);
        cudaFree(w->b64);
        cudaFree(w->b32);
        cudaFree(w->eig);
        if (w->ev_fork) cudaEventDestroy(w->ev_fork);
        if (w->aux) cudaStreamDestroy(w->aux);
        delete w;
        return st;
    }
    g_ws[key] = w;
    *out = w;
    return HTS_OK;
}

static hts_status ensure(Workspace *w, const Geom &g) {
    const size_t nref = (size_t)g.nref, hw = (size_t)g.H * g.W;
    HTS_TRY(grow(w->idx, w->cap_idx, nref * g.K, "cudaMalloc(idx)"));
    HTS_TRY(grow(w->fb, w->cap_fb, nref, "cudaMalloc(fallback)"));
    HTS_TRY(grow(w->redo, w->cap_redo, nref, "cudaMalloc(redo)"));
    HTS_TRY(grow(w->xlist, w->cap_x, nref * XLIST_PER_REF, "cudaMalloc(xlist)"));
    HTS_TRY(grow(w->xskip, w->cap_xskip, nref, "cudaMalloc(xskip)"));
    HTS_TRY(grow(w->green, w->cap_green, nref, "cudaMalloc(green)"));
    HTS_TRY(grow(w->acc, w->cap_chw, hw * g.C, "cudaMalloc(acc)"));
    HTS_TRY(grow(w->wcount, w->cap_hw, hw, "cudaMalloc(weights)"));
    HTS_TRY(grow(w->cov, w->cap_cov, cov_partial_count(g), "cudaMalloc(cov)"));
    return HTS_OK;
}

// ----------------------------------------------------------- validation

hts_status validate(int H, int W, int C, const hts_params *p, Geom *g) {
    if (!p) return fail(HTS_EINVAL, "params is NULL");
    if (p->ps != PS) return fail(HTS_EUNSUPPORTED, "only ps = 8 is built");
    if (C != 1 && C != 3) return fail(HTS_EINVAL, "C must be 1 or 3");
    if (H < PS || W < PS) return fail(HTS_EINVAL, "image smaller than a patch");
    if ((long long)H * W * C > 0x7fffffffll) return fail(HTS_EINVAL, "image too large for 32-bit indices");
    if (p->K != 2 && p->K != 4 && p->K != 8 && p->K != 16 && p->K != 32)
        return fail(HTS_EINVAL, "K must be a power of two in [2, 32]");
    if (p->win < 3 || (p->win % 2) == 0) return fail(HTS_EINVAL, "win must be odd and >= 3");
    if (p->win > MAX_WIN) return fail(HTS_EUNSUPPORTED, "win > 63 is not built");
    if (p->step < 1 || p->step > PS) return fail(HTS_EINVAL, "step must be in [1, ps]");
    if (!(p->gamma_gcp > 0) || !std::isfinite(p->gamma_gcp)) return fail(HTS_EINVAL, "gamma_gcp must be > 0");
    if (!(p->beta > 0) || !std::isfinite(p->beta)) return fail(HTS_EINVAL, "beta must be > 0");
    if (!(p->tau_mult >= 0) || !std::isfinite(p->tau_mult)) return fail(HTS_EINVAL, "tau_mult must be >= 0");
    if (!std::isfinite(p->gamma_rank)) return fail(HTS_EINVAL, "gamma_rank must be finite");
    if (p->precision < 0 || p->precision > 2) return fail(HTS_EINVAL, "precision must be 0, 1 or 2");
    const int R = (p->win - 1) / 2;
    const long long cap = (long long)std::min(R + 1, H - PS + 1) * std::min(R + 1, W - PS + 1);
    if (cap < p->K) return fail(HTS_EINVAL, "search window holds fewer than K patch positions");
    g->H = H;
    g->W = W;
    g->C = C;
    g->step = p->step;
    g->R = R;
    g->K = p->K;
    g->ny = grid_count(H, p->step);
    g->nx = grid_count(W, p->step);
    g->nref = g->ny * g->nx;
    return HTS_OK;
}

// ------------------------------------------------------------- basis

// Doubles in a basis of ns stored slices: [ns][2 (U, V)][8][8][2 (re, im)].
static inline size_t basis_doubles(int ns) { return (size_t)ns * 2 * 64 * 2; }
// Doubles of one 8x8 complex matrix.
constexpr int MAT_DOUBLES = 64 * 2;

static hts_status alloc_basis(int C, hts_basis **out) {
    int dev = 0;
    HTS_TRY(cuda_ok(cudaGetDevice(&dev), "cudaGetDevice"));
    hts_basis *b = new hts_basis();
    b->C = C;
    b->ns = C / 2 + 1;
    b->has_eig = 0;
    b->device = dev;
    b->b64 = nullptr;
    b->b32 = nullptr;
    b->eig = nullptr;
    hts_status st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&b->b64), basis_doubles(b->ns) * sizeof(double)), "cudaMalloc(basis)");
    if (st == HTS_OK) st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&b->b32), basis_doubles(b->ns) * sizeof(float)), "cudaMalloc(basis)");
    if (st == HTS_OK) st = cuda_ok(dev_malloc(reinterpret_cast<void **>(&b->eig), b->ns * 16 * sizeof(double)), "cudaMalloc(basis)");
    if (st != HTS_OK) {
        cudaFree(b->b64);
        cudaFree(b->b32);
        cudaFree(b->eig);
        delete b;
        return st;
    }
    *out = b;
    return HTS_OK;
}

static void free_basis(hts_basis *b) {
    if (!b) return;
    cudaFree(b->b64);
    cudaFree(b->b32);
    cudaFree(b->eig);
    delete b;
}

// ------------------------------------------------------------- pipeline

// Basis pointers used by one call: caller's or freshly estimated.
struct BasisRef {
    const double *b64;
    const float *b32;
    const double *eig;
};

static hts_status prepare(const float *img, const Geom &g, const hts_params &p, const hts_basis *basis,
                          bool need_sigma, Workspace *w, cudaStream_t s, BasisRef *br) {
    HTS_TRY(cuda_ok(cudaMemsetAsync(w->st, 0, sizeof(DevState), s), "cudaMemsetAsync(state)"));
    const bool est = (basis == nullptr) || (need_sigma && !basis->has_eig);
    if (est) HTS_TRY(launch_basis(img, g, w->cov, w->b64, w->b32, w->eig, s));
    br->b64 = basis ? basis->b64 : w->b64;
    br->b32 = basis ? basis->b32 : w->b32;
    br->eig = (basis && basis->has_eig) ? basis->eig : w->eig;
    return HTS_OK;
}

hts_status check_basis(const hts_basis *basis, int C) {
    if (!basis) return HTS_OK;
    if (basis->C != C) return fail(HTS_EINVAL, "basis was built for another channel count");
    int dev = 0;
    HTS_TRY(cuda_ok(cudaGetDevice(&dev), "cudaGetDevice"));
    if (basis->device != dev) return fail(HTS_EINVAL, "basis lives on another device");
    return HTS_OK;
}

// The global basis (k_cov, k_cov_sum, k_jacobi) and the noise floor depend
// only on the reference patches, the grouping and the rank vote only on the
// image: the first chain runs on the workspace's second stream while the
// second runs on the caller's stream; the threshold waits for both.
hts_status launch_grouping(const float *img, const Geom &g, const hts_params &p, int32_t *idx, uint8_t *green,
                           int32_t *fb, DevState *st, cudaStream_t s, bool flags_done) {
    if (p.precision != 1) return launch_match(img, g, p.gamma_gcp, idx, green, fb, st, s);
    if (g.C == 3 && !flags_done) HTS_TRY(launch_gcp_flags(img, g, p.gamma_gcp, green, s));
    return launch_match_tc(img, g, p.gamma_gcp, idx, green, fb, st, s);
}

hts_status denoise_run(const float *noisy, float *out, const Geom &g, float sigma, const hts_basis *basis,
                       const hts_params &p, const Bufs &b, cudaStream_t s, float *sigma_ref, double fallback_factor,
                       hts_fcn *fcn, float *ra_buf, cudaEvent_t map_ready) {
    const Bufs *w = &b;
    const size_t hw = (size_t)g.H * g.W;
    HTS_TRY(cuda_ok(cudaMemsetAsync(w->st, 0, sizeof(DevState), s), "cudaMemsetAsync(state)"));
    HTS_TRY(cuda_ok(cudaMemsetAsync(w->acc, 0, hw * g.C * sizeof(long long), s), "cudaMemsetAsync(acc)"));
    HTS_TRY(cuda_ok(cudaMemsetAsync(w->wcount, 0, hw * sizeof(int), s), "cudaMemsetAsync(weights)"));
    // a noise map without a check needs no estimate; a checked map is compared with the estimate
    const bool need_sigma = sigma < 0 && (sigma_ref == nullptr || fallback_factor > 0);
    const bool est = (basis == nullptr) || (need_sigma && !basis->has_eig);
    const double *b64 = basis ? basis->b64 : w->b64;
    const float *b32 = basis ? basis->b32 : w->b32;
    const double *eig = (basis && basis->has_eig) ? basis->eig : w->eig;
    const bool fork = est || need_sigma;
    // the precision form's Eq. 9 flags go first: the basis chain is then launched beside the tensor-core
    // matcher, whose blocks (one per SM) would otherwise wait behind the covariance's
    const bool flags_first = p.precision == 1 && g.C == 3;
    if (flags_first) HTS_TRY(launch_gcp_flags(noisy, g, p.gamma_gcp, w->green, s));
    if (fork) {
        HTS_TRY(cuda_ok(cudaEventRecord(w->ev_fork, s), "cudaEventRecord"));
        HTS_TRY(cuda_ok(cudaStreamWaitEvent(w->aux, w->ev_fork, 0), "cudaStreamWaitEvent"));
        if (est) HTS_TRY(launch_basis(noisy, g, w->cov, w->b64, w->b32, w->eig, w->aux));
        if (need_sigma) HTS_TRY(launch_sigma_floor(g, p, eig, w->st, w->aux));
        HTS_TRY(cuda_ok(cudaEventRecord(w->ev_join, w->aux), "cudaEventRecord"));
    }
    HTS_TRY(launch_grouping(noisy, g, p, w->idx, w->green, w->fb, w->st, s, flags_first));
    if (need_sigma && p.adjust_rank) HTS_TRY(launch_sigma_vote(noisy, g, p, w->idx, w->redo, w->st, s));
    if (fork) HTS_TRY(cuda_ok(cudaStreamWaitEvent(s, w->ev_join, 0), "cudaStreamWaitEvent"));
    if (need_sigma) HTS_TRY(launch_sigma_final(g, p, w->st, s));
    else HTS_TRY(launch_set_sigma(sigma > 0 ? (double)sigma : 0.0, g, p, w->st, s));
    if (map_ready) HTS_TRY(cuda_ok(cudaStreamWaitEvent(s, map_ready, 0), "cudaStreamWaitEvent"));
    if (sigma_ref && fallback_factor > 0) HTS_TRY(launch_learned_check(sigma_ref, g.nref, fallback_factor, w->st, s));
    float *mean_est = nullptr;
    if (fcn) {  // enhancement strategy: refined mean patch of every group (Eq. 24-25)
        float *means = ra_buf, *refined = ra_buf + (size_t)g.nref * g.C * 64;
        HTS_TRY(launch_group_means(noisy, g, w->idx, means, s));
        HTS_TRY(fcn_refine_state(fcn, means, g.nref, w->st, b32, refined, s));
        mean_est = refined;
    }
    return launch_filter(noisy, g, w->idx, b64, b32, w->acc, w->wcount, w->redo, w->xlist, w->xskip, w->st, out,
                         p.precision == 0 ? 1 : 0, sigma_ref, fallback_factor > 0 ? 1 : 0, tau_scale(g, p), s,
                         mean_est);
}

static hts_status denoise_impl(const float *noisy, float *out, const Geom &g, float sigma, const hts_basis *basis,
                               const hts_params &p, Workspace *w, cudaStream_t s) {
    HTS_TRY(ensure(w, g));
    return denoise_run(noisy, out, g, sigma, basis, p, *w, s);
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t bufs_bytes(const Geom &g) {
    const size_t nref = (size_t)g.nref, hw = (size_t)g.H * g.W;
    return align256(sizeof(DevState)) + align256(2 * 256 * sizeof(double)) + align256(2 * 256 * sizeof(float)) +
           align256(32 * sizeof(double)) + align256(nref * g.K * sizeof(int32_t)) + align256(nref) +
           2 * align256(nref * sizeof(int32_t)) + align256(nref * XLIST_PER_REF * sizeof(int4)) + align256(nref) +
           align256(hw * g.C * sizeof(long long)) + align256(hw * sizeof(int)) +
           align256(cov_partial_count(g) * sizeof(double)) + align256(nref * sizeof(float));
}

void bufs_carve(const Geom &g, unsigned char *base, Bufs *b) {
    const size_t nref = (size_t)g.nref, hw = (size_t)g.H * g.W;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + o;
        o += align256(bytes);
        return p;
    };
    b->st = reinterpret_cast<DevState *>(take(sizeof(DevState)));
    b->b64 = reinterpret_cast<double *>(take(2 * 256 * sizeof(double)));
    b->b32 = reinterpret_cast<float *>(take(2 * 256 * sizeof(float)));
    b->eig = reinterpret_cast<double *>(take(32 * sizeof(double)));
    b->idx = reinterpret_cast<int32_t *>(take(nref * g.K * sizeof(int32_t)));
    b->green = reinterpret_cast<uint8_t *>(take(nref));
    b->fb = reinterpret_cast<int32_t *>(take(nref * sizeof(int32_t)));
    b->redo = reinterpret_cast<int32_t *>(take(nref * sizeof(int32_t)));
    b->xlist = reinterpret_cast<int4 *>(take(nref * XLIST_PER_REF * sizeof(int4)));
    b->xskip = reinterpret_cast<uint8_t *>(take(nref));
    b->acc = reinterpret_cast<long long *>(take(hw * g.C * sizeof(long long)));
    b->wcount = reinterpret_cast<int *>(take(hw * sizeof(int)));
    b->cov = reinterpret_cast<double *>(take(cov_partial_count(g) * sizeof(double)));
    b->sref = reinterpret_cast<float *>(take(nref * sizeof(float)));
}

}  // namespace hts

using namespace hts;

extern "C" {

hts_status hts_params_default(hts_params *p) {
    if (!p) return fail(HTS_EINVAL, "params is NULL");
    p->ps = 8;
    p->K = 16;
    p->win = 21;
    p->step = 4;
    p->gamma_gcp = 1.2;
    p->beta = 1.2;
    p->gamma_rank = 0.0;
    p->tau_mult = 1.0;
    p->adjust_rank = 1;
    p->mp_correct = 1;
    p->precision = 0;
    return HTS_OK;
}

int hts_num_refs(int H, int W, const hts_params *p) {
    if (!p || p->ps != PS || H < PS || W < PS || p->step < 1 || p->step > PS) return 0;
    return grid_count(H, p->step) * grid_count(W, p->step);
}

hts_status hts_estimate_basis(const float *img, int H, int W, int C, const hts_params *p, hts_basis **out,
                              void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!img || !out) return fail(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    hts_basis *b;
    HTS_TRY(alloc_basis(C, &b));
    hts_status st = launch_basis(img, g, w->cov, b->b64, b->b32, b->eig, s);
    if (st == HTS_OK) st = cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (st != HTS_OK) {
        free_basis(b);
        return st;
    }
    b->has_eig = 1;
    *out = b;
    return HTS_OK;
}

hts_status hts_basis_create(const double *host_basis, const double *host_eigvals, int C, hts_basis **out) {
    if (!host_basis || !out) return fail(HTS_EINVAL, "NULL pointer");
    if (C != 1 && C != 3) return fail(HTS_EINVAL, "C must be 1 or 3");
    const int ns = C / 2 + 1;
    for (int j = 0; j < ns; ++j)
        for (int m = 0; m < 2; ++m) {
            const double *M = host_basis + (size_t)(j * 2 + m) * MAT_DOUBLES;
            for (int e = 0; e < MAT_DOUBLES; ++e)
                if (!std::isfinite(M[e])) return fail(HTS_EINVAL, "basis holds a non-finite value");
            if (j == 0)
                for (int e = 0; e < 64; ++e)
                    if (M[2 * e + 1] != 0.0) return fail(HTS_EINVAL, "slice 0 of the basis must be real");
            for (int i1 = 0; i1 < 8; ++i1)
                for (int i2 = 0; i2 < 8; ++i2) {
                    double re = 0, im = 0;  // (M^H M)[i1][i2]
                    for (int a = 0; a < 8; ++a) {
                        const double xr = M[(a * 8 + i1) * 2], xi = M[(a * 8 + i1) * 2 + 1];
                        const double yr = M[(a * 8 + i2) * 2], yi = M[(a * 8 + i2) * 2 + 1];
                        re += xr * yr + xi * yi;
                        im += xr * yi - xi * yr;
                    }
                    const double want = (i1 == i2) ? 1.0 : 0.0;
                    if (std::fabs(re - want) > 1e-6 || std::fabs(im) > 1e-6)
                        return fail(HTS_EINVAL, "basis matrices must be unitary");
                }
        }
    hts_basis *b;
    HTS_TRY(alloc_basis(C, &b));
    float f[4 * MAT_DOUBLES];
    const size_t nd = basis_doubles(ns);
    for (size_t e = 0; e < nd; ++e) f[e] = (float)host_basis[e];
    hts_status st = cuda_ok(cudaMemcpy(b->b64, host_basis, nd * sizeof(double), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (st == HTS_OK) st = cuda_ok(cudaMemcpy(b->b32, f, nd * sizeof(float), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (st == HTS_OK && host_eigvals) {
        st = cuda_ok(cudaMemcpy(b->eig, host_eigvals, ns * 16 * sizeof(double), cudaMemcpyHostToDevice), "cudaMemcpy");
        b->has_eig = 1;
    }
    if (st != HTS_OK) {
        free_basis(b);
        return st;
    }
    *out = b;
    return HTS_OK;
}

hts_status hts_basis_read(const hts_basis *b, double *host_basis, double *host_eigvals, int *C_out) {
    if (!b) return fail(HTS_EINVAL, "basis is NULL");
    if (C_out) *C_out = b->C;
    if (host_basis) HTS_TRY(cuda_ok(cudaMemcpy(host_basis, b->b64, basis_doubles(b->ns) * sizeof(double), cudaMemcpyDeviceToHost), "cudaMemcpy"));
    if (host_eigvals) {
        if (!b->has_eig) return fail(HTS_EINVAL, "basis has no eigenvalues");
        HTS_TRY(cuda_ok(cudaMemcpy(host_eigvals, b->eig, b->ns * 16 * sizeof(double), cudaMemcpyDeviceToHost), "cudaMemcpy"));
    }
    return HTS_OK;
}

hts_status hts_basis_free(hts_basis *b) {
    free_basis(b);
    return HTS_OK;
}

hts_status hts_basis_save(const hts_basis *b, const char *path) {
    if (!b || !path) return fail(HTS_EINVAL, "NULL pointer");
    double hb[4 * MAT_DOUBLES], he[32];
    HTS_TRY(hts_basis_read(b, hb, nullptr, nullptr));
    if (b->has_eig) HTS_TRY(hts_basis_read(b, nullptr, he, nullptr));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(HTS_EINVAL, std::string("cannot open ") + path);
    const char magic[8] = {'H', 'T', 'S', 'B', '1', 0, 0, 0};
    const int hdr[2] = {b->C, b->has_eig};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 2, f) == 2 &&
              std::fwrite(hb, sizeof(double), basis_doubles(b->ns), f) == basis_doubles(b->ns);
    if (ok && b->has_eig) ok = std::fwrite(he, sizeof(double), b->ns * 16, f) == (size_t)b->ns * 16;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? HTS_OK : fail(HTS_EINVAL, "write failed");
}

hts_status hts_basis_load(const char *path, hts_basis **out) {
    if (!path || !out) return fail(HTS_EINVAL, "NULL pointer");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(HTS_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int hdr[2];
    double hb[4 * MAT_DOUBLES], he[32];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "HTSB1", 5) == 0 &&
              std::fread(hdr, sizeof(int), 2, f) == 2 && (hdr[0] == 1 || hdr[0] == 3);
    const int ns = ok ? hdr[0] / 2 + 1 : 0;
    if (ok) ok = std::fread(hb, sizeof(double), basis_doubles(ns), f) == basis_doubles(ns);
    if (ok && hdr[1]) ok = std::fread(he, sizeof(double), ns * 16, f) == (size_t)ns * 16;
    std::fclose(f);
    if (!ok) return fail(HTS_EINVAL, "not a basis file");
    return hts_basis_create(hb, hdr[1] ? he : nullptr, hdr[0], out);
}

hts_status hts_match(const float *img, int H, int W, int C, const hts_params *p, int32_t *idx_out,
                     uint8_t *green_out, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!img || !idx_out) return fail(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    HTS_TRY(cuda_ok(cudaMemsetAsync(w->st, 0, sizeof(DevState), s), "cudaMemsetAsync(state)"));
    return launch_grouping(img, g, *p, idx_out, green_out, w->fb, w->st, s);
}

hts_status hts_estimate_sigma(const float *img, int H, int W, int C, const hts_basis *basis, const hts_params *p,
                              double *sigma_out, hts_sigma_info *info, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!img || !sigma_out) return fail(HTS_EINVAL, "NULL pointer");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    BasisRef br;
    HTS_TRY(prepare(img, g, *p, basis, true, w, s, &br));
    if (p->adjust_rank) HTS_TRY(launch_grouping(img, g, *p, w->idx, w->green, w->fb, w->st, s));
    HTS_TRY(launch_sigma(img, g, *p, br.eig, w->idx, w->redo, w->st, s));
    DevState hs;
    HTS_TRY(cuda_ok(cudaMemcpyAsync(&hs, w->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync"));
    HTS_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    *sigma_out = hs.sigma_hat;
    if (info) {
        info->sigma_hat = hs.sigma_hat;
        info->sigma_est = hs.sigma_est;
        info->votes = hs.votes;
        info->nref = g.nref;
        info->adjusted = hs.adjusted;
        info->uncertain = hs.vote_uncertain;
    }
    return device_status(hs.error);
}

hts_status hts_denoise(const float *noisy, float *out, int H, int W, int C, float sigma, const hts_basis *basis,
                       const hts_params *p, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy || !out) return fail(HTS_EINVAL, "NULL pointer");
    if (noisy == out) return fail(HTS_EINVAL, "out may not alias noisy");
    if (std::isnan(sigma) || std::isinf(sigma)) return fail(HTS_EINVAL, "sigma must be finite");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    return denoise_impl(noisy, out, g, sigma, basis, *p, w, s);
}

hts_status hts_denoise_host(const float *noisy_host, float *out_host, int H, int W, int C, float sigma,
                            const hts_basis *basis, const hts_params *p, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy_host || !out_host) return fail(HTS_EINVAL, "NULL pointer");
    if (std::isnan(sigma) || std::isinf(sigma)) return fail(HTS_EINVAL, "sigma must be finite");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    const size_t n = (size_t)H * W * C;
    HTS_TRY(grow(w->io_in, w->cap_in, n, "cudaMalloc(io)"));
    HTS_TRY(grow(w->io_out, w->cap_out, n, "cudaMalloc(io)"));
    HTS_TRY(cuda_ok(cudaMemcpyAsync(w->io_in, noisy_host, n * sizeof(float), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(H2D)"));
    HTS_TRY(denoise_impl(w->io_in, w->io_out, g, sigma, basis, *p, w, s));
    HTS_TRY(cuda_ok(cudaMemcpyAsync(out_host, w->io_out, n * sizeof(float), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)"));
    int err = 0;
    HTS_TRY(cuda_ok(cudaMemcpyAsync(&err, &w->st->error, sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)"));
    HTS_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    return device_status(err);
}

hts_status hts_denoise_sigma_map(const float *noisy, float *out, int H, int W, int C, const float *sigma_ref,
                                 const hts_basis *basis, const hts_params *p, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy || !out || !sigma_ref) return fail(HTS_EINVAL, "NULL pointer");
    if (noisy == out) return fail(HTS_EINVAL, "out may not alias noisy");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    return denoise_run(noisy, out, g, -1.f, basis, *p, *w, s, const_cast<float *>(sigma_ref), 0.0);
}

hts_status hts_denoise_learned(const float *noisy, float *out, int H, int W, int C, hts_cnn *net,
                               const hts_basis *basis, const hts_params *p, double fallback_factor, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy || !out || !net) return fail(HTS_EINVAL, "NULL pointer");
    if (noisy == out) return fail(HTS_EINVAL, "out may not alias noisy");
    if (!(fallback_factor > 1.0) || !std::isfinite(fallback_factor))
        return fail(HTS_EINVAL, "fallback_factor must be > 1");
    if (hts_cnn_channels(net) != C) return fail(HTS_EINVAL, "network built for another channel count");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    HTS_TRY(grow(w->sref, w->cap_sref, (size_t)g.nref, "cudaMalloc(sigma map)"));
    HTS_TRY(cnn_sigma_refs(net, noisy, g, w->sref, s));
    return denoise_run(noisy, out, g, -1.f, basis, *p, *w, s, w->sref, fallback_factor);
}

hts_status hts_denoise_learned_host(const float *noisy_host, float *out_host, int H, int W, int C, hts_cnn *net,
                                    const hts_basis *basis, const hts_params *p, double fallback_factor,
                                    void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy_host || !out_host || !net) return fail(HTS_EINVAL, "NULL pointer");
    if (!(fallback_factor > 1.0) || !std::isfinite(fallback_factor))
        return fail(HTS_EINVAL, "fallback_factor must be > 1");
    if (hts_cnn_channels(net) != C) return fail(HTS_EINVAL, "network built for another channel count");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    const size_t n = (size_t)H * W * C;
    HTS_TRY(grow(w->io_in, w->cap_in, n, "cudaMalloc(io)"));
    HTS_TRY(grow(w->io_out, w->cap_out, n, "cudaMalloc(io)"));
    HTS_TRY(cuda_ok(cudaMemcpyAsync(w->io_in, noisy_host, n * sizeof(float), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(H2D)"));
    HTS_TRY(hts_denoise_learned(w->io_in, w->io_out, H, W, C, net, basis, p, fallback_factor, stream));
    HTS_TRY(cuda_ok(cudaMemcpyAsync(out_host, w->io_out, n * sizeof(float), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)"));
    int err = 0;
    HTS_TRY(cuda_ok(cudaMemcpyAsync(&err, &w->st->error, sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)"));
    HTS_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    return device_status(err);
}

hts_status hts_denoise_ra(const float *noisy, float *out, int H, int W, int C, float sigma, hts_fcn *fcn,
                          const hts_basis *basis, const hts_params *p, void *stream) {
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    if (!noisy || !out || !fcn) return fail(HTS_EINVAL, "NULL pointer");
    if (noisy == out) return fail(HTS_EINVAL, "out may not alias noisy");
    if (!std::isfinite(sigma)) return fail(HTS_EINVAL, "sigma must be finite");
    if (p->precision == 0) return fail(HTS_EUNSUPPORTED, "the enhancement strategy needs precision 1 or 2");
    if (hts_fcn_channels(fcn) != C) return fail(HTS_EINVAL, "network built for another channel count");
    if (hts_fcn_group_size(fcn) != p->K) return fail(HTS_EINVAL, "network built for another group size");
    HTS_TRY(check_basis(basis, C));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    HTS_TRY(ensure(w, g));
    HTS_TRY(grow(w->ra, w->cap_ra, (size_t)2 * g.nref * C * 64, "cudaMalloc(enhancement)"));
    return denoise_run(noisy, out, g, sigma, basis, *p, *w, s, nullptr, 0.0, fcn, w->ra);
}

hts_status hts_last_stats(hts_stats *out, void *stream) {
    if (!out) return fail(HTS_EINVAL, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace *w;
    HTS_TRY(get_ws(s, &w));
    DevState hs;
    HTS_TRY(cuda_ok(cudaMemcpyAsync(&hs, w->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync"));
    HTS_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    out->nref = hs.nref;
    out->match_reranked = hs.match_reranked;
    out->match_fallback = hs.match_fallback;
    out->filter_redo = hs.filter_redo;
    out->filter_exact = hs.filter_exact;
    out->vote_uncertain = hs.vote_uncertain;
    out->sigma = hs.sigma_hat;
    out->tau = hs.tau;
    out->filter_fixed = hs.filter_fixed;
    out->learned = hs.learned;
    out->learned_ratio = hs.learned_ratio;
    out->device_error = hs.error;
    return device_status(hs.error);
}

hts_status hts_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (auto &r : g_recs) {
        g_pool.push_back(r.e0);
        g_pool.push_back(r.e1);
    }
    g_recs.clear();
    g_prof = true;
    return HTS_OK;
}

hts_status hts_profile_end(hts_kernel_time *out, int max, int *n_out) {
    std::lock_guard<std::mutex> lk(g_pmu);
    g_prof = false;
    int n = 0;
    hts_status st = HTS_OK;
    for (auto &r : g_recs) {
        if (cudaEventSynchronize(r.e1) != cudaSuccess) {
            st = fail(HTS_ECUDA, "cudaEventSynchronize");
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) {
            st = fail(HTS_ECUDA, "cudaEventElapsedTime");
            break;
        }
        int k = 0;
        while (k < n && std::strcmp(out[k].name, r.name) != 0) ++k;
        if (k == n) {
            if (n >= max) continue;
            std::memset(out[n].name, 0, sizeof(out[n].name));
            std::strncpy(out[n].name, r.name, sizeof(out[n].name) - 1);
            out[n].total_ms = 0.0;
            out[n].launches = 0;
            ++n;
        }
        out[k].total_ms += ms;
        out[k].launches += 1;
    }
    if (n_out) *n_out = n;
    return st;
}

hts_status hts_fault_inject(const char *spec) {
    fault_env();  // the environment's setting, if any, is read first and then replaced
    long long v[FAULT_KINDS];
    if (!parse_fault(spec, v)) return fail(HTS_EINVAL, "fault spec: expected kind:N[,kind:N] with kind alloc, launch or wait, N >= 1");
    for (int k = 0; k < FAULT_KINDS; ++k) g_fault[k].store(v[k]);
    return HTS_OK;
}

const char *hts_last_error(void) { return g_err.c_str(); }

uint64_t hts_launch_count(void) { return g_launches.load(); }

const char *hts_version(void) { return "hts 0.1 (sm_103a)"; }

hts_status hts_shutdown(void) {
    batch_shutdown();
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_ws) {
        Workspace *w = kv.second;
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(w->device);
        cudaFree(w->idx);
        cudaFree(w->green);
        cudaFree(w->fb);
        cudaFree(w->redo);
        cudaFree(w->xlist);
        cudaFree(w->xskip);
        cudaFree(w->acc);
        cudaFree(w->wcount);
        cudaFree(w->cov);
        cudaFree(w->b64);
        cudaFree(w->b32);
        cudaFree(w->eig);
        cudaFree(w->st);
        cudaFree(w->io_in);
        cudaFree(w->io_out);
        cudaFree(w->sref);
        cudaFree(w->ra);
        if (w->ev_fork) cudaEventDestroy(w->ev_fork);
        if (w->ev_join) cudaEventDestroy(w->ev_join);
        if (w->aux) cudaStreamDestroy(w->aux);
        cudaSetDevice(prev);
        delete w;
    }
    g_ws.clear();
    return HTS_OK;
}

}  // extern "C"
