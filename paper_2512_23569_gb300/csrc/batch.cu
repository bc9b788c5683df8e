// Batched Haar-tSVD (hts_denoise_batch): many independent images of mixed
// sizes and channel counts denoised by ONE CUDA-graph launch.
//
// The full pipeline of every image (basis, grouping, noise level, filter) is
// captured once per batch signature (sizes, channel counts, which noise
// levels are estimated, parameters) into a graph whose branches run on
// several streams ("lanes") at once, each image with its own slot of one
// device arena, so that the graph neither allocates nor synchronises.  A
// later call with the same signature but other image pointers or noise levels
// re-captures and updates the instantiated graph in place.
//
// An autotuner runs on the first call of a signature: for every image
// geometry not tuned before it times each valid tile shape of the filter
// (k_filter_tile) on that geometry's first image, and for the batch it times
// the graph built for 1, 2, 4 and 8 lanes (images are dealt to lanes largest
// first, each to the least-loaded lane).  Every choice gives bit-identical
// output (the aggregation is exact integer arithmetic and every group is
// computed independently), so tuning changes only the speed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "cnn_internal.h"
#include "hts_internal.h"

namespace hts {
namespace {

#define HTS_TRY(expr)                \
    do {                             \
        hts_status _s = (expr);      \
        if (_s != HTS_OK) return _s; \
    } while (0)

hts_status cu(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HTS_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return report(e == cudaErrorMemoryAllocation ? HTS_ENOMEM : HTS_ECUDA, m.c_str());
}

constexpr int MAX_LANES = 8;

struct Sig {
    int device = 0;
    std::vector<int> dims;          // per image: H, W, C, estimated sigma (0/1), caller's sigma map (0/1)
    std::vector<unsigned char> par;  // per image: the bytes of its parameters
    const hts_cnn *net = nullptr;    // learned form: the network, its readout window, the fallback factor
    int window = 0;
    double factor = 0.0;
    bool operator<(const Sig &o) const {
        if (device != o.device) return device < o.device;
        if (dims != o.dims) return dims < o.dims;
        if (net != o.net) return net < o.net;
        if (window != o.window) return window < o.window;
        if (factor != o.factor) return factor < o.factor;
        return par < o.par;
    }
};

struct Plan {
    Sig sig;
    std::vector<Geom> geo;
    std::vector<hts_params> par;  // per image
    std::vector<double> work;  // relative cost per image, for the lane assignment
    unsigned char *arena = nullptr;
    std::vector<Bufs> bufs;
    cudaStream_t origin = nullptr;
    cudaStream_t lanes[MAX_LANES] = {};
    cudaStream_t auxs[MAX_LANES] = {};
    cudaEvent_t ev_lane[MAX_LANES] = {};
    std::vector<cudaEvent_t> ev_img;  // fork and join of every image
    cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    // learned form: the networks' forwards run one after another on their own stream, into buffers of
    // the plan sized for the largest image; image i's filter waits for ev_map[i]
    // phased form (every image on the tensor-core filter): the matcher and the filter run as one launch
    // per group of images (matcher: same K; filter: same C and K) over a job table in device memory
    bool phased = false;
    struct Group {
        int K = 0, C = 0, first = 0, njobs = 0, nitems = 0, start_off = 0, queue_off = 0;
    };
    std::vector<Group> mgroups, fgroups;
    std::vector<int> mjob_of, fjob_of;            // image -> row of the job tables (-1: none)
    std::vector<unsigned char> mjob_h, fjob_h;    // the job tables (host copies, uploaded at each capture)
    std::vector<int> starts_h;                    // every group's item / tile prefix sums, then queue counters
    unsigned char *mjob_d = nullptr, *fjob_d = nullptr;
    int *starts_d = nullptr;
    cudaEvent_t ev_phase[4] = {};
    int fshape = -1;         // autotuned: the filter's tile shape for every image (-1: each geometry's model)
    bool largest_first = false;  // autotuned: the matcher's queue takes the largest images first
    hts_cnn *net = nullptr;
    cudaStream_t cnn_stream = nullptr;
    cudaEvent_t ev_cnn = nullptr;
    std::vector<cudaEvent_t> ev_map;
    __half *h16[2] = {};
    float *cmap = nullptr, *crows = nullptr;
    int nlanes = 0;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    std::vector<hts_image> bound;  // pointers and noise levels the graph was captured with
    int captures = 0, updates = 0;
    unsigned long long last_use = 0;
};

std::mutex g_bmu;
std::map<Sig, Plan *> g_plans;
std::map<std::pair<int, cudaStream_t>, Plan *> g_last;  // most recent plan per (device, caller stream)
unsigned long long g_tick = 0;
constexpr size_t MAX_PLANS = 4;

void destroy_plan(Plan *P) {
    if (!P) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(P->sig.device);
    if (P->origin) cudaStreamSynchronize(P->origin);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    for (int l = 0; l < MAX_LANES; ++l) {
        if (P->lanes[l]) cudaStreamDestroy(P->lanes[l]);
        if (P->auxs[l]) cudaStreamDestroy(P->auxs[l]);
        if (P->ev_lane[l]) cudaEventDestroy(P->ev_lane[l]);
    }
    for (cudaEvent_t e : P->ev_img) cudaEventDestroy(e);
    for (cudaEvent_t e : P->ev_map) cudaEventDestroy(e);
    for (cudaEvent_t e : {P->ev_start, P->ev_in, P->ev_out, P->ev_t0, P->ev_t1, P->ev_cnn})
        if (e) cudaEventDestroy(e);
    if (P->origin) cudaStreamDestroy(P->origin);
    if (P->cnn_stream) cudaStreamDestroy(P->cnn_stream);
    cudaFree(P->arena);
    cudaFree(P->h16[0]);
    cudaFree(P->h16[1]);
    cudaFree(P->cmap);
    cudaFree(P->crows);
    cudaFree(P->mjob_d);
    cudaFree(P->fjob_d);
    cudaFree(P->starts_d);
    for (cudaEvent_t e : P->ev_phase)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete P;
}

hts_status create_plan(const Sig &sig, const std::vector<Geom> &geo, const std::vector<hts_params> &par,
                       hts_cnn *net, Plan **out) {
    Plan *P = new Plan();
    P->sig = sig;
    P->geo = geo;
    P->par = par;
    P->net = net;
    const int n = (int)geo.size();
    std::vector<size_t> off(n + 1, 0);
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + bufs_bytes(geo[i]);
    hts_status st = cu(dev_malloc(reinterpret_cast<void **>(&P->arena), std::max<size_t>(off[n], 256)),
                       "cudaMalloc(batch arena)");
    int lo = 0, hi = 0;
    if (st == HTS_OK) st = cu(cudaDeviceGetStreamPriorityRange(&lo, &hi), "cudaDeviceGetStreamPriorityRange");
    if (st == HTS_OK) st = cu(cudaStreamCreateWithFlags(&P->origin, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int l = 0; l < MAX_LANES && st == HTS_OK; ++l) {
        st = cu(cudaStreamCreateWithFlags(&P->lanes[l], cudaStreamNonBlocking), "cudaStreamCreate");
        if (st == HTS_OK)
            st = cu(cudaStreamCreateWithPriority(&P->auxs[l], cudaStreamNonBlocking, hi), "cudaStreamCreate");
        if (st == HTS_OK)
            st = cu(cudaEventCreateWithFlags(&P->ev_lane[l], cudaEventDisableTiming), "cudaEventCreate");
    }
    for (int i = 0; i < 2 * n && st == HTS_OK; ++i) {
        cudaEvent_t e = nullptr;
        st = cu(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        if (st == HTS_OK) P->ev_img.push_back(e);
    }
    for (cudaEvent_t *e : {&P->ev_start, &P->ev_in, &P->ev_out})
        if (st == HTS_OK) st = cu(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "cudaEventCreate");
    for (cudaEvent_t *e : {&P->ev_t0, &P->ev_t1})
        if (st == HTS_OK) st = cu(cudaEventCreate(e), "cudaEventCreate");
    if (net && st == HTS_OK) {
        size_t px = 0, rows = 0;
        for (const Geom &g : geo) {
            px = std::max(px, (size_t)g.H * g.W);
            rows = std::max(rows, (size_t)g.H * g.nx);
        }
        st = cu(dev_malloc(&P->h16[0], px * 32 * sizeof(__half)), "cudaMalloc(batch network buffers)");
        if (st == HTS_OK) st = cu(dev_malloc(&P->h16[1], px * 32 * sizeof(__half)), "cudaMalloc(batch network buffers)");
        if (st == HTS_OK) st = cu(dev_malloc(&P->cmap, px * sizeof(float)), "cudaMalloc(batch network buffers)");
        if (st == HTS_OK) st = cu(dev_malloc(&P->crows, rows * sizeof(float)), "cudaMalloc(batch network buffers)");
        if (st == HTS_OK) st = cu(cudaStreamCreateWithFlags(&P->cnn_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        if (st == HTS_OK) st = cu(cudaEventCreateWithFlags(&P->ev_cnn, cudaEventDisableTiming), "cudaEventCreate");
        for (int i = 0; i < n && st == HTS_OK; ++i) {
            cudaEvent_t e = nullptr;
            st = cu(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
            if (st == HTS_OK) P->ev_map.push_back(e);
        }
    }
    if (st != HTS_OK) {
        destroy_plan(P);
        return st;
    }
    P->bufs.resize(n);
    P->work.resize(n);
    for (int i = 0; i < n; ++i) {
        bufs_carve(geo[i], P->arena + off[i], &P->bufs[i]);
        P->work[i] = (double)geo[i].nref * (geo[i].C == 3 ? 4.0 : 1.0) * geo[i].K;
    }
    // the phased form: every image in a tensor-core form whose filter takes its geometry
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, sig.device);
    bool phased = n > 0;
    std::vector<unsigned char> probe(std::max(filter_tc_job_size(), match_tc_job_size()));
    for (int i = 0; i < n && phased; ++i)
        phased = par[i].precision >= 1 &&
                 filter_tc_job(nullptr, geo[i], nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0.0, nsm,
                               probe.data()) >= 0;
    if (phased) {
        P->phased = true;
        P->mjob_of.assign(n, -1);
        P->fjob_of.assign(n, -1);
        // groups: matcher by K (precision 1 images), filter by (C, K); jobs of a group contiguous
        for (int pass = 0; pass < 2; ++pass) {
            auto &groups = pass == 0 ? P->mgroups : P->fgroups;
            auto &job_of = pass == 0 ? P->mjob_of : P->fjob_of;
            int row = 0;
            for (int i = 0; i < n; ++i) {
                if (job_of[i] >= 0 || (pass == 0 && par[i].precision != 1)) continue;
                Plan::Group gr;
                gr.K = geo[i].K;
                gr.C = pass == 0 ? 0 : geo[i].C;
                gr.first = row;
                for (int j = i; j < n; ++j)
                    if (job_of[j] < 0 && geo[j].K == gr.K && (pass == 0 ? par[j].precision == 1 : geo[j].C == gr.C)) {
                        job_of[j] = row++;
                        ++gr.njobs;
                    }
                groups.push_back(gr);
            }
        }
        int off2 = 0;
        for (auto *gs : {&P->mgroups, &P->fgroups})
            for (auto &gr : *gs) {
                gr.start_off = off2;
                off2 += gr.njobs + 1;
            }
        for (auto &gr : P->mgroups) gr.queue_off = off2++;
        P->starts_h.assign(off2, 0);
        P->mjob_h.assign(std::max<size_t>(1, P->mgroups.empty() ? 0 : n) * match_tc_job_size(), 0);
        P->fjob_h.assign((size_t)n * filter_tc_job_size(), 0);
        st = cu(dev_malloc(&P->mjob_d, P->mjob_h.size()), "cudaMalloc(batch job tables)");
        if (st == HTS_OK) st = cu(dev_malloc(&P->fjob_d, P->fjob_h.size()), "cudaMalloc(batch job tables)");
        if (st == HTS_OK) st = cu(dev_malloc(&P->starts_d, P->starts_h.size() * sizeof(int)), "cudaMalloc(batch job tables)");
        for (cudaEvent_t &e : P->ev_phase)
            if (st == HTS_OK) st = cu(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        if (st != HTS_OK) {
            destroy_plan(P);
            return st;
        }
    }
    *out = P;
    return HTS_OK;
}

// The job tables of the phased form for these image pointers, uploaded to the plan's device copies.
hts_status upload_jobs(Plan &P, const hts_image *imgs) {
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.sig.device);
    const int n = (int)P.geo.size();
    const size_t ms = match_tc_job_size(), fs = filter_tc_job_size();
    std::vector<int> items_m(n, 0), items_f(n, 0);  // work items per job-table row
    for (int i = 0; i < n; ++i) {
        const Bufs &b = P.bufs[i];
        const Geom &g = P.geo[i];
        if (P.mjob_of[i] >= 0)
            items_m[P.mjob_of[i]] =
                match_tc_job(imgs[i].noisy, g, b.idx, b.green, b.fb, b.st, P.mjob_h.data() + P.mjob_of[i] * ms);
        const float *sref = P.net ? b.sref : imgs[i].sigma_map;
        items_f[P.fjob_of[i]] = filter_tc_job(imgs[i].noisy, g, b.idx, b.b32, b.acc, b.wcount, b.st, sref,
                                              P.net ? 1 : 0, tau_scale(g, P.par[i]), nsm,
                                              P.fjob_h.data() + P.fjob_of[i] * fs, P.fshape);
    }
    // the matcher's queue order within each group: as given, or the largest images first (rows swapped
    // together with their item counts; the results do not depend on the order)
    if (P.largest_first)
        for (auto &gr : P.mgroups) {
            std::vector<int> rows(gr.njobs);
            std::iota(rows.begin(), rows.end(), gr.first);
            std::stable_sort(rows.begin(), rows.end(), [&](int a, int b) { return items_m[a] > items_m[b]; });
            std::vector<unsigned char> tab((size_t)gr.njobs * ms);
            std::vector<int> it(gr.njobs);
            for (int j = 0; j < gr.njobs; ++j) {
                std::memcpy(tab.data() + (size_t)j * ms, P.mjob_h.data() + (size_t)rows[j] * ms, ms);
                it[j] = items_m[rows[j]];
            }
            std::memcpy(P.mjob_h.data() + (size_t)gr.first * ms, tab.data(), tab.size());
            for (int j = 0; j < gr.njobs; ++j) items_m[gr.first + j] = it[j];
        }
    // every group's prefix sums of work items (rows in job-table order)
    for (int pass = 0; pass < 2; ++pass)
        for (auto &gr : pass == 0 ? P.mgroups : P.fgroups) {
            const auto &items = pass == 0 ? items_m : items_f;
            int acc = 0;
            for (int j = 0; j < gr.njobs; ++j) {
                P.starts_h[gr.start_off + j] = acc;
                acc += items[gr.first + j];
            }
            P.starts_h[gr.start_off + gr.njobs] = acc;
            gr.nitems = acc;
        }
    HTS_TRY(cu(cudaMemcpy(P.mjob_d, P.mjob_h.data(), P.mjob_h.size(), cudaMemcpyHostToDevice), "cudaMemcpy(jobs)"));
    HTS_TRY(cu(cudaMemcpy(P.fjob_d, P.fjob_h.data(), P.fjob_h.size(), cudaMemcpyHostToDevice), "cudaMemcpy(jobs)"));
    return cu(cudaMemcpy(P.starts_d, P.starts_h.data(), P.starts_h.size() * sizeof(int), cudaMemcpyHostToDevice),
              "cudaMemcpy(jobs)");
}

// Lane of every image: largest first, each to the least-loaded lane.
std::vector<int> assign_lanes(const Plan &P, int nl) {
    const int n = (int)P.geo.size();
    std::vector<int> order(n), lane(n, 0);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P.work[a] > P.work[b]; });
    std::vector<double> load(nl, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[i] = l;
        load[l] += P.work[i];
    }
    return lane;
}

// Buffers of image i when it runs on lane l.
Bufs slot(const Plan &P, int i, int l) {
    Bufs b = P.bufs[i];
    b.aux = P.auxs[l];
    b.ev_fork = P.ev_img[2 * i];
    b.ev_join = P.ev_img[2 * i + 1];
    return b;
}

// Image i's pipeline on stream s: as hts_denoise, hts_denoise_sigma_map (the caller's map) or
// hts_denoise_learned (the plan's network map, ready once ev_map[i] has fired).
hts_status run_image(Plan &P, const hts_image *imgs, int i, const Bufs &b, cudaStream_t s) {
    if (P.net)
        return denoise_run(imgs[i].noisy, imgs[i].out, P.geo[i], -1.f, nullptr, P.par[i], b, s, b.sref,
                           P.sig.factor, nullptr, nullptr, P.ev_map[i]);
    if (imgs[i].sigma_map)
        return denoise_run(imgs[i].noisy, imgs[i].out, P.geo[i], -1.f, nullptr, P.par[i], b, s,
                           const_cast<float *>(imgs[i].sigma_map), 0.0);
    return denoise_run(imgs[i].noisy, imgs[i].out, P.geo[i], imgs[i].sigma, nullptr, P.par[i], b, s);
}

// Images in the order their work is dealt to lanes (largest first).
std::vector<int> work_order(const Plan &P) {
    std::vector<int> order(P.geo.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P.work[a] > P.work[b]; });
    return order;
}

// The phased form of the batch on nl lanes: per image on its lane the small steps, and between them the
// two heavy kernels as single launches over all images (one per group), on the plan's stream:
//   A  state and sums cleared, Eq. 9 flags, the basis chain and noise floor on the lane's second stream;
//   B  the tensor-core matcher over every (image, tile, plane pass) of the precision-1 images;
//   C  rescue (precision 1) or the exact grouping (precision 2), the rank vote, the noise level, the
//      learned map's check;
//   D  the tensor-core filter over every (image, tile);
//   E  the normalisation.
// Every image's result equals its per-image call, bit for bit (the same kernels on the same work items;
// integer aggregation).
hts_status capture_phases(Plan &P, const hts_image *imgs, const std::vector<int> &lane, int nl) {
    const int n = (int)P.geo.size();
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.sig.device);
    auto join_lanes = [&](cudaEvent_t ev) -> hts_status {  // origin waits for every lane, then the lanes for it
        for (int l = 0; l < nl; ++l) {
            HTS_TRY(cu(cudaEventRecord(P.ev_lane[l], P.lanes[l]), "cudaEventRecord"));
            HTS_TRY(cu(cudaStreamWaitEvent(P.origin, P.ev_lane[l], 0), "cudaStreamWaitEvent"));
        }
        return cu(cudaEventRecord(ev, P.origin), "cudaEventRecord");
    };
    auto lanes_wait = [&](cudaEvent_t ev) -> hts_status {
        for (int l = 0; l < nl; ++l) HTS_TRY(cu(cudaStreamWaitEvent(P.lanes[l], ev, 0), "cudaStreamWaitEvent"));
        return HTS_OK;
    };
    // A
    for (int i = 0; i < n; ++i) {
        const Bufs b = slot(P, i, lane[i]);
        const Geom &g = P.geo[i];
        const hts_params &p = P.par[i];
        cudaStream_t s = P.lanes[lane[i]];
        const size_t hw = (size_t)g.H * g.W;
        // as run_image: a map (the network's or the caller's) stands for sigma; only a checked map needs the estimate
        const float sig = (P.net || imgs[i].sigma_map) ? -1.f : imgs[i].sigma;
        const bool need_sigma = sig < 0 && (imgs[i].sigma_map == nullptr || P.net);
        HTS_TRY(cu(cudaMemsetAsync(b.st, 0, sizeof(DevState), s), "cudaMemsetAsync(state)"));
        HTS_TRY(cu(cudaMemsetAsync(b.acc, 0, hw * g.C * sizeof(long long), s), "cudaMemsetAsync(acc)"));
        HTS_TRY(cu(cudaMemsetAsync(b.wcount, 0, hw * sizeof(int), s), "cudaMemsetAsync(weights)"));
        if (p.precision == 1 && g.C == 3) HTS_TRY(launch_gcp_flags(imgs[i].noisy, g, p.gamma_gcp, b.green, s));
        HTS_TRY(cu(cudaEventRecord(b.ev_fork, s), "cudaEventRecord"));
        HTS_TRY(cu(cudaStreamWaitEvent(b.aux, b.ev_fork, 0), "cudaStreamWaitEvent"));
        HTS_TRY(launch_basis(imgs[i].noisy, g, b.cov, b.b64, b.b32, b.eig, b.aux));
        if (need_sigma) HTS_TRY(launch_sigma_floor(g, p, b.eig, b.st, b.aux));
        HTS_TRY(cu(cudaEventRecord(b.ev_join, b.aux), "cudaEventRecord"));
    }
    HTS_TRY(join_lanes(P.ev_phase[0]));
    // B
    for (const auto &gr : P.mgroups)
        HTS_TRY(launch_match_tc_batch(gr.K, P.mjob_h.data() + gr.first * match_tc_job_size(),
                                      P.mjob_d + gr.first * match_tc_job_size(), P.starts_d + gr.start_off,
                                      gr.njobs, gr.nitems, P.starts_d + gr.queue_off, nsm, P.origin));
    HTS_TRY(cu(cudaEventRecord(P.ev_phase[1], P.origin), "cudaEventRecord"));
    HTS_TRY(lanes_wait(P.ev_phase[1]));
    // C
    for (int i = 0; i < n; ++i) {
        const Bufs b = slot(P, i, lane[i]);
        const Geom &g = P.geo[i];
        const hts_params &p = P.par[i];
        cudaStream_t s = P.lanes[lane[i]];
        const float sig = (P.net || imgs[i].sigma_map) ? -1.f : imgs[i].sigma;
        const bool need_sigma = sig < 0 && (imgs[i].sigma_map == nullptr || P.net);
        if (p.precision == 1) HTS_TRY(launch_match_rescue(imgs[i].noisy, g, b.idx, b.green, b.fb, b.st, s));
        else HTS_TRY(launch_match(imgs[i].noisy, g, p.gamma_gcp, b.idx, b.green, b.fb, b.st, s));
        if (need_sigma && p.adjust_rank) HTS_TRY(launch_sigma_vote(imgs[i].noisy, g, p, b.idx, b.redo, b.st, s));
        HTS_TRY(cu(cudaStreamWaitEvent(s, b.ev_join, 0), "cudaStreamWaitEvent"));
        if (need_sigma) HTS_TRY(launch_sigma_final(g, p, b.st, s));
        else HTS_TRY(launch_set_sigma(sig > 0 ? (double)sig : 0.0, g, p, b.st, s));
        if (P.net) {
            HTS_TRY(cu(cudaStreamWaitEvent(s, P.ev_map[i], 0), "cudaStreamWaitEvent"));
            HTS_TRY(launch_learned_check(b.sref, g.nref, P.sig.factor, b.st, s));
        }
    }
    HTS_TRY(join_lanes(P.ev_phase[2]));
    // D
    for (const auto &gr : P.fgroups)
        HTS_TRY(launch_filter_tc_batch(gr.C, gr.K, P.fjob_h.data() + gr.first * filter_tc_job_size(),
                                       P.fjob_d + gr.first * filter_tc_job_size(), P.starts_d + gr.start_off,
                                       gr.njobs, gr.nitems, nsm, P.origin));
    HTS_TRY(cu(cudaEventRecord(P.ev_phase[3], P.origin), "cudaEventRecord"));
    HTS_TRY(lanes_wait(P.ev_phase[3]));
    // E
    for (int i = 0; i < n; ++i) {
        const Bufs b = slot(P, i, lane[i]);
        const Geom &g = P.geo[i];
        HTS_TRY(launch_normalize_box(b.acc, b.wcount, imgs[i].out, g.H, g.W, g.C, P.lanes[lane[i]]));
    }
    return HTS_OK;
}

// Records the whole batch on nl lanes into a new graph.
hts_status capture(Plan &P, const hts_image *imgs, int nl, cudaGraph_t *out, unsigned long long *kernels) {
    const int n = (int)P.geo.size();
    const std::vector<int> lane = assign_lanes(P, nl);
    if (P.phased) HTS_TRY(upload_jobs(P, imgs));
    reset_captured_launches();
    HTS_TRY(cu(cudaStreamBeginCapture(P.origin, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture"));
    hts_status st = cu(cudaEventRecord(P.ev_start, P.origin), "cudaEventRecord");
    for (int l = 0; l < nl && st == HTS_OK; ++l) st = cu(cudaStreamWaitEvent(P.lanes[l], P.ev_start, 0), "cudaStreamWaitEvent");
    if (P.net && st == HTS_OK) {  // the networks' maps, largest image first, into the images' slots
        st = cu(cudaStreamWaitEvent(P.cnn_stream, P.ev_start, 0), "cudaStreamWaitEvent");
        for (int i : work_order(P)) {
            if (st != HTS_OK) break;
            st = cnn_sigma_refs_into(P.net, imgs[i].noisy, P.geo[i], P.h16[0], P.h16[1], P.cmap, P.crows,
                                     P.bufs[i].sref, P.cnn_stream);
            if (st == HTS_OK) st = cu(cudaEventRecord(P.ev_map[i], P.cnn_stream), "cudaEventRecord");
        }
        if (st == HTS_OK) st = cu(cudaEventRecord(P.ev_cnn, P.cnn_stream), "cudaEventRecord");
    }
    if (P.phased) {
        if (st == HTS_OK) st = capture_phases(P, imgs, lane, nl);
    } else {
        for (int i = 0; i < n && st == HTS_OK; ++i) st = run_image(P, imgs, i, slot(P, i, lane[i]), P.lanes[lane[i]]);
    }
    for (int l = 0; l < nl && st == HTS_OK; ++l) {
        st = cu(cudaEventRecord(P.ev_lane[l], P.lanes[l]), "cudaEventRecord");
        if (st == HTS_OK) st = cu(cudaStreamWaitEvent(P.origin, P.ev_lane[l], 0), "cudaStreamWaitEvent");
    }
    if (P.net && st == HTS_OK) st = cu(cudaStreamWaitEvent(P.origin, P.ev_cnn, 0), "cudaStreamWaitEvent");
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(P.origin, &g);
    if (st != HTS_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    HTS_TRY(cu(e, "cudaStreamEndCapture"));
    *out = g;
    *kernels = captured_launches();
    return HTS_OK;
}

hts_status instantiate(cudaGraph_t g, cudaGraphExec_t *exec) {
    return cu(cudaGraphInstantiate(exec, g, 0), "cudaGraphInstantiate");
}

// Milliseconds of one launch of exec on the plan's stream (after one warm-up launch).
hts_status time_exec(Plan &P, cudaGraphExec_t exec, float *ms) {
    HTS_TRY(cu(cudaGraphLaunch(exec, P.origin), "cudaGraphLaunch"));
    HTS_TRY(cu(cudaEventRecord(P.ev_t0, P.origin), "cudaEventRecord"));
    HTS_TRY(cu(cudaGraphLaunch(exec, P.origin), "cudaGraphLaunch"));
    HTS_TRY(cu(cudaEventRecord(P.ev_t1, P.origin), "cudaEventRecord"));
    HTS_TRY(cu(cudaEventSynchronize(P.ev_t1), "cudaEventSynchronize"));
    return cu(cudaEventElapsedTime(ms, P.ev_t0, P.ev_t1), "cudaEventElapsedTime");
}

// Tile shape of every geometry of the batch that has none yet.
hts_status tune_tiles(Plan &P, const hts_image *imgs) {
    const int n = (int)P.geo.size();
    std::vector<std::vector<int>> done;
    for (int i = 0; i < n; ++i) {
        const Geom &g = P.geo[i];
        TileChoice have;
        if (tuned_tile(g, &have)) continue;
        const std::vector<int> key = {g.H, g.W, g.C, g.K, g.R, g.step};
        if (std::find(done.begin(), done.end(), key) != done.end()) continue;
        done.push_back(key);
        TileChoice cands[8];
        const int nc = tile_candidates(g, cands, 8);
        TileChoice best = cands[0];
        float best_ms = 1e30f;
        for (int c = 0; c < nc && nc > 1; ++c) {
            force_tile(&cands[c]);
            float total = 0.f;
            hts_status st = HTS_OK;
            for (int rep = 0; rep < 3 && st == HTS_OK; ++rep) {  // rep 0 warms up
                if (rep == 1) st = cu(cudaEventRecord(P.ev_t0, P.origin), "cudaEventRecord");
                if (st == HTS_OK)
                    st = denoise_run(imgs[i].noisy, imgs[i].out, g, imgs[i].sigma, nullptr, P.par[i], slot(P, i, 0),
                                     P.origin);
            }
            if (st == HTS_OK) st = cu(cudaEventRecord(P.ev_t1, P.origin), "cudaEventRecord");
            if (st == HTS_OK) st = cu(cudaEventSynchronize(P.ev_t1), "cudaEventSynchronize");
            if (st == HTS_OK) st = cu(cudaEventElapsedTime(&total, P.ev_t0, P.ev_t1), "cudaEventElapsedTime");
            force_tile(nullptr);
            HTS_TRY(st);
            if (total < best_ms) {
                best_ms = total;
                best = cands[c];
            }
        }
        set_tuned_tile(g, best);
    }
    return HTS_OK;
}

// First call of a signature: tile shapes, then the lane count, keeping the fastest graph.
hts_status build(Plan &P, const hts_image *imgs) {
    HTS_TRY(tune_tiles(P, imgs));
    const int n = (int)P.geo.size();
    float best_ms = 1e30f;
    for (int nl : {1, 2, 4, 8}) {
        if (nl > 1 && nl > n) break;
        cudaGraph_t g = nullptr;
        unsigned long long k = 0;
        HTS_TRY(capture(P, imgs, nl, &g, &k));
        cudaGraphExec_t ex = nullptr;
        hts_status st = instantiate(g, &ex);
        cudaGraphDestroy(g);
        HTS_TRY(st);
        ++P.captures;
        float ms = 0.f;
        st = time_exec(P, ex, &ms);
        if (st != HTS_OK) {
            cudaGraphExecDestroy(ex);
            return st;
        }
        count_launches(2 * k);
        if (ms < best_ms) {
            best_ms = ms;
            if (P.exec) cudaGraphExecDestroy(P.exec);
            P.exec = ex;
            P.nlanes = nl;
            P.kernels = k;
        } else {
            cudaGraphExecDestroy(ex);
        }
    }
    if (P.phased) {
        // the search schedule of the phased form: the filter's tile shape (each geometry's model, or one
        // shape for all: 8x8, 4x8, 4x4, 2x4 groups) and the matcher's queue order, each kept if faster
        auto trial = [&](int fshape, bool lf) -> hts_status {
            const int f0 = P.fshape;
            const bool l0 = P.largest_first;
            P.fshape = fshape;
            P.largest_first = lf;
            cudaGraph_t g = nullptr;
            unsigned long long k = 0;
            HTS_TRY(capture(P, imgs, P.nlanes, &g, &k));
            cudaGraphExec_t ex = nullptr;
            hts_status st = instantiate(g, &ex);
            cudaGraphDestroy(g);
            HTS_TRY(st);
            ++P.captures;
            float ms = 0.f;
            st = time_exec(P, ex, &ms);
            if (st != HTS_OK) {
                cudaGraphExecDestroy(ex);
                return st;
            }
            count_launches(2 * k);
            if (ms < best_ms) {
                best_ms = ms;
                cudaGraphExecDestroy(P.exec);
                P.exec = ex;
                P.kernels = k;
            } else {
                cudaGraphExecDestroy(ex);
                P.fshape = f0;
                P.largest_first = l0;
            }
            return HTS_OK;
        };
        for (int fsh : {0, 1, 2, 3}) HTS_TRY(trial(fsh, P.largest_first));
        HTS_TRY(trial(P.fshape, !P.largest_first));
        HTS_TRY(upload_jobs(P, imgs));  // the device tables of the kept schedule
    }
    P.bound.assign(imgs, imgs + n);
    return HTS_OK;
}

bool same_binding(const Plan &P, const hts_image *imgs) {
    for (size_t i = 0; i < P.bound.size(); ++i) {
        const hts_image &a = P.bound[i], &b = imgs[i];
        if (a.noisy != b.noisy || a.out != b.out || a.sigma_map != b.sigma_map ||
            std::memcmp(&a.sigma, &b.sigma, sizeof(float)) != 0)
            return false;
    }
    return true;
}

// Same signature, new pointers or noise levels: capture again and update the
// instantiated graph (re-instantiate if the update is refused).
hts_status rebind(Plan &P, const hts_image *imgs) {
    cudaGraph_t g = nullptr;
    unsigned long long k = 0;
    HTS_TRY(capture(P, imgs, P.nlanes, &g, &k));
    ++P.captures;
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(P.exec, g, &info) == cudaSuccess) {
        ++P.updates;
    } else {
        cudaGetLastError();
        cudaGraphExecDestroy(P.exec);
        P.exec = nullptr;
        hts_status st = instantiate(g, &P.exec);
        if (st != HTS_OK) {
            cudaGraphDestroy(g);
            return st;
        }
    }
    cudaGraphDestroy(g);
    P.kernels = k;
    P.bound.assign(imgs, imgs + P.geo.size());
    return HTS_OK;
}

}  // namespace

void batch_shutdown() {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto &kv : g_plans) destroy_plan(kv.second);
    g_plans.clear();
    g_last.clear();
}

}  // namespace hts

using namespace hts;

namespace hts {
namespace {

hts_status batch_impl(const hts_image *imgs, int n, const hts_params *p, hts_cnn *net, double factor,
                      void *stream) {
    if (n < 0 || (n > 0 && !imgs)) return report(HTS_EINVAL, "bad batch");
    if (!p) return report(HTS_EINVAL, "params is NULL");
    std::vector<Geom> geo(n);
    std::vector<hts_params> par(n);
    Sig sig;
    if (net) {
        sig.net = net;
        sig.window = hts_cnn_window(net);
        sig.factor = factor;
    }
    for (int i = 0; i < n; ++i) {
        const hts_params *pi = imgs[i].params ? imgs[i].params : p;
        HTS_TRY(validate(imgs[i].H, imgs[i].W, imgs[i].C, pi, &geo[i]));
        std::memset(&par[i], 0, sizeof(hts_params));  // field by field: padding stays zero
        par[i].ps = pi->ps;
        par[i].K = pi->K;
        par[i].win = pi->win;
        par[i].step = pi->step;
        par[i].gamma_gcp = pi->gamma_gcp;
        par[i].beta = pi->beta;
        par[i].gamma_rank = pi->gamma_rank;
        par[i].tau_mult = pi->tau_mult;
        par[i].adjust_rank = pi->adjust_rank;
        par[i].mp_correct = pi->mp_correct;
        par[i].precision = pi->precision;
        const unsigned char *pb = reinterpret_cast<const unsigned char *>(&par[i]);
        sig.par.insert(sig.par.end(), pb, pb + sizeof(hts_params));
        if (!imgs[i].noisy || !imgs[i].out || imgs[i].noisy == imgs[i].out)
            return report(HTS_EINVAL, "bad image pointers in batch");
        if (imgs[i].sigma != imgs[i].sigma || imgs[i].sigma == __builtin_inff() || imgs[i].sigma == -__builtin_inff())
            return report(HTS_EINVAL, "sigma must be finite");
        if (net && imgs[i].sigma_map) return report(HTS_EINVAL, "the learned batch takes no caller sigma maps");
        if (net && hts_cnn_channels(net) != imgs[i].C)
            return report(HTS_EINVAL, "network built for another channel count");
        const bool est = net || imgs[i].sigma_map || imgs[i].sigma < 0;
        sig.dims.insert(sig.dims.end(),
                        {imgs[i].H, imgs[i].W, imgs[i].C, est ? 1 : 0, imgs[i].sigma_map ? 1 : 0});
    }
    if (n == 0) return HTS_OK;
    HTS_TRY(cu(cudaGetDevice(&sig.device), "cudaGetDevice"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lk(g_bmu);
    Plan *P = nullptr;
    auto it = g_plans.find(sig);
    bool fresh = false;
    if (it != g_plans.end()) {
        P = it->second;
    } else {
        if (g_plans.size() >= MAX_PLANS) {  // drop the least recently used plan
            auto lru = std::min_element(g_plans.begin(), g_plans.end(), [](const auto &a, const auto &b) {
                return a.second->last_use < b.second->last_use;
            });
            for (auto l = g_last.begin(); l != g_last.end();) l = (l->second == lru->second) ? g_last.erase(l) : std::next(l);
            destroy_plan(lru->second);
            g_plans.erase(lru);
        }
        HTS_TRY(create_plan(sig, geo, par, net, &P));
        g_plans[sig] = P;
        fresh = true;
    }
    P->last_use = ++g_tick;
    // the caller's stream hands over to the plan's stream and back
    HTS_TRY(cu(cudaEventRecord(P->ev_in, s), "cudaEventRecord"));
    HTS_TRY(cu(cudaStreamWaitEvent(P->origin, P->ev_in, 0), "cudaStreamWaitEvent"));
    if (fresh) HTS_TRY(build(*P, imgs));
    else if (!same_binding(*P, imgs)) HTS_TRY(rebind(*P, imgs));
    HTS_TRY(cu(cudaGraphLaunch(P->exec, P->origin), "cudaGraphLaunch"));
    count_launches(P->kernels);
    HTS_TRY(cu(cudaEventRecord(P->ev_out, P->origin), "cudaEventRecord"));
    HTS_TRY(cu(cudaStreamWaitEvent(s, P->ev_out, 0), "cudaStreamWaitEvent"));
    g_last[std::make_pair(sig.device, s)] = P;
    return HTS_OK;
}

}  // namespace

void batch_drop_net(const hts_cnn *net) {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (it->second->net != net) {
            ++it;
            continue;
        }
        Plan *P = it->second;
        for (auto l = g_last.begin(); l != g_last.end();) l = (l->second == P) ? g_last.erase(l) : std::next(l);
        destroy_plan(P);
        it = g_plans.erase(it);
    }
}

}  // namespace hts

extern "C" hts_status hts_denoise_batch(const hts_image *imgs, int n, const hts_params *p, void *stream) {
    return batch_impl(imgs, n, p, nullptr, 0.0, stream);
}

extern "C" hts_status hts_denoise_batch_learned(const hts_image *imgs, int n, hts_cnn *net, double fallback_factor,
                                                const hts_params *p, void *stream) {
    if (!net) return report(HTS_EINVAL, "network is NULL");
    if (!(fallback_factor > 1.0) || !std::isfinite(fallback_factor))
        return report(HTS_EINVAL, "fallback_factor must be > 1");
    return batch_impl(imgs, n, p, net, fallback_factor, stream);
}

extern "C" hts_status hts_last_batch_stats(hts_stats *out, int n, hts_batch_info *info, void *stream) {
    if (n < 0 || (n > 0 && !out)) return report(HTS_EINVAL, "bad arguments");
    int dev = 0;
    HTS_TRY(cu(cudaGetDevice(&dev), "cudaGetDevice"));
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_last.find(std::make_pair(dev, static_cast<cudaStream_t>(stream)));
    if (it == g_last.end()) return report(HTS_EINVAL, "no batch has run on this stream");
    Plan *P = it->second;
    const int m = std::min(n, (int)P->geo.size());
    HTS_TRY(cu(cudaStreamSynchronize(P->origin), "cudaStreamSynchronize"));
    int err = 0;
    for (int i = 0; i < m; ++i) {
        DevState hs;
        HTS_TRY(cu(cudaMemcpy(&hs, P->bufs[i].st, sizeof(DevState), cudaMemcpyDeviceToHost), "cudaMemcpy"));
        hts_stats &o = out[i];
        std::memset(&o, 0, sizeof(o));
        o.nref = hs.nref;
        o.match_reranked = hs.match_reranked;
        o.match_fallback = hs.match_fallback;
        o.filter_redo = hs.filter_redo;
        o.filter_exact = hs.filter_exact;
        o.vote_uncertain = hs.vote_uncertain;
        o.sigma = hs.sigma_hat;
        o.tau = hs.tau;
        o.filter_fixed = hs.filter_fixed;
        o.learned = hs.learned;
        o.learned_ratio = hs.learned_ratio;
        o.device_error = hs.error;
        if (hs.error != 0 && err != 2) err = hs.error;
    }
    if (info) {
        info->images = (int)P->geo.size();
        info->lanes = P->nlanes;
        info->kernels = (int)P->kernels;
        info->captures = P->captures;
        info->updates = P->updates;
        info->phased = P->phased ? 1 : 0;
    }
    return device_status(err);
}

extern "C" hts_status hts_tuned_tile(int H, int W, int C, const hts_params *p, int *ty, int *tx) {
    if (!ty || !tx) return report(HTS_EINVAL, "NULL pointer");
    Geom g;
    HTS_TRY(validate(H, W, C, p, &g));
    TileChoice c;
    if (!tuned_tile(g, &c)) {
        *ty = -1;
        *tx = -1;
    } else {
        *ty = c.ty;
        *tx = c.tx;
    }
    return HTS_OK;
}
