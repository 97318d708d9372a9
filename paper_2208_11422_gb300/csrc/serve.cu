// Serving: continuous batching of light-field RL reconstructions over resident
// PSF sets (lfd_server_* / lfd_submit / lfd_poll, include/lfd.h).
//
// Fig. 1 of the paper moves the PSF to the GPU once and estimates the memory a
// reconstruction needs before allocating it. Here several PSF sets stay
// resident as FFT spectra, and each request's footprint is reserved in one
// device arena when it is admitted.
//
// One scheduler thread drives every set on the set's own CUDA stream. A set is
// either idle or has one tick in flight. A tick enqueues:
//   1. the copies of finished frames' results to their v_out;
//   2. one RL iteration of every iterating frame. The forward projection runs
//      over all their FFT columns (tiles) as one transform / contraction /
//      transform chain per max_cols columns; the backprojection likewise; then
//      per frame the exact low-sensitivity correction, the update and the
//      metric;
//   3. the start of newly admitted frames: their data and cosine tables, and
//      H^T 1. H^T 1 is the backprojection of an all-ones image, done in the
//      same backward chain as step 2, followed by the low-sensitivity list,
//      its exact values and 1 / H^T 1;
//   4. a copy of the frames' entropy and flux to pinned host memory, then an
//      event.
// When the event has passed, the scheduler applies each frame's stopping rule
// (the one lfd_rl_iterate uses), retires finished frames, and admits queued
// requests whose footprint fits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fft_proj.h"
#include "lfd_internal.h"
#include "tc_cgemm.h"

namespace lfd {

int64_t align256(int64_t b) { return (b + 255) & ~(int64_t)255; }

namespace {

using Clock = std::chrono::steady_clock;

}  // namespace

// First-fit bookkeeping of offsets in [0, cap) with coalescing on release
// (host only; the server's device arena is one allocation managed by it).
int64_t FreeList::alloc(int64_t bytes) {
    bytes = align256(bytes);
    if (bytes <= 0) return -1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < bytes) continue;
        const int64_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest > 0) free_[off + bytes] = rest;
        taken_[off] = bytes;
        used += bytes;
        peak = std::max(peak, used);
        return off;
    }
    return -1;
}
bool FreeList::release(int64_t off) {
    auto t = taken_.find(off);
    if (t == taken_.end()) return false;
    int64_t size = t->second;
    taken_.erase(t);
    used -= size;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && next->first == off + size) {
        size += next->second;
        next = free_.erase(next);
    }
    if (next != free_.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += size;
            return true;
        }
    }
    free_[off] = size;
    return true;
}

namespace {

class Arena {
  public:
    char* base = nullptr;
    int64_t cap = 0;
    FreeList fl;

    cudaError_t init(int64_t bytes) {
        if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc((void**)&base, (size_t)bytes);
        if (e != cudaSuccess) {
            base = nullptr;
            return e;
        }
        cap = bytes;
        fl.reset(bytes);
        return cudaSuccess;
    }
    int64_t alloc(int64_t bytes) { return fl.alloc(bytes); }
    void release(int64_t off) { fl.release(off); }
    ~Arena() {
        if (base) cudaFree(base);
    }
};

enum class JobState { Queued, New, Iter, Finishing, Done };

struct Job {
    uint64_t ticket = 0;
    lfd_request req{};
    int set = 0;
    Geo g{};
    int tiles_x = 0, ntile = 0, XS = 0, YS = 0, max_iter = 0, nflux = 0;
    int64_t bytes = 0, off = -1;
    // device buffers, carved from the arena block
    float *ycm = nullptr, *vcm[2] = {nullptr, nullptr}, *xcm = nullptr, *invcm = nullptr;
    float *rcm = nullptr, *rimg = nullptr, *mip = nullptr;
    float2* cosW = nullptr;  // FP64 basis split as FP32 hi + lo
    double *cosH = nullptr, *G = nullptr, *rowE2 = nullptr, *coef = nullptr;
    double* flux_part = nullptr;
    int* low = nullptr;
    int* n_low = nullptr;
    unsigned* mx = nullptr;
    int cur = 0, ran = 0, done = 0, res_buf = 0;
    std::vector<double> E, Fl;
    JobState state = JobState::Queued;
    lfd_status status = LFD_OK;
    bool y_dev = false, v_dev = false;
    Clock::time_point t_submit, t_admit, t_done;
};

// footprint of a frame (and the layout carve() gives its block)
int64_t job_layout(Job* j, char* base) {
    const Geo& g = j->g;
    const int64_t L2 = (int64_t)g.Ly * g.Lx, vox = (int64_t)g.C * L2, img = (int64_t)g.H * g.W;
    int64_t o = 0;
    auto take = [&](int64_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += align256(bytes);
        return p;
    };
    j->ycm = (float*)take(4 * g.S * L2);
    j->vcm[0] = (float*)take(4 * vox);
    j->vcm[1] = (float*)take(4 * vox);
    j->xcm = (float*)take(4 * vox);
    j->invcm = (float*)take(4 * vox);
    j->rcm = (float*)take(4 * g.S * L2);
    j->rimg = (float*)take(4 * img);
    j->mip = (float*)take(4 * img);
    j->cosW = (float2*)take(8 * (int64_t)j->XS * g.W);
    j->cosH = (double*)take(8 * (int64_t)j->YS * g.H);
    j->G = (double*)take(8 * (int64_t)g.H * j->XS);
    j->rowE2 = (double*)take(8 * (int64_t)g.H);
    j->coef = (double*)take(8 * ((int64_t)j->XS * j->YS + kMetricScratch));
    j->flux_part = (double*)take(8 * (int64_t)j->nflux);
    j->low = (int*)take(4 * vox);
    j->n_low = (int*)take(4);
    j->mx = (unsigned*)take(4);
    return o;
}

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct PsfSet {
    Geo gmax{};
    FftPlan plan{};
    FftBuffers fb{};
    LoPlanes lo{};         // adaptive lo planes of the PSF spectra (split BF16)
    float* psf = nullptr;  // [Nz][N][N][P][P] for the exact backprojection
    std::vector<void*> owned;
    int max_tiles = 0, XSmax = 0, YSmax = 0;
    int64_t tab_stride = 0, resident = 0;
    FrameCols* d_fr = nullptr;
    int* d_colf = nullptr;
    FrameCols* h_fr = nullptr;  // pinned
    int* h_colf = nullptr;      // pinned
    double* d_hist = nullptr;   // [2][mf] entropy, flux
    double* h_hist = nullptr;   // pinned copy
    double* h_tab = nullptr;    // pinned cosine tables of the frames a tick starts
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Job*> iter, fresh, finishing;       // membership between ticks
    std::vector<Job*> ran_iter, ran_new, ran_fin;   // what the tick in flight covers
    int64_t tick_cols = 0;

    ~PsfSet() {
        if (fb.cg) cgemm_destroy(fb.cg);
        cgemm_free_lo(&lo);
        for (void* p : owned) cudaFree(p);
        if (h_fr) cudaFreeHost(h_fr);
        if (h_colf) cudaFreeHost(h_colf);
        if (h_hist) cudaFreeHost(h_hist);
        if (h_tab) cudaFreeHost(h_tab);
        if (ev) cudaEventDestroy(ev);
        if (st) cudaStreamDestroy(st);
    }
    template <class T>
    cudaError_t dev(T** p, int64_t count) {
        const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        if (injected_alloc_failure()) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        cudaError_t e = cudaMalloc((void**)p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            return e;
        }
        owned.push_back(*p);
        resident += (int64_t)bytes;
        return cudaSuccess;
    }
};

}  // namespace
}  // namespace lfd

using namespace lfd;

struct lfd_server {
    lfd_server_options opt{};
    int device = 0, sm_count = 0;
    std::vector<std::unique_ptr<PsfSet>> sets;
    Arena arena;
    bool started = false, stop = false;
    mutable std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> queue;
    std::unordered_map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    std::thread thr;
    std::string err;
    lfd_server_stats stats{};
};

namespace {

void finish_job(lfd_server* s, Job* j, lfd_status st) {
    j->status = st;
    j->state = JobState::Done;
    j->t_done = Clock::now();
    if (j->req.entropy_hist)
        for (int k = 0; k < j->max_iter; ++k) j->req.entropy_hist[k] = k < j->ran ? j->E[k] : NAN;
    if (st == LFD_OK) ++s->stats.completed;
    s->cv_done.notify_all();
}

// every frame of the set ends with status st (after a failed launch or wait);
// their arena blocks stay reserved, as kernels may still touch them
void fail_set(lfd_server* s, PsfSet& ps, lfd_status st, const std::string& why) {
    s->err = why;
    for (auto* v : {&ps.iter, &ps.fresh, &ps.finishing, &ps.ran_iter, &ps.ran_new, &ps.ran_fin}) {
        for (Job* j : *v)
            if (j->state != JobState::Done) finish_job(s, j, st);
        v->clear();
    }
    ps.busy = false;
}

// the tick in flight has finished: stopping rules, retirements, promotions
void complete_tick(lfd_server* s, PsfSet& ps) {
    if (ps.fb.cg) {
        const int te = cgemm_error(ps.fb.cg);
        if (te != 0) {
            fail_set(s, ps, LFD_ETIMEDOUT,
                     "tensor-core contraction gave up waiting (code " + std::to_string(te) + ")");
            return;
        }
    }
    const int mf = s->opt.max_frames_per_set;
    for (Job* j : ps.ran_fin) {
        s->arena.release(j->off);
        finish_job(s, j, LFD_OK);
    }
    ps.ran_fin.clear();
    std::vector<Job*> keep;
    for (size_t i = 0; i < ps.ran_iter.size(); ++i) {
        Job* j = ps.ran_iter[i];
        const int k = j->ran;
        j->E.push_back(ps.h_hist[i]);
        j->Fl.push_back(ps.h_hist[mf + i]);
        j->ran = k + 1;
        // E_{k+1} < E_k: the frame keeps v^k, still in buffer cur
        if (j->req.stop_at_predicted && k >= 1 && j->E[k] < j->E[k - 1]) {
            j->done = k;
            j->res_buf = j->cur;
        } else {
            j->cur ^= 1;
            if (j->ran < j->max_iter) {
                keep.push_back(j);
                continue;
            }
            j->done = j->ran;
            j->res_buf = j->cur;
        }
        j->state = JobState::Finishing;
        ps.finishing.push_back(j);
    }
    s->stats.frame_iterations += (int64_t)ps.ran_iter.size();
    for (Job* j : ps.ran_new) {
        j->state = JobState::Iter;
        keep.push_back(j);
    }
    ps.iter.swap(keep);
    ps.ran_iter.clear();
    ps.ran_new.clear();
    ps.busy = false;
}

#define TICK_CK(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_); \
    } while (0)

// Issues the work of one tick of a set (its lists already swapped in):
// results out, the column table, new frames' inputs, the projections, the
// updates and metrics, the histories to the host and the tick's event.
// Touches only the set's own buffers and the device buffers of its frames in
// flight, which no client call reads, so it runs without the server's lock.
// Returns "" or what failed.
std::string launch_tick(lfd_server* s, PsfSet& ps) {
    cudaGetLastError();  // the launch checks below read the thread's last error
    const lfd_options& o = s->opt.opt;
    const int mf = s->opt.max_frames_per_set;
    cudaStream_t st = ps.st;
    const Geo& gs = ps.gmax;

    // 1. results out (stack order), straight into v_out or through xcm
    for (Job* j : ps.ran_fin) {
        const Geo& g = j->g;
        float* dst = j->v_dev ? j->req.v_out : j->xcm;
        TICK_CK(launch_depoly_volume_cm(j->vcm[j->res_buf], g, dst, st));
        if (!j->v_dev)
            TICK_CK(cudaMemcpyAsync(j->req.v_out, j->xcm, sizeof(float) * (size_t)g.C * g.Ly * g.Lx,
                                    cudaMemcpyDeviceToHost, st));
    }

    // column table: iterating frames first, then the new ones
    if ((int)(ps.ran_iter.size() + ps.ran_new.size()) > mf) return "more frames in a tick than max_frames_per_set";
    int nfr = 0, col = 0, iter_cols = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (Job* j : pass == 0 ? ps.ran_iter : ps.ran_new) {
            FrameCols& d = ps.h_fr[nfr];
            d.vsrc = j->vcm[j->cur];
            d.rsrc = pass == 0 ? j->rcm : nullptr;
            d.rcm = j->rcm;
            d.ycm = j->ycm;
            d.rimg = j->rimg;
            d.xcm = j->xcm;
            d.Ly = j->g.Ly;
            d.Lx = j->g.Lx;
            d.tiles_x = j->tiles_x;
            d.col0 = col;
            for (int t = 0; t < j->ntile; ++t) ps.h_colf[col + t] = nfr;
            col += j->ntile;
            ++nfr;
        }
        if (pass == 0) iter_cols = col;
    }
    const int all_cols = col;
    if (nfr > 0) {
        TICK_CK(cudaMemcpyAsync(ps.d_fr, ps.h_fr, sizeof(FrameCols) * nfr, cudaMemcpyHostToDevice, st));
        TICK_CK(cudaMemcpyAsync(ps.d_colf, ps.h_colf, sizeof(int) * all_cols, cudaMemcpyHostToDevice, st));
    }

    // 3a. new frames: data, cosine tables, start volume
    for (size_t i = 0; i < ps.ran_new.size(); ++i) {
        Job* j = ps.ran_new[i];
        const Geo& g = j->g;
        const float* ysrc = j->req.y;
        if (!j->y_dev) {
            TICK_CK(cudaMemcpyAsync(j->rimg, j->req.y, sizeof(float) * (size_t)g.H * g.W,
                                    cudaMemcpyHostToDevice, st));
            ysrc = j->rimg;
        }
        TICK_CK(launch_poly_image_cm(ysrc, g, j->ycm, st));
        double* tab = ps.h_tab + (int64_t)i * ps.tab_stride;
        const std::vector<float2> tw = split_table(dct_table(j->XS, g.W));
        const std::vector<double> th = dct_table(j->YS, g.H);
        static_assert(sizeof(float2) == sizeof(double), "one table entry either way");
        std::memcpy(tab, tw.data(), tw.size() * sizeof(float2));
        std::memcpy(tab + tw.size(), th.data(), th.size() * sizeof(double));
        TICK_CK(cudaMemcpyAsync(j->cosW, tab, tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        TICK_CK(cudaMemcpyAsync(j->cosH, tab + tw.size(), th.size() * sizeof(double),
                                cudaMemcpyHostToDevice, st));
        TICK_CK(launch_fill_cm(j->vcm[0], (int64_t)g.C * g.Ly * g.Lx, 1.0f, st));
    }

    // 2. forward and backward projections over the columns, max_cols at a time
    const int mc = s->opt.max_cols;
    for (int c0 = 0; c0 < iter_cols; c0 += mc)
        TICK_CK(fft_forward_tab(ps.plan, gs, ps.fb, ps.d_fr, ps.d_colf, c0, std::min(mc, iter_cols - c0),
                                o.eps, st));
    for (int c0 = 0; c0 < all_cols; c0 += mc)
        TICK_CK(fft_backward_tab(ps.plan, gs, ps.fb, ps.d_fr, ps.d_colf, c0, std::min(mc, all_cols - c0), st));
    for (size_t i = 0; i < ps.ran_iter.size(); ++i) {
        Job* j = ps.ran_iter[i];
        const Geo& g = j->g;
        TICK_CK(launch_exact_bwd_dev(j->low, j->n_low, j->rimg, ps.psf, g, j->xcm, st));
        TICK_CK(launch_update_cm(j->vcm[j->cur], j->vcm[j->cur ^ 1], j->xcm, j->invcm, g, 1, j->mip,
                                 j->flux_part, st));
        TICK_CK(launch_metric(j->mip, j->cosW, j->cosH, g.H, g.W, j->XS, j->YS, o.l2_over_region, j->G,
                              j->rowE2, j->coef, j->flux_part, j->nflux, ps.d_hist + i, ps.d_hist + mf + i,
                              st, 1, 1));
    }
    // 3b. new frames: low-sensitivity list, exact H^T 1 there, 1 / H^T 1
    for (Job* j : ps.ran_new) {
        const Geo& g = j->g;
        const int64_t vox = (int64_t)g.C * g.Ly * g.Lx;
        TICK_CK(launch_low_list(j->xcm, vox, kLowSensitivity, j->mx, j->low, j->n_low, st));
        TICK_CK(launch_exact_bwd_dev(j->low, j->n_low, nullptr, ps.psf, g, j->xcm, st));
        TICK_CK(launch_inv_cm(j->xcm, vox, j->invcm, st));
    }
    // 4. entropy and flux to the host, then the event
    const size_t ni = ps.ran_iter.size();
    if (ni > 0) {
        TICK_CK(cudaMemcpyAsync(ps.h_hist, ps.d_hist, ni * sizeof(double), cudaMemcpyDeviceToHost, st));
        TICK_CK(cudaMemcpyAsync(ps.h_hist + mf, ps.d_hist + mf, ni * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    }
    TICK_CK(cudaEventRecord(ps.ev, st));
    ps.tick_cols = iter_cols;
    return std::string();
}

// Starts a tick of the set: swaps its lists in under the lock, issues the
// launches with the lock released (client threads may submit, poll and
// cancel meanwhile), then takes the lock back for the bookkeeping.
void enqueue_tick(lfd_server* s, PsfSet& ps, std::unique_lock<std::mutex>& lk) {
    ps.ran_fin.swap(ps.finishing);
    ps.ran_iter = ps.iter;
    ps.ran_new.swap(ps.fresh);
    lk.unlock();
    const std::string why = launch_tick(s, ps);
    lk.lock();
    if (!why.empty()) {
        fail_set(s, ps, why.rfind("more frames", 0) == 0 ? LFD_EINTERNAL : LFD_ECUDA, why);
        return;
    }
    ps.busy = true;
    ++s->stats.ticks;
    s->stats.columns += ps.tick_cols;
}

void admit(lfd_server* s) {
    const int mf = s->opt.max_frames_per_set;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Job* j = *it;
        PsfSet& ps = *s->sets[j->set];
        // frames of the set: iterating, started by the tick in flight, waiting to start
        if ((int)(ps.iter.size() + ps.ran_new.size() + ps.fresh.size()) >= mf) {
            ++it;
            continue;
        }
        const int64_t off = s->arena.alloc(j->bytes);
        if (off < 0) break;  // first come, first served: wait for memory
        j->off = off;
        job_layout(j, s->arena.base + off);
        j->state = JobState::New;
        j->t_admit = Clock::now();
        ps.fresh.push_back(j);
        ++s->stats.admitted;
        it = s->queue.erase(it);
    }
}

void scheduler(lfd_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progressed = false;
        for (auto& up : s->sets) {
            PsfSet& ps = *up;
            if (!ps.busy) continue;
            const cudaError_t q = cudaEventQuery(ps.ev);
            if (q == cudaErrorNotReady) {
                // "not ready" is recorded as the thread's last error; clear it
                // so the next launch check (cudaGetLastError) does not see it
                cudaGetLastError();
                continue;
            }
            if (q != cudaSuccess) {
                fail_set(s, ps, LFD_ECUDA, std::string("tick: ") + cudaGetErrorString(q));
            } else {
                complete_tick(s, ps);
            }
            progressed = true;
        }
        if (s->stop)
            while (!s->queue.empty()) {  // cancel what has not started
                Job* j = s->queue.front();
                s->queue.pop_front();
                ++s->stats.cancelled;
                finish_job(s, j, LFD_ECANCELED);
            }
        if (s->arena.base) admit(s);
        bool any_work = false;
        for (size_t si = 0; si < s->sets.size(); ++si) {  // (sets are fixed once requests arrive)
            PsfSet& ps = *s->sets[si];
            const bool work = !ps.iter.empty() || !ps.fresh.empty() || !ps.finishing.empty();
            any_work = any_work || work || ps.busy;
            if (!ps.busy && work) {
                enqueue_tick(s, ps, lk);
                progressed = true;
            }
        }
        if (s->stop && !any_work && s->queue.empty()) break;
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
}

lfd_status add_psf(lfd_server* s, const float* psf, int P, int N, int Nz, int maxH, int maxW, int* set_id) {
    const lfd_options& o = s->opt.opt;
    Geo g{};
    std::string why;
    if (!make_geo(P, N, Nz, maxH, maxW, &g, &why)) {
        s->err = why;
        return LFD_EINVAL;
    }
    auto ps = std::make_unique<PsfSet>();
    ps->gmax = g;
    // tensor-core contraction: split BF16 (three products per term) or BF16
    // PSF spectra (two); FP32 runs on the CUDA cores
    const int products = o.precision == LFD_BF16X3 ? 3 : o.precision == LFD_BF16 ? 2 : 0;
    if (!fft_plan_for(g, &ps->plan, o.fft_size, std::max(1, s->opt.max_frames_per_set / 8), products)) {
        s->err = "no FFT tiling fits this PSF / sensor shape";
        return LFD_EUNSUPPORTED;
    }
    const FftPlan& p = ps->plan;
    const bool split = products != 0;  // tensor-core planes and contraction
    if (split) {
        int major = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, s->device);
        if (major != 10) {
            s->err = "the tensor-core FFT contraction needs an sm_10x (Blackwell) device";
            return LFD_EUNSUPPORTED;
        }
    }
    const int mf = s->opt.max_frames_per_set, ncolp = s->opt.max_cols;
    ps->max_tiles = p.ntile;
    if (lfd_region_size(N, maxH, maxW, o.dML_um, o.Q, o.NA, o.lambda_um, &ps->XSmax, &ps->YSmax) != LFD_OK)
        return LFD_EINVAL;
    if (o.XS > 0) ps->XSmax = o.XS;
    if (o.YS > 0) ps->YSmax = o.YS;
    ps->tab_stride = (int64_t)ps->XSmax * maxW + (int64_t)ps->YSmax * maxH;
#define ADD_CK(call)                                                             \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            s->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return e_ == cudaErrorMemoryAllocation ? LFD_ENOMEM : LFD_ECUDA;     \
        }                                                                        \
    } while (0)
    ADD_CK(cudaStreamCreateWithFlags(&ps->st, cudaStreamNonBlocking));
    ADD_CK(cudaEventCreateWithFlags(&ps->ev, cudaEventDisableTiming));
    const int64_t psf_count = (int64_t)Nz * N * N * P * P;
    ADD_CK(ps->dev(&ps->psf, psf_count));
    ADD_CK(cudaMemcpyAsync(ps->psf, psf, sizeof(float) * psf_count, cudaMemcpyDefault, ps->st));
    FftBuffers& b = ps->fb;
    b.ncolp = ncolp;
    if (split) {
        for (int i = 0; i < 4; ++i)
            if (products == 3 || i % 2 == 0)  // BF16 spectra: hi planes only
                ADD_CK(ps->dev(&b.Wp[i], (int64_t)p.bins * g.S * p.Cw));
        // the four data planes of each 8-channel group side by side (one block)
        ADD_CK(ps->dev(&b.Xp[0], 4 * (int64_t)p.bins * ncolp * p.Cw));
        ADD_CK(ps->dev(&b.Yp[0], 4 * (int64_t)p.bins * ncolp * p.Sw));
        for (int i = 1; i < 4; ++i) {
            b.Xp[i] = b.Xp[0] + (int64_t)i * ncolp * p.bins * 8;
            b.Yp[i] = b.Yp[0] + (int64_t)i * ncolp * p.bins * 8;
        }
    } else {
        ADD_CK(ps->dev(&b.Wf, (int64_t)p.bins * g.S * p.Cf));
    }
    ADD_CK(ps->dev(&b.Xh, (int64_t)p.bins * ncolp * p.Cf));
    ADD_CK(ps->dev(&b.Yh, (int64_t)p.bins * ncolp * p.Sf));
    {  // PSF spectra from the packed taps (freed afterwards)
        float* W32 = nullptr;
        ADD_CK(cudaMalloc((void**)&W32, sizeof(float) * (size_t)g.taps() * g.Spad * g.Cpad));
        cudaError_t e = launch_repack_psf(ps->psf, g, W32, nullptr, nullptr, ps->st);
        if (e == cudaSuccess) e = fft_init(p, g, W32, b, ps->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ps->st);
        cudaFree(W32);
        ADD_CK(e);
    }
    if (split) {
        CgemmBuffers cb{};
        cb.bins = p.bins;
        cb.ntile = p.ntile;
        cb.ncolp = ncolp;
        cb.max_cols = o.contraction_cols;
        cb.S = g.S;
        cb.C = g.C;
        cb.Sw = p.Sw;
        cb.Cw = p.Cw;
        cb.Sf = p.Sf;
        cb.Cf = p.Cf;
        for (int i = 0; i < 4; ++i) cb.W[i] = b.Wp[i];
        cb.X = b.Xp[0];
        cb.Y = b.Yp[0];
        cb.Yout = b.Yh;
        cb.Xout = b.Xh;
        if (products == 3 && o.spectra_lo_tau > 0.f) {
            // adaptive lo planes: keep the tiles that matter, free the full lo planes
            ADD_CK(cgemm_compact_lo(cb, o.spectra_lo_tau, ps->st, &ps->lo, &ps->resident));
            for (int i : {1, 3}) {
                ps->owned.erase(std::find(ps->owned.begin(), ps->owned.end(), (void*)b.Wp[i]));
                cudaFree(b.Wp[i]);
                ps->resident -= (int64_t)p.bins * g.S * p.Cw * (int64_t)sizeof(__nv_bfloat16);
                b.Wp[i] = nullptr;
                cb.W[i] = nullptr;
            }
            cb.lo = ps->lo;
        }
        std::string why2;
        const cudaError_t ce = cgemm_init(cb, s->sm_count, &b.cg, &why2);
        if (ce != cudaSuccess) {
            s->err = "cgemm_init: " + (why2.empty() ? std::string(cudaGetErrorString(ce)) : why2);
            return LFD_ECUDA;
        }
    }
    ADD_CK(ps->dev(&ps->d_fr, mf));
    ADD_CK(ps->dev(&ps->d_colf, (int64_t)mf * ps->max_tiles));
    ADD_CK(ps->dev(&ps->d_hist, 2LL * mf));
    ADD_CK(cudaMallocHost((void**)&ps->h_fr, sizeof(FrameCols) * mf));
    ADD_CK(cudaMallocHost((void**)&ps->h_colf, sizeof(int) * (size_t)mf * ps->max_tiles));
    ADD_CK(cudaMallocHost((void**)&ps->h_hist, sizeof(double) * 2 * mf));
    ADD_CK(cudaMallocHost((void**)&ps->h_tab, sizeof(double) * (size_t)mf * ps->tab_stride));
#undef ADD_CK
    *set_id = (int)s->sets.size();
    s->stats.resident_bytes += ps->resident;
    s->sets.push_back(std::move(ps));
    return LFD_OK;
}

}  // namespace

extern "C" {

void lfd_server_default_options(lfd_server_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    lfd_default_options(&o->opt);
    o->opt.precision = LFD_BF16X3;
    o->opt.variant = LFD_FFT;
    o->arena_bytes = 0;
    o->max_frames_per_set = 32;
    o->max_cols = 128;
    o->max_queue = 4096;
    o->max_iter = 40;
}

lfd_status lfd_server_create(const lfd_server_options* opt_in, lfd_server** out) {
    if (!out) return LFD_EINVAL;
    *out = nullptr;
    lfd_server_options o;
    if (opt_in) o = *opt_in; else lfd_server_default_options(&o);
    if (o.opt.contraction_cols != 0 && o.opt.contraction_cols != 16 && o.opt.contraction_cols != 32 &&
        o.opt.contraction_cols != 64)
        return LFD_EINVAL;
    if (o.opt.precision != LFD_FP32 && o.opt.precision != LFD_BF16 && o.opt.precision != LFD_BF16X3)
        return LFD_EINVAL;
    if (!(o.opt.eps >= 0.f)) return LFD_EINVAL;
    if (o.opt.fft_size != 0 && o.opt.fft_size != 32 && o.opt.fft_size != 64) return LFD_EINVAL;
    if (o.max_frames_per_set < 1 || o.max_frames_per_set > 1024) return LFD_EINVAL;
    if (o.max_cols < 16 || o.max_cols > 4096 || o.max_cols % 16 != 0) return LFD_EINVAL;
    if (o.max_queue < 1 || o.max_iter < 1 || o.arena_bytes < 0) return LFD_EINVAL;
    o.opt.variant = LFD_FFT;
    lfd_server* s = new (std::nothrow) lfd_server();
    if (!s) return LFD_ENOMEM;
    s->opt = o;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return LFD_ECUDA;
    }
    try {
        s->thr = std::thread(scheduler, s);
    } catch (...) {
        delete s;
        return LFD_ENOMEM;
    }
    *out = s;
    return LFD_OK;
}

lfd_status lfd_server_add_psf(lfd_server* s, const float* psf, int P, int Nnum, int Nz, int max_H, int max_W,
                              int* set_id) {
    if (!s || !psf || !set_id) return LFD_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) {
        s->err = "PSF sets are added before the first submit";
        return LFD_EBUSY;
    }
    cudaSetDevice(s->device);
    return add_psf(s, psf, P, Nnum, Nz, max_H, max_W, set_id);
}

lfd_status lfd_submit(lfd_server* s, const lfd_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return LFD_EINVAL;
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return LFD_ENOMEM;
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->stats.submitted;
    auto reject = [&](lfd_status st, const char* why) {
        ++s->stats.rejected;
        s->err = why;
        return st;
    };
    if (r->set_id < 0 || r->set_id >= (int)s->sets.size()) return reject(LFD_EINVAL, "unknown PSF set");
    if (!r->y || !r->v_out) return reject(LFD_EINVAL, "NULL y or v_out");
    if (r->max_iter < 0) return reject(LFD_EINVAL, "max_iter < 0");
    PsfSet& ps = *s->sets[r->set_id];
    const Geo& gs = ps.gmax;
    if (r->H > gs.H || r->W > gs.W) return reject(LFD_EINVAL, "frame larger than the set's maximum");
    j->req = *r;
    j->set = r->set_id;
    std::string why;
    if (!make_geo(gs.P, gs.N, gs.Nz, r->H, r->W, &j->g, &why)) return reject(LFD_EINVAL, "H, W not multiples of Nnum");
    const lfd_options& o = s->opt.opt;
    if (o.XS > 0 && o.YS > 0) {
        j->XS = o.XS;
        j->YS = o.YS;
    } else if (lfd_region_size(gs.N, r->H, r->W, o.dML_um, o.Q, o.NA, o.lambda_um, &j->XS, &j->YS) != LFD_OK) {
        return reject(LFD_EINVAL, "region size");
    }
    if (j->XS > r->W || j->YS > r->H) return reject(LFD_EINVAL, "XS / YS larger than the frame");
    j->tiles_x = (j->g.Lx + ps.plan.B - 1) / ps.plan.B;
    j->ntile = j->tiles_x * ((j->g.Ly + ps.plan.B - 1) / ps.plan.B);
    j->max_iter = r->max_iter > 0 ? r->max_iter : s->opt.max_iter;
    j->nflux = update_cm_blocks(j->g);
    j->bytes = job_layout(j.get(), nullptr);
    if (!s->started) {
        size_t fr = 0, tot = 0;
        cudaSetDevice(s->device);
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return reject(LFD_ECUDA, "cudaMemGetInfo failed");
        }
        int64_t want = s->opt.arena_bytes > 0 ? s->opt.arena_bytes : (int64_t)(0.85 * (double)fr);
        want &= ~(int64_t)255;
        if (s->arena.init(want) != cudaSuccess) {
            cudaGetLastError();
            return reject(LFD_ENOMEM, "arena allocation failed");
        }
        s->stats.arena_bytes = want;
        s->started = true;
    }
    if (j->bytes > s->arena.cap) return reject(LFD_ENOMEM, "the frame alone needs more than the arena");
    if ((int)s->queue.size() >= s->opt.max_queue) return reject(LFD_EBUSY, "queue full");
    j->y_dev = device_ptr(r->y);
    j->v_dev = device_ptr(r->v_out);
    j->ticket = s->next_ticket++;
    j->t_submit = Clock::now();
    *ticket = j->ticket;
    Job* jp = j.release();
    s->jobs[jp->ticket] = jp;
    s->queue.push_back(jp);
    s->cv_work.notify_one();
    return LFD_OK;
}

lfd_status lfd_poll(lfd_server* s, uint64_t ticket, int64_t timeout_us, lfd_result* res) {
    if (!s) return LFD_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return LFD_EINVAL;
    Job* j = it->second;
    auto done = [&] { return j->state == JobState::Done; };
    if (!done()) {
        if (timeout_us == 0) return LFD_ENOTREADY;
        if (timeout_us < 0) {
            s->cv_done.wait(lk, done);
        } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
            return LFD_ETIMEDOUT;
        }
    }
    if (res) {
        res->status = j->status;
        res->iters_done = j->done;
        res->iters_run = j->ran;
        res->predicted = j->ran > 0 ? lfd_predict_stop(j->E.data(), j->ran) : 0;
        const auto us = [](Clock::duration d) {
            return (int64_t)std::chrono::duration_cast<std::chrono::microseconds>(d).count();
        };
        res->queue_us = j->status == LFD_ECANCELED ? -1 : us(j->t_admit - j->t_submit);
        res->latency_us = us(j->t_done - j->t_submit);
    }
    s->jobs.erase(ticket);
    delete j;
    return LFD_OK;
}

lfd_status lfd_cancel(lfd_server* s, uint64_t ticket) {
    if (!s) return LFD_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return LFD_EINVAL;
    Job* j = it->second;
    if (j->state != JobState::Queued) return LFD_EBUSY;
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), j));
    ++s->stats.cancelled;
    finish_job(s, j, LFD_ECANCELED);
    return LFD_OK;
}

lfd_status lfd_server_stats_get(const lfd_server* cs, lfd_server_stats* out) {
    if (!cs || !out) return LFD_EINVAL;
    lfd_server* s = const_cast<lfd_server*>(cs);
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->arena_bytes = s->arena.cap;
    out->arena_peak_bytes = s->arena.fl.peak;
    out->queued = (int)s->queue.size();
    int inflight = 0;
    for (auto& ps : s->sets)
        inflight += (int)(ps->iter.size() + ps->fresh.size() + ps->finishing.size() + ps->ran_fin.size());
    out->in_flight = inflight;
    return LFD_OK;
}

// The scheduler thread may replace s->err at any time, so the message is
// copied under the server's lock into a buffer of the calling thread; the
// pointer stays valid until this thread's next call.
const char* lfd_server_last_error(const lfd_server* s) {
    if (!s) return "NULL server";
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(s->mu);
    copy = s->err;
    return copy.c_str();
}

void lfd_server_destroy(lfd_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->thr.joinable()) s->thr.join();
    for (auto& ps : s->sets)
        if (ps->st) cudaStreamSynchronize(ps->st);
    for (auto& kv : s->jobs) delete kv.second;
    s->jobs.clear();
    s->sets.clear();
    delete s;
}

}  // extern "C"
