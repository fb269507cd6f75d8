// server.cu -- continuous-batching solve server (amg_server_*).
//
// One worker thread owns the device work.  Each registered hierarchy has a
// K-column batch (K = batch width >= max_batch) on its own stream and moves
// through its own cycle -- admit queued requests into free columns, one PCG
// iteration, and when some column's recurrence residual reached its
// tolerance (or its iteration budget) the true-residual check -- driven by
// polling its stream's completion event.  Hierarchies do not wait for one
// another: a small hierarchy runs many iterations while a large one runs one,
// and while the worker admits or retires requests of one hierarchy the
// others keep the device busy.  The batch workspace is allocated on first
// use, within the memory budget, and released when the hierarchy goes idle.
// A column's arithmetic does not depend on the other columns, so a request's
// result is the same alone and in any mix.
//
// Host copies stay off the worker: submit uploads the right-hand side into a
// device buffer of the request (from a staging pool with its own budget) and
// wait downloads the result from another, so admitting a request is a
// device-side scatter and retiring one a device-side gather, both queued on
// the hierarchy's stream without a host wait.  When the staging budget is
// used up (or set to none), a request goes through the worker's pinned host
// buffer instead, as a synchronous copy.
//
// Every wait of the worker for device work -- an iteration, a residual
// check, a host staging copy -- polls an event with the limit
// opt.wait_limit_ms.  When one runs out the worker stops and every request
// not yet finished ends with AMG_TIMEOUT.  The copies between the caller's
// memory and the device in submit and wait run to completion before those
// calls return: the caller may free that memory afterwards.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "batch_ops.cuh"
#include "hierarchy.cuh"

namespace amg {
void set_last_error(const std::string &msg);
}

using namespace amg;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket = 0;
    int hid = 0;
    int32_t n = 0;
    std::vector<double> b, x;  // host copies: host staging, or the zero solution
    double *d_b = nullptr;     // the right-hand side staged on the device at submit
    double *d_x = nullptr;     // the result staged on the device at retirement
    int64_t staged = 0;        // staging bytes the request holds
    cudaEvent_t ev = nullptr;  // upload at submit, then the result's gather
    double tol = 1e-8;
    double bnorm = 0.0;
    amg_solve_info info{};
    int status = AMG_NOT_CONVERGED;
    bool done = false;
    bool has_result = false;   // x (host or d_x) holds the solution
    Clock::time_point submitted;
};

struct Slot {
    Request *req = nullptr;
    int its = 0, reps = 0;
    double rnorm = 0.0;
    bool out_of_budget = false;  // retire as not converged after the residual check
};

// where a hierarchy is in its cycle
enum Phase { kIdle = 0, kIter = 1, kResid = 2 };

struct HState {
    Hierarchy *h = nullptr;
    int32_t n = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    BatchWS *ws = nullptr;
    int64_t ws_bytes = 0;
    std::vector<Slot> slots;
    std::deque<Request *> queue;
    DevBuf dstage;          // n doubles: admission / retirement staging
    double *hstage = nullptr;  // pinned n doubles
    cudaEvent_t copy_ev = nullptr;  // host staging copies
    Phase phase = kIdle;
    Clock::time_point launched_at;
};

}  // namespace

struct amg_server {
    amg_server_opts opt{};
    int K = 8;
    std::vector<std::unique_ptr<HState>> hs;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::thread worker;
    bool stop = false;
    int64_t queued = 0;
    uint64_t next_ticket = 1;
    int64_t budget = 0, in_use = 0;
    int device = 0;
    std::string fatal;
    int fatal_status = AMG_ERR_CUDA;
    // device staging of requests (submit uploads, wait downloads)
    cudaMemPool_t pool = nullptr;
    cudaStream_t io = nullptr;
    int64_t stage_cap = 0;
    std::atomic<int64_t> staged{0};
};

namespace {

// the calling thread works on the server's device for the guard's lifetime
struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&old) != cudaSuccess) old = -1;
        if (old != dev) AMG_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
    }
};

// Waits for `ev` by polling it, at most opt.wait_limit_ms (AMG_TIMEOUT).
void poll_event(const amg_server *S, cudaEvent_t ev, const char *what) {
    const auto t0 = Clock::now();
    while (true) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return;
        if (e != cudaErrorNotReady) throw Error(AMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        if (std::chrono::duration<double, std::milli>(Clock::now() - t0).count() > (double)S->opt.wait_limit_ms)
            throw Error(AMG_TIMEOUT, std::string(what) + " ran past the server's wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Waits, bounded, for the work queued on `s` so far (host staging copies).
void poll_stream(const amg_server *S, cudaStream_t s, cudaEvent_t ev, const char *what) {
    AMG_CUDA(cudaEventRecord(ev, s));
    poll_event(S, ev, what);
}

// Stream-ordered allocation of `bytes` from the staging pool, within the
// staging budget; nullptr when the budget or the pool has no room (the
// request then goes through host staging).
double *stage_alloc(amg_server *S, int64_t bytes, cudaStream_t s) {
    if (!S->pool) return nullptr;
    if (injected_allocation_failure()) return nullptr;  // as a full pool
    int64_t cur = S->staged.load();
    do {
        if (cur + bytes > S->stage_cap) return nullptr;
    } while (!S->staged.compare_exchange_weak(cur, cur + bytes));
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, (size_t)bytes, S->pool, s) != cudaSuccess) {
        (void)cudaGetLastError();  // an allocation failure is not sticky
        S->staged -= bytes;
        return nullptr;
    }
    return static_cast<double *>(p);
}

// free a staged buffer of the request, stream-ordered on `s`
void stage_free(amg_server *S, Request *r, double *&p, cudaStream_t s) {
    if (!p) return;
    const int64_t bytes = (int64_t)sizeof(double) * r->n;
    AMG_CUDA(cudaFreeAsync(p, s));
    p = nullptr;
    r->staged -= bytes;
    S->staged -= bytes;
}

// the device resources of a request that leaves the server (no throw)
void drop_request(amg_server *S, Request *r) {
    for (double **p : {&r->d_b, &r->d_x})
        if (*p) cudaFreeAsync(*p, S->io);
    r->d_b = r->d_x = nullptr;
    S->staged -= r->staged;
    r->staged = 0;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
}

int64_t batch_bytes(const Hierarchy &h, int K) {
    int64_t xb = h.opt.precision == AMG_PREC_FP64 ? 8 : 4;
    int64_t cyc = 0;
    for (int l = 0; l < h.nlev(); ++l) cyc += 4 * xb * (int64_t)h.lev[l]->n() * K;
    int64_t n0 = h.lev[0]->n();
    int64_t pcg = 7 * 8 * n0 * K + (xb == 4 ? (h.nlev() == 1 ? 2 : 1) * 4 * n0 * K : 0);
    return cyc + pcg + (1 << 20);
}

void finish_request(amg_server *S, HState &H, int c, int status, double tt) {
    Slot &sl = H.slots[c];
    Request *r = sl.req;
    BatchWS &w = *H.ws;
    const int64_t bytes = (int64_t)sizeof(double) * H.n;
    // X column -> a device buffer of the request, which wait copies to the
    // caller; the column slot can take a new request right behind the gather
    double *dx = stage_alloc(S, bytes, H.stream);
    std::vector<double> x;
    if (dx) {
        bat::gather_column(H.n, w.K, c, w.X.as<double>(), dx, H.stream);
        AMG_CUDA(cudaEventRecord(r->ev, H.stream));
    } else {  // host staging
        bat::gather_column(H.n, w.K, c, w.X.as<double>(), H.dstage.as<double>(), H.stream);
        AMG_CUDA(cudaMemcpyAsync(H.hstage, H.dstage.ptr, bytes, cudaMemcpyDeviceToHost, H.stream));
        poll_stream(S, H.stream, H.copy_ev, "result download (host staging)");
        x.assign(H.hstage, H.hstage + H.n);  // outside the lock: clients keep submitting and waiting
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (dx) {
        r->d_x = dx;
        r->staged += bytes;
    } else {
        r->x = std::move(x);
    }
    r->status = status;
    r->has_result = true;
    r->info.iterations = sl.its;
    r->info.replacements = sl.reps;
    r->info.status = status;
    r->info.final_relres = r->bnorm > 0 ? std::sqrt(tt) / r->bnorm : 0.0;
    r->info.conv_factor = sl.its > 0 && r->bnorm > 0 ? std::pow(sl.rnorm / r->bnorm, 1.0 / sl.its) : 0.0;
    r->info.solve_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->submitted).count();
    r->done = true;
    sl = Slot();
    w.h_active()[c] = 0;
    S->cv_done.notify_all();
}

// admit queued requests into free columns of one hierarchy (worker thread)
bool admit(amg_server *S, HState &H) {
    std::vector<std::pair<int, Request *>> adm;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (H.queue.empty()) return false;
        if (!H.ws) {
            int64_t need = batch_bytes(*H.h, S->K);
            if (S->in_use + need > S->budget) return false;  // wait for memory
            H.ws_bytes = need;
            S->in_use += need;
        }
        for (int c = 0; c < S->K && !H.queue.empty(); ++c) {
            if (H.slots[c].req) continue;
            adm.push_back({c, H.queue.front()});
            H.queue.pop_front();
            S->queued--;
        }
    }
    if (!H.ws) {
        try {
            H.ws = &batch_workspace(*H.h, S->K, H.stream);
        } catch (const Error &e) {
            if (e.status != AMG_ERR_OOM) throw;
            std::lock_guard<std::mutex> lk(S->mu);  // no memory now: requeue in order
            for (auto it = adm.rbegin(); it != adm.rend(); ++it) H.queue.push_front(it->second);
            S->queued += (int64_t)adm.size();
            S->in_use -= H.ws_bytes;
            H.ws_bytes = 0;
            return false;
        }
        for (int c = 0; c < S->K; ++c) H.ws->h_active()[c] = 0;
    }
    BatchWS &w = *H.ws;
    // only the columns admitted now restart (beta = 0); running columns go on
    for (int c = 0; c < S->K; ++c) w.h_start()[c] = 0;
    for (auto &a : adm) {
        int c = a.first;
        Request *r = a.second;
        const double *src = r->d_b;
        if (!src) {  // host staging
            std::memcpy(H.hstage, r->b.data(), sizeof(double) * H.n);
            AMG_CUDA(cudaMemcpyAsync(H.dstage.ptr, H.hstage, sizeof(double) * H.n, cudaMemcpyHostToDevice, H.stream));
            src = H.dstage.as<double>();
        }
        bat::scatter_column(H.n, w.K, c, src, w.B.as<double>(), H.stream);
        bat::scatter_column(H.n, w.K, c, src, w.R.as<double>(), H.stream, w.R32.as<float>());
        bat::zero_column(H.n, w.K, c, w.X.as<double>(), H.stream);
        bat::zero_column(H.n, w.K, c, w.P.as<double>(), H.stream);
        bat::zero_column(H.n, w.K, c, w.Q.as<double>(), H.stream);
        if (r->d_b) {
            stage_free(S, r, r->d_b, H.stream);  // after the scatters, in stream order
        } else {
            poll_stream(S, H.stream, H.copy_ev, "right-hand side upload (host staging)");  // the buffers are reused
            std::vector<double>().swap(r->b);
        }
        H.slots[c].req = r;
        H.slots[c].its = H.slots[c].reps = 0;
        H.slots[c].rnorm = r->bnorm;
        w.h_active()[c] = 1;
        w.h_start()[c] = 1;
    }
    if (!adm.empty()) batch_push_flags(w, H.stream);
    return !adm.empty();
}

void release_if_idle(amg_server *S, HState &H) {
    if (!H.ws) return;
    for (auto &sl : H.slots)
        if (sl.req) return;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!H.queue.empty()) return;
    H.h->batch.erase(S->K);
    H.ws = nullptr;
    S->in_use -= H.ws_bytes;
    H.ws_bytes = 0;
}

// the worker stops: every request not yet finished ends with `status`
void fail_all(amg_server *S, const std::string &msg, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = msg;
    S->fatal_status = status;
    for (auto &kv : S->reqs) {
        Request *r = kv.second.get();
        if (!r->done) {
            r->done = true;
            r->status = status;
            r->info.status = status;
        }
    }
    for (auto &H : S->hs) {
        H->queue.clear();
        for (auto &sl : H->slots) sl = Slot();
    }
    S->queued = 0;
    S->cv_done.notify_all();
}

bool has_live(const HState &H) {
    for (auto &sl : H.slots)
        if (sl.req) return true;
    return false;
}

// admit, then one iteration if any column is live (else idle)
void start_iteration(amg_server *S, HState &H) {
    admit(S, H);
    if (!H.ws || !has_live(H)) {
        H.phase = kIdle;
        release_if_idle(S, H);
        return;
    }
    batch_iteration(*H.h, *H.ws, H.stream);
    AMG_CUDA(cudaEventRecord(H.done_ev, H.stream));
    H.phase = kIter;
    H.launched_at = Clock::now();
}

// an iteration finished: retire broken-down columns, flag candidates and
// columns out of budget for the true-residual check, or go on
void after_iteration(amg_server *S, HState &H) {
    BatchWS &w = *H.ws;
    bool check = false, changed = false;
    for (int c = 0; c < S->K; ++c) {
        Slot &sl = H.slots[c];
        if (!sl.req || !w.h_active()[c]) continue;
        sl.its++;
        const double pq = w.h_pq()[c], rho = w.h_rho()[c], rr = w.h_rr()[c];
        w.h_mask()[c] = 0;
        if (!(pq > 0.0) || !(rho > 0.0) || !std::isfinite(rr)) {
            finish_request(S, H, c, AMG_BREAKDOWN, rr);
            changed = true;
            continue;
        }
        sl.rnorm = std::sqrt(rr);
        if (sl.rnorm <= sl.req->tol * sl.req->bnorm) {
            w.h_mask()[c] = 1;
            check = true;
        } else if (sl.its >= S->opt.max_it) {
            sl.out_of_budget = true;
            check = true;
        }
    }
    if (changed) {
        for (int c = 0; c < S->K; ++c) w.h_start()[c] = 0;
        batch_push_flags(w, H.stream);
    }
    if (check) {
        batch_true_residual(*H.h, w, H.stream);
        AMG_CUDA(cudaEventRecord(H.done_ev, H.stream));
        H.phase = kResid;
        H.launched_at = Clock::now();
        return;
    }
    start_iteration(S, H);
}

// the true residuals are in: retire converged and out-of-budget columns,
// replace the residual of the others, then go on
void after_residual(amg_server *S, HState &H) {
    BatchWS &w = *H.ws;
    bool replace = false, changed = false;
    for (int c = 0; c < S->K; ++c) {
        Slot &sl = H.slots[c];
        if (!sl.req) continue;
        const double tt = w.h_tt()[c];
        if (w.h_mask()[c]) {
            const double tn = std::sqrt(tt);
            sl.rnorm = tn;
            if (tn <= sl.req->tol * sl.req->bnorm) {
                w.h_mask()[c] = 0;
                finish_request(S, H, c, AMG_OK, tt);
                changed = true;
                continue;
            }
            sl.reps++;
            replace = true;
        }
        if (sl.req && sl.out_of_budget) {
            w.h_mask()[c] = 0;
            finish_request(S, H, c, AMG_NOT_CONVERGED, tt);
            changed = true;
        }
    }
    if (replace) {
        AMG_CUDA(cudaMemcpyAsync(w.mask.ptr, w.h_mask(), sizeof(int) * w.K, cudaMemcpyHostToDevice, H.stream));
        bat::copy_masked_columns(H.n, w.K, w.T.as<double>(), w.R.as<double>(), w.mask.as<int>(), H.stream,
                                 w.R32.as<float>());
    }
    for (int c = 0; c < S->K; ++c) w.h_mask()[c] = 0;
    if (changed) {
        for (int c = 0; c < S->K; ++c) w.h_start()[c] = 0;
        batch_push_flags(w, H.stream);
    }
    start_iteration(S, H);
}

void worker_loop(amg_server *S) {
    cudaSetDevice(S->device);
    try {
        while (true) {
            bool queued;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                queued = S->queued > 0;
                bool busy = queued;
                for (auto &H : S->hs) busy |= H->phase != kIdle || has_live(*H);
                if (S->stop && !busy) break;
                if (!busy) {
                    S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                    continue;
                }
            }
            bool progressed = false;
            for (auto &Hp : S->hs) {
                HState &H = *Hp;
                if (H.phase == kIdle) {
                    bool waiting;
                    {
                        std::lock_guard<std::mutex> lk(S->mu);
                        waiting = !H.queue.empty();
                    }
                    if (waiting || has_live(H)) {
                        start_iteration(S, H);
                        progressed |= H.phase != kIdle;
                    }
                    continue;
                }
                const cudaError_t e = cudaEventQuery(H.done_ev);
                if (e == cudaErrorNotReady) {
                    if (std::chrono::duration<double, std::milli>(Clock::now() - H.launched_at).count() >
                        (double)S->opt.wait_limit_ms)
                        throw Error(AMG_TIMEOUT, H.phase == kIter ? "a batch iteration ran past the wait limit"
                                                                  : "a residual check ran past the wait limit");
                    continue;
                }
                if (e != cudaSuccess) throw Error(AMG_ERR_CUDA, std::string("stream failed: ") + cudaGetErrorString(e));
                progressed = true;
                if (H.phase == kIter) after_iteration(S, H);
                else after_residual(S, H);
            }
            if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    } catch (const Error &e) {
        fail_all(S, e.what(), e.status == AMG_TIMEOUT ? AMG_TIMEOUT : AMG_ERR_CUDA);
    } catch (const std::exception &e) {
        fail_all(S, e.what(), AMG_ERR_CUDA);
    }
}

}  // namespace

extern "C" {

void amg_server_opts_default(amg_server_opts *o) {
    if (!o) return;
    o->max_batch = 32;
    o->hbm_budget = 0;
    o->max_queue = 4096;
    o->max_it = 500;
    o->stage_budget = 0;
    o->wait_limit_ms = 120000;
}

amg_status amg_server_create(const amg_server_opts *o, amg_server **out) {
    try {
        set_last_error("");
        if (!out) { set_last_error("out is NULL"); return AMG_ERR_INVALID; }
        *out = nullptr;
        amg_server_opts opt;
        if (o) opt = *o; else amg_server_opts_default(&opt);
        if (opt.max_batch < 1 || opt.max_batch > 64 || opt.max_queue < 1 || opt.max_it < 1 || opt.hbm_budget < 0 ||
            opt.stage_budget < -1 || opt.wait_limit_ms < 1) {
            set_last_error("server options out of range (max_batch 1..64, max_queue >= 1, max_it >= 1, "
                           "hbm_budget >= 0, stage_budget >= -1, wait_limit_ms >= 1)");
            return AMG_ERR_INVALID;
        }
        auto S = std::make_unique<amg_server>();
        S->opt = opt;
        S->K = bat::batch_width(opt.max_batch);
        AMG_CUDA(cudaGetDevice(&S->device));
        if (opt.hbm_budget > 0) {
            S->budget = opt.hbm_budget;
        } else {
            size_t fr = 0, tot = 0;
            AMG_CUDA(cudaMemGetInfo(&fr, &tot));
            S->budget = (int64_t)(fr * 0.7);  // with the default staging quarter on top: 7/8 of free HBM
        }
        S->stage_cap = opt.stage_budget > 0 ? opt.stage_budget : opt.stage_budget == 0 ? S->budget / 4 : 0;
        AMG_CUDA(cudaStreamCreateWithFlags(&S->io, cudaStreamNonBlocking));
        if (S->stage_cap > 0) {
            cudaMemPoolProps pp{};
            pp.allocType = cudaMemAllocationTypePinned;
            pp.location.type = cudaMemLocationTypeDevice;
            pp.location.id = S->device;
            AMG_CUDA(cudaMemPoolCreate(&S->pool, &pp));
            uint64_t keep = (uint64_t)S->stage_cap;  // freed blocks stay with the pool up to the budget
            AMG_CUDA(cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        S->worker = std::thread(worker_loop, S.get());
        *out = S.release();
        return AMG_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return AMG_ERR_CUDA;
    }
}

// the CUDA objects of a hierarchy state that never joined the server
void drop_hstate(HState &H) {
    if (H.stream) cudaStreamSynchronize(H.stream);
    if (H.stream) cudaStreamDestroy(H.stream);
    if (H.done_ev) cudaEventDestroy(H.done_ev);
    if (H.copy_ev) cudaEventDestroy(H.copy_ev);
    if (H.hstage) cudaFreeHost(H.hstage);
    H.stream = nullptr;
    H.done_ev = H.copy_ev = nullptr;
    H.hstage = nullptr;
}

amg_status amg_server_register(amg_server *S, amg_hierarchy *h, int *hid) {
    set_last_error("");
    if (!S || !h || !hid) { set_last_error("NULL argument"); return AMG_ERR_INVALID; }
    auto H = std::make_unique<HState>();
    try {
        H->h = &h->h;
        H->n = h->h.lev[0]->n();
        H->slots.resize(S->K);
        AMG_CUDA(cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking));
        AMG_CUDA(cudaEventCreateWithFlags(&H->done_ev, cudaEventDisableTiming));
        AMG_CUDA(cudaEventCreateWithFlags(&H->copy_ev, cudaEventDisableTiming));
        H->dstage.alloc(sizeof(double) * (H->n + kPad));
        AMG_CUDA(cudaMallocHost(&H->hstage, sizeof(double) * (H->n + kPad)));
        ensure_workspace(h->h, H->stream);
        poll_stream(S, H->stream, H->copy_ev, "hierarchy workspace preparation");
        std::lock_guard<std::mutex> lk(S->mu);
        *hid = (int)S->hs.size();
        S->hs.push_back(std::move(H));
        return AMG_OK;
    } catch (const Error &e) {
        drop_hstate(*H);
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        drop_hstate(*H);
        set_last_error(e.what());
        return AMG_ERR_CUDA;
    }
}

amg_status amg_server_submit(amg_server *S, int hid, const double *b, double tol, uint64_t *ticket) {
    set_last_error("");
    if (!S || !b || !ticket) { set_last_error("NULL argument"); return AMG_ERR_INVALID; }
    if (!(tol > 0.0) || !std::isfinite(tol)) { set_last_error("tol must be > 0"); return AMG_ERR_INVALID; }
    auto r = std::make_unique<Request>();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (hid < 0 || hid >= (int)S->hs.size()) { set_last_error("unknown hierarchy id"); return AMG_ERR_INVALID; }
        if (!S->fatal.empty()) { set_last_error("server stopped: " + S->fatal); return (amg_status)S->fatal_status; }
        if (S->queued >= S->opt.max_queue) { set_last_error("queue full"); return AMG_REJECTED; }
        r->n = S->hs[hid]->n;
    }
    const int32_t n = r->n;
    double s2 = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        if (!std::isfinite(b[i])) { set_last_error("b has a non-finite value"); return AMG_ERR_INVALID; }
        s2 += b[i] * b[i];
    }
    r->bnorm = std::sqrt(s2);
    r->tol = tol;
    r->hid = hid;
    if (r->bnorm == 0.0) {  // x = 0 solves it
        r->x.assign(n, 0.0);
        r->done = true;
        r->has_result = true;
        r->status = AMG_OK;
    } else {
        try {
            DeviceGuard dg(S->device);
            AMG_CUDA(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
            const int64_t bytes = (int64_t)sizeof(double) * n;
            r->d_b = stage_alloc(S, bytes, S->io);
            if (r->d_b) {
                r->staged = bytes;
                AMG_CUDA(cudaMemcpyAsync(r->d_b, b, bytes, cudaMemcpyHostToDevice, S->io));
                AMG_CUDA(cudaEventRecord(r->ev, S->io));
                // runs to completion, unbounded: the device reads the caller's b, which
                // is the caller's again once submit returns
                AMG_CUDA(cudaEventSynchronize(r->ev));
            } else {
                r->b.assign(b, b + n);
            }
        } catch (const Error &e) {
            drop_request(S, r.get());
            set_last_error(e.what());
            return e.status;
        }
    }
    r->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    Request *rp = r.get();
    const bool done = r->done;
    S->reqs[rp->ticket] = std::move(r);
    if (!done) {
        S->hs[hid]->queue.push_back(rp);
        S->queued++;
        S->cv_work.notify_all();
    }
    return AMG_OK;
}

amg_status amg_server_wait(amg_server *S, uint64_t ticket, double *x, int timeout_ms, amg_solve_info *info) {
    set_last_error("");
    if (!S || !x) { set_last_error("NULL argument"); return AMG_ERR_INVALID; }
    std::unique_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) { set_last_error("unknown ticket"); return AMG_ERR_INVALID; }
        Request *rp = it->second.get();
        bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return rp->done; });
        if (!ok) { set_last_error("request not finished within the time limit"); return AMG_TIMEOUT; }
        r = std::move(it->second);
        S->reqs.erase(it);
        if (!r->has_result) set_last_error("server stopped: " + S->fatal);
    }
    amg_status st = (amg_status)r->status;
    try {  // the copy to the caller runs outside the lock
        DeviceGuard dg(S->device);
        if (r->has_result) {
            if (r->d_x) {
                AMG_CUDA(cudaStreamWaitEvent(S->io, r->ev, 0));
                AMG_CUDA(cudaMemcpyAsync(x, r->d_x, sizeof(double) * r->n, cudaMemcpyDeviceToHost, S->io));
                stage_free(S, r.get(), r->d_x, S->io);
                AMG_CUDA(cudaEventRecord(r->ev, S->io));
                AMG_CUDA(cudaEventSynchronize(r->ev));  // unbounded: the device writes the caller's x
            } else {
                std::memcpy(x, r->x.data(), sizeof(double) * r->x.size());
            }
        }
        drop_request(S, r.get());
    } catch (const Error &e) {
        drop_request(S, r.get());
        set_last_error(e.what());
        return e.status;
    }
    if (info) *info = r->info;
    return st;
}

void amg_server_destroy(amg_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto &H : S->hs)
        if (H->stream) cudaStreamSynchronize(H->stream);  // gathers into results not yet waited for
    for (auto &kv : S->reqs) drop_request(S, kv.second.get());  // requests never waited for
    S->reqs.clear();
    for (auto &H : S->hs) {
        if (H->ws) H->h->batch.erase(S->K);
        if (H->stream) cudaStreamDestroy(H->stream);
        if (H->done_ev) cudaEventDestroy(H->done_ev);
        if (H->copy_ev) cudaEventDestroy(H->copy_ev);
        if (H->hstage) cudaFreeHost(H->hstage);
    }
    if (S->io) {
        cudaStreamSynchronize(S->io);
        cudaStreamDestroy(S->io);
    }
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
}

}  // extern "C"
