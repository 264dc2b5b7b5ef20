// serve.cu -- bfi_server: integration jobs admitted as they arrive, with
// adaptive splitting of subvolumes (Sec. 3: the integration volume is
// subdivided until every part converges; the value of any region is computed
// separately and summed).
//
// One scheduler thread owns the queue.  A job is a sequence of passes (the
// first over its own subvolumes, then one per round of splitting).  A pass is
// admitted when one of the server's streams is free and its device memory
// (inputs, scratch, outputs: one block from the server's stream-ordered pool)
// fits in what remains of the budget; it then runs hint, integrand and merge
// kernels on that stream, copies its records to the stream's page-locked
// staging buffer, returns its memory to the pool and signals the scheduler
// from a host callback.  Passes of different jobs overlap on the device.  The
// scheduler never waits on the device: it sleeps on a condition variable that
// submissions and callbacks notify (and re-checks every 2 ms).
#include "bfi.h"
#include "bfi_host.h"
#include "bfi_kernels.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Request {
    std::mutex m;
    std::condition_variable cv;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled, 4 failed
    bfi_status status = BFI_OK;
    std::string message;
    bfi_lattice lat{};
    uint32_t seed = 0, job_id = 0;
    int d = 0, R = 0, SL = 0, TL = 0;
    int64_t nsub_initial = 0, leaf_cap = 0, pending = 0;
    uint32_t next_sid = 0;
    int passes = 0;
    uint64_t samples = 0;
    std::vector<double> leaf_slots, leaf_lo, leaf_hi, totals;
    std::vector<uint32_t> leaf_sid;
    bfi_work work{};  // counted work of every pass so far
    Clock::time_point t_submit, t_start, t_done;
    bool started = false;
    std::atomic<bool> cancel{false};
};

// Device block of one pass: byte offsets, 256-aligned.
struct Layout {
    size_t off, smp, hint, stats, fbuf, part, lo, hi, sid, slots, tot, total;
};

struct Pass {
    std::shared_ptr<Request> req;
    int64_t nsub = 0;
    std::vector<double> lo, hi;
    std::vector<uint64_t> samples;
    std::vector<uint32_t> sid;
    std::vector<int64_t> off;  // chunk table
    int64_t nchunks = 0;
    bfi::ChunkLayout chunks;
    float window = 0.f;
    Layout L{};
};

Layout layout_for(int64_t nsub, int64_t nchunks, int d, int K, int SL, int TL) {
    Layout L;
    size_t o = 0;
    L.off = o;   o += round_up(sizeof(int64_t) * (nsub + 1));
    L.smp = o;   o += round_up(sizeof(uint64_t) * nsub);
    L.hint = o;  o += round_up(sizeof(float) * nsub);
    L.stats = o; o += round_up(4 * sizeof(unsigned long long));  // evaluated, fully screened, stage 1, next chunk
    L.fbuf = o;  o += round_up(sizeof(double) * 2 * nsub);
    L.part = o;  o += round_up(sizeof(double) * static_cast<size_t>(nchunks > 0 ? nchunks : 1) * (K + 2));
    L.lo = o;    o += round_up(sizeof(double) * nsub * d);
    L.hi = o;    o += round_up(sizeof(double) * nsub * d);
    L.sid = o;   o += round_up(sizeof(uint32_t) * nsub);
    L.slots = o; o += round_up(sizeof(double) * nsub * SL);
    L.tot = o;   o += round_up(sizeof(double) * TL);
    L.total = o;
    return L;
}

std::shared_ptr<Pass> make_pass(const std::shared_ptr<Request> &r, bfi_precision) {
    auto p = std::make_shared<Pass>();
    p->req = r;
    return p;
}

// Chunk table, window and device layout once the pass's subvolumes are set.
void finalize_pass(Pass &p, bfi_precision precision) {
    const Request &r = *p.req;
    p.nsub = static_cast<int64_t>(p.samples.size());
    uint64_t total = 0, n_max = 1;
    for (uint64_t n : p.samples) {
        total += n;
        n_max = std::max(n_max, n);
    }
    p.chunks = bfi::plan_chunk_layout(p.samples.data(), p.nsub);
    p.off.assign(p.nsub + 1, 0);
    for (int64_t s = 0; s < p.nsub; ++s) p.off[s + 1] = p.off[s] + p.chunks.chunks_of(s, p.samples[s]);
    p.nchunks = p.off[p.nsub];
    p.window = bfi::plan_negligible_window(precision, n_max);
    p.L = layout_for(p.nsub, p.nchunks, r.d, 2 + 3 * r.R, r.SL, r.TL);
}

}  // namespace

struct bfi_server;

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    double *stage = nullptr;  // page-locked: the pass's slots then totals
    size_t stage_cap = 0;     // doubles
    bool busy = false;
    bool draining = false;    // its pass failed in flight; the slot is reused once the pass's callback arrives
    std::shared_ptr<Pass> pass;
    struct Ctx {
        bfi_server *srv;
        int index;
    } ctx{};
};

}  // namespace

struct bfi_server {
    bfi_server_config cfg{};
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;
    int sms = 1;
    std::mutex m;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Pass>> queue;
    std::deque<int> finished;
    uint64_t bytes_in_use = 0;
    bfi_server_stats st{};
    bool stopping = false;
    bool exited = false;      // the scheduler has left its loop (set under m, cv notified)
    bool broken = false;      // the scheduler stopped on an error: nothing more is admitted
    int32_t fault_point = 0;  // injected fault (host side): the point and how many passes reach it first
    int64_t fault_skip = 0;
    std::thread worker;
};

struct bfi_request {
    std::shared_ptr<Request> r;
    bfi_server *srv;
};

namespace {

void end_request(Request &r, int state, bfi_status status, const char *message) {
    std::lock_guard<std::mutex> lock(r.m);
    if (r.state >= 2) return;
    r.state = state;
    r.status = status;
    if (message) r.message = message;
    r.t_done = Clock::now();
    r.cv.notify_all();
}

// True when the injected fault fires at 'point' for this pass (one-shot).
bool take_fault(bfi_server *s, int32_t point) {
    std::lock_guard<std::mutex> lock(s->m);
    if (s->fault_point != point) return false;
    if (s->fault_skip > 0) {
        --s->fault_skip;
        return false;
    }
    s->fault_point = 0;
    return true;
}

void CUDART_CB on_pass_done(void *p) {
    auto *c = static_cast<Slot::Ctx *>(p);
    std::lock_guard<std::mutex> lock(c->srv->m);
    c->srv->finished.push_back(c->index);
    c->srv->cv.notify_all();
}

// Enqueue a pass on slot k's stream.  Called by the scheduler only.
bfi_status launch_pass(bfi_server *s, int k, Pass &p, std::string &msg) {
    Slot &sl = s->slots[k];
    Request &r = *p.req;
    cudaStream_t st = sl.stream;
    const size_t stage_need = static_cast<size_t>(p.nsub) * r.SL + r.TL + 3;  // records, totals, 3 counters
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) msg = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaSuccess;
    };
    if (sl.stage_cap < stage_need) {  // rare: grow the staging buffer (the stream is idle)
        if (sl.stage) cudaFreeHost(sl.stage);
        sl.stage = nullptr;
        sl.stage_cap = 0;
        if (!cuda(cudaHostAlloc(reinterpret_cast<void **>(&sl.stage), sizeof(double) * stage_need, 0),
                  "page-locked staging allocation"))
            return BFI_E_NOMEM;
        sl.stage_cap = stage_need;
    }
    const bfi::ShapeKernels *shape = bfi::find_shape(r.lat.nx, r.lat.nt);
    const bfi_precision prec = s->cfg.precision;
    void *block = nullptr;
    if (take_fault(s, BFI_FAULT_POOL_ALLOC)) {
        msg = "pool allocation: injected failure";
        return BFI_E_NOMEM;
    }
    if (!cuda(cudaMallocFromPoolAsync(&block, p.L.total, s->pool, st), "pool allocation")) return BFI_E_NOMEM;
    unsigned char *b = static_cast<unsigned char *>(block);
    auto at = [&](size_t o) { return static_cast<void *>(b + o); };
    bool ok = cuda(cudaMemcpyAsync(at(p.L.off), p.off.data(), sizeof(int64_t) * (p.nsub + 1), cudaMemcpyHostToDevice, st), "copy") &&
              cuda(cudaMemcpyAsync(at(p.L.smp), p.samples.data(), sizeof(uint64_t) * p.nsub, cudaMemcpyHostToDevice, st), "copy") &&
              cuda(cudaMemcpyAsync(at(p.L.lo), p.lo.data(), sizeof(double) * p.nsub * r.d, cudaMemcpyHostToDevice, st), "copy") &&
              cuda(cudaMemcpyAsync(at(p.L.hi), p.hi.data(), sizeof(double) * p.nsub * r.d, cudaMemcpyHostToDevice, st), "copy") &&
              cuda(cudaMemcpyAsync(at(p.L.sid), p.sid.data(), sizeof(uint32_t) * p.nsub, cudaMemcpyHostToDevice, st), "copy") &&
              cuda(cudaMemsetAsync(at(p.L.stats), 0, 4 * sizeof(unsigned long long), st), "memset");
    int per_sm = 1;
    if (ok) ok = cuda(shape->occupancy[prec](r.lat.nx, r.lat.nt, &per_sm), "occupancy");
    const bfi::LatticeParams lp{r.lat.nx, r.lat.nt, r.lat.nu, r.lat.D, r.lat.a, r.lat.tau, r.lat.nonlinear, r.lat.mass2};
    const double *lo = static_cast<const double *>(at(p.L.lo)), *hi = static_cast<const double *>(at(p.L.hi));
    double *slots = static_cast<double *>(at(p.L.slots)), *totals = static_cast<double *>(at(p.L.tot));
    if (ok && p.nchunks > 0) {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(p.nchunks, int64_t(s->sms) * std::max(per_sm, 1)));
        bfi::IntegrandArgs a{lo,
                             hi,
                             static_cast<const uint32_t *>(at(p.L.sid)),
                             static_cast<const uint64_t *>(at(p.L.smp)),
                             static_cast<const int64_t *>(at(p.L.off)),
                             static_cast<double *>(at(p.L.part)),
                             static_cast<float *>(at(p.L.hint)),
                             static_cast<unsigned long long *>(at(p.L.stats)),
                             p.nsub,
                             p.nchunks,
                             p.chunks.chunk_samples,
                             p.window,
                             static_cast<unsigned long long *>(at(p.L.stats)) + 1,
                             static_cast<unsigned long long *>(at(p.L.stats)) + 2,
                             static_cast<unsigned long long *>(at(p.L.stats)) + 3,
                             p.chunks.tail_sub,
                             p.chunks.tail_chunk_samples};
        ok = cuda(shape->integrand[prec](a, lp, r.seed, r.job_id, static_cast<int>(grid), st), "integrand launch");
    }
    if (ok && take_fault(s, BFI_FAULT_LAUNCH)) {
        msg = "merge launch: injected failure";
        ok = false;
    }
    if (ok) {
        const bfi::MergeArgs mg{lo, hi, static_cast<const int64_t *>(at(p.L.off)), static_cast<const double *>(at(p.L.part)),
                                slots, p.nsub, r.R, r.d, 0, 0.0};
        const bfi::TotalsArgs tg{slots, totals, static_cast<double *>(at(p.L.fbuf)), p.nsub, r.R};
        ok = cuda(bfi::launch_merges(mg, tg, st), "merge launch") &&
             cuda(cudaMemcpyAsync(sl.stage, slots, sizeof(double) * p.nsub * r.SL, cudaMemcpyDeviceToHost, st), "copy") &&
             cuda(cudaMemcpyAsync(sl.stage + static_cast<size_t>(p.nsub) * r.SL, totals, sizeof(double) * r.TL,
                                  cudaMemcpyDeviceToHost, st), "copy") &&
             cuda(cudaMemcpyAsync(sl.stage + static_cast<size_t>(p.nsub) * r.SL + r.TL, at(p.L.stats),
                                  3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st), "copy");
    }
    cudaFreeAsync(block, st);  // stream-ordered: after the copies
    if (!ok) {
        cudaStreamSynchronize(st);
        return BFI_E_CUDA;
    }
    if (!cuda(cudaLaunchHostFunc(st, on_pass_done, &sl.ctx), "host callback")) {
        cudaStreamSynchronize(st);
        return BFI_E_CUDA;
    }
    {
        std::lock_guard<std::mutex> lock(r.m);
        if (!r.started) {
            r.started = true;
            r.t_start = Clock::now();
        }
        r.state = 1;
    }
    return BFI_OK;
}

// Results of a finished pass (records in 'stage'): split what has not
// converged, keep the rest as leaves; queue the next pass or finish the job.
void finish_pass(bfi_server *s, Pass &p, const double *stage) {
    Request &r = *p.req;
    if (r.cancel.load()) {
        end_request(r, 3, BFI_E_CANCELLED, "cancelled");
        std::lock_guard<std::mutex> lock(s->m);
        s->st.cancelled++;
        return;
    }
    std::unique_lock<std::mutex> rl(r.m);  // leaves and counters are read by bfi_request_get_info
    r.passes++;
    uint64_t pass_samples = 0;
    for (uint64_t n : p.samples) pass_samples += n;
    r.samples += pass_samples;
    {  // the pass's work counters follow its records and totals in the staging buffer
        unsigned long long c[3];
        std::memcpy(c, stage + static_cast<size_t>(p.nsub) * r.SL + r.TL, sizeof c);
        const bfi::ShapeKernels *shape = bfi::find_shape(r.lat.nx, r.lat.nt);
        const uint64_t full = pass_samples - c[2];
        r.work.samples += pass_samples;
        r.work.evaluated += c[0];
        r.work.stage1 += c[2];
        r.work.full_screen += full;
        r.work.survivors += shape && shape->two_stage ? c[1] - full : 0;
        r.work.two_stage_shape = shape && shape->two_stage ? 1 : 0;
        r.work.rest_screen = r.work.two_stage_shape && r.lat.nt == 2 && r.lat.nx % 2 == 0 &&
                             static_cast<float>(0.5 * r.lat.mass2) == 0.f;
    }
    auto next = make_pass(p.req, s->cfg.precision);
    const double thr = s->cfg.split_rel_var;
    const bool may_split = thr > 0.0 && r.passes <= s->cfg.max_split_rounds;
    const int d = r.d;
    for (int64_t k = 0; k < p.nsub; ++k) {
        const double *q = stage + static_cast<size_t>(k) * r.SL;
        const double n = q[0], sw = q[3], sw2 = q[4];
        bool split = false;
        if (may_split && n >= 2.0 && sw > 0.0) {
            const double relvar = (n * sw2 - sw * sw) / ((n - 1.0) * sw * sw);
            const int64_t leaves = static_cast<int64_t>(r.leaf_sid.size()) + static_cast<int64_t>(next->samples.size());
            split = relvar > thr && leaves + 2 + (p.nsub - k - 1) <= r.leaf_cap;
        }
        const double *lo = p.lo.data() + k * d, *hi = p.hi.data() + k * d;
        if (split) {
            int dim = 0;
            for (int j = 1; j < d; ++j)
                if (hi[j] - lo[j] > hi[dim] - lo[dim]) dim = j;
            const double mid = 0.5 * (lo[dim] + hi[dim]);
            for (int side = 0; side < 2; ++side) {
                next->lo.insert(next->lo.end(), lo, lo + d);
                next->hi.insert(next->hi.end(), hi, hi + d);
                if (side == 0) next->hi[next->hi.size() - d + dim] = mid;
                else next->lo[next->lo.size() - d + dim] = mid;
                next->samples.push_back(p.samples[k]);
                next->sid.push_back(r.next_sid++);
            }
        } else {
            r.leaf_slots.insert(r.leaf_slots.end(), q, q + r.SL);
            r.leaf_lo.insert(r.leaf_lo.end(), lo, lo + d);
            r.leaf_hi.insert(r.leaf_hi.end(), hi, hi + d);
            r.leaf_sid.push_back(p.sid[k]);
        }
    }
    if (!next->samples.empty()) {
        rl.unlock();
        finalize_pass(*next, s->cfg.precision);
        std::lock_guard<std::mutex> lock(s->m);
        s->queue.push_front(next);  // a started job goes ahead of new ones
        s->st.queued++;
        s->cv.notify_all();
        return;
    }
    r.totals.assign(r.TL, 0.0);
    const bfi_status ms = bfi_merge_host(r.lat.nx, static_cast<int64_t>(r.leaf_sid.size()), r.leaf_slots.data(),
                                         r.totals.data());
    rl.unlock();
    end_request(r, ms == BFI_OK ? 2 : 4, ms, ms == BFI_OK ? nullptr : "merge failed");
    std::lock_guard<std::mutex> lock(s->m);
    s->st.completed++;
}

// A pass that failed after admission: its job fails with 'status', its
// memory returns to the budget.  The caller holds s->m.
void fail_running(bfi_server *s, Slot &sl, bfi_status status, const std::string &msg,
                  std::unique_lock<std::mutex> &lk) {
    std::shared_ptr<Pass> pass = sl.pass;
    sl.pass.reset();
    s->bytes_in_use -= pass->L.total;
    s->st.running--;
    s->st.failed++;
    lk.unlock();
    end_request(*pass->req, 4, status, msg.c_str());
    lk.lock();
}

void scheduler_loop(bfi_server *s, std::unique_lock<std::mutex> &lk) {
    for (;;) {
        while (!s->finished.empty()) {
            const int k = s->finished.front();
            s->finished.pop_front();
            Slot &sl = s->slots[k];
            if (sl.draining) {  // the late callback of a pass that already failed: the slot is free again
                sl.draining = false;
                sl.busy = false;
                continue;
            }
            // The callback ran, so the stream has passed every kernel and copy
            // of the pass: an error status now is the pass's, and its records
            // in the staging buffer are not to be read.
            lk.unlock();
            cudaError_t e = take_fault(s, BFI_FAULT_COMPLETION) ? cudaErrorLaunchFailure : cudaStreamQuery(sl.stream);
            if (take_fault(s, BFI_FAULT_SCHEDULER)) throw std::runtime_error("injected scheduler failure");
            lk.lock();
            if (e != cudaSuccess && e != cudaErrorNotReady) {
                sl.busy = false;
                fail_running(s, sl, BFI_E_CUDA, std::string("pass failed on the device: ") + cudaGetErrorString(e), lk);
                continue;
            }
            std::shared_ptr<Pass> pass = sl.pass;
            sl.pass.reset();
            sl.busy = false;
            s->bytes_in_use -= pass->L.total;
            s->st.running--;
            for (uint64_t n : pass->samples) s->st.samples += n;
            lk.unlock();
            finish_pass(s, *pass, sl.stage);
            lk.lock();
        }
        // A pass whose stream reports an error before its callback (after an
        // asynchronous failure the callback may never run) fails now; its slot
        // drains until the callback arrives.
        for (Slot &sl : s->slots) {
            if (!sl.busy || sl.draining) continue;
            const cudaError_t e = cudaStreamQuery(sl.stream);
            if (e == cudaSuccess || e == cudaErrorNotReady) continue;
            sl.draining = true;
            fail_running(s, sl, BFI_E_CUDA, std::string("pass failed on the device: ") + cudaGetErrorString(e), lk);
        }
        while (!s->queue.empty()) {
            std::shared_ptr<Pass> pass = s->queue.front();
            Request &r = *pass->req;
            if (r.cancel.load() || s->stopping) {
                s->queue.pop_front();
                s->st.queued--;
                s->st.cancelled++;
                lk.unlock();
                end_request(r, 3, BFI_E_CANCELLED, "cancelled");
                lk.lock();
                continue;
            }
            if (pass->L.total > s->cfg.memory_budget) {
                s->queue.pop_front();
                s->st.queued--;
                s->st.failed++;
                lk.unlock();
                char msg[160];
                std::snprintf(msg, sizeof msg, "a pass needs %zu bytes, more than the memory budget", pass->L.total);
                end_request(r, 4, BFI_E_NOMEM, msg);
                lk.lock();
                continue;
            }
            int k = -1;
            for (int i = 0; i < static_cast<int>(s->slots.size()); ++i)
                if (!s->slots[i].busy) {
                    k = i;
                    break;
                }
            if (k < 0 || s->bytes_in_use + pass->L.total > s->cfg.memory_budget) break;
            s->queue.pop_front();
            s->st.queued--;
            s->st.running++;
            s->slots[k].busy = true;
            s->slots[k].pass = pass;
            s->bytes_in_use += pass->L.total;
            s->st.bytes_peak = std::max<uint64_t>(s->st.bytes_peak, s->bytes_in_use);
            lk.unlock();
            std::string msg;
            const bfi_status rc = launch_pass(s, k, *pass, msg);
            lk.lock();
            if (rc != BFI_OK) {
                s->slots[k].busy = false;
                fail_running(s, s->slots[k], rc, msg, lk);
            }
        }
        bool busy = false;
        for (const Slot &sl : s->slots) busy = busy || (sl.busy && !sl.draining);
        if (s->stopping && s->queue.empty() && !busy && s->finished.empty()) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

// The scheduler thread.  If its loop stops on an exception (a failed host
// allocation, or an injected fault), every job still queued or running fails
// with BFI_E_NOMEM and a message, so that no wait is left without an end, and
// the server admits nothing more.
void scheduler(bfi_server *s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->m);
    std::string why;
    try {
        scheduler_loop(s, lk);
    } catch (const std::exception &e) {
        why = e.what();
    } catch (...) {
        why = "unknown exception";
    }
    if (!lk.owns_lock()) lk.lock();
    if (!why.empty()) {
        s->broken = true;
        const std::string msg = "the server's scheduler stopped: " + why;
        std::vector<std::shared_ptr<Request>> ended;
        for (auto &p : s->queue) ended.push_back(p->req);
        s->st.failed += s->queue.size();
        s->st.queued = 0;
        s->queue.clear();
        for (Slot &sl : s->slots)
            if (sl.busy && !sl.draining && sl.pass) {
                ended.push_back(sl.pass->req);
                s->st.failed++;
                s->st.running--;
                sl.draining = true;  // its stream still finishes; destroy waits for it
            }
        s->finished.clear();
        lk.unlock();
        for (auto &r : ended) end_request(*r, 4, BFI_E_NOMEM, msg.c_str());
        lk.lock();
    }
    s->exited = true;
    s->cv.notify_all();
}

bfi_status fail_msg(bfi_status st, const std::string &m) { return bfi::set_error(st, m.c_str()); }

}  // namespace

extern "C" {

bfi_status bfi_server_create(bfi_server **out, const bfi_server_config *config) {
    if (!out || !config) return bfi::set_error(BFI_E_INVALID, "out and config must be non-NULL");
    *out = nullptr;
    if (config->slots < 1) return bfi::set_error(BFI_E_INVALID, "slots must be >= 1");
    if (config->precision != BFI_FP64 && config->precision != BFI_FP32)
        return bfi::set_error(BFI_E_INVALID, "precision must be BFI_FP64 or BFI_FP32");
    if (config->memory_budget == 0) return bfi::set_error(BFI_E_INVALID, "memory_budget must be > 0");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(config->device);
    if (e != cudaSuccess) return fail_msg(BFI_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    auto *s = new (std::nothrow) bfi_server();
    if (!s) return bfi::set_error(BFI_E_NOMEM, "host allocation failed");
    s->cfg = *config;
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, config->device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = config->device;
    e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = config->memory_budget;
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->slots.resize(config->slots);
    for (int k = 0; k < config->slots && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->slots[k].stream, cudaStreamNonBlocking);
        s->slots[k].ctx = Slot::Ctx{s, k};
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        for (auto &sl : s->slots)
            if (sl.stream) cudaStreamDestroy(sl.stream);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return fail_msg(BFI_E_CUDA, std::string("server set-up: ") + cudaGetErrorString(e));
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return BFI_OK;
}

bfi_status bfi_server_shutdown(bfi_server *s, int64_t timeout_ms) {
    if (!s) return bfi::set_error(BFI_E_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->m);
    s->stopping = true;
    s->cv.notify_all();
    auto done = [&] { return s->exited; };
    if (timeout_ms < 0)
        s->cv.wait(lk, done);
    else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return bfi::set_error(BFI_E_TIMEOUT, "running passes did not finish within the timeout");
    return BFI_OK;
}

bfi_status bfi_server_inject_fault(bfi_server *s, int32_t point, int64_t nth) {
    if (!s || point < BFI_FAULT_NONE || point > BFI_FAULT_SCHEDULER || nth < 0)
        return bfi::set_error(BFI_E_INVALID, "server is NULL, or unknown fault point, or nth < 0");
    std::lock_guard<std::mutex> lock(s->m);
    s->fault_point = point;
    s->fault_skip = nth;
    return BFI_OK;
}

bfi_status bfi_server_destroy(bfi_server *s) {
    if (!s) return BFI_OK;
    bfi_server_shutdown(s, -1);
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    for (auto &sl : s->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        if (sl.stage) cudaFreeHost(sl.stage);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
    return BFI_OK;
}

bfi_status bfi_server_get_stats(bfi_server *s, bfi_server_stats *stats) {
    if (!s || !stats) return bfi::set_error(BFI_E_INVALID, "server or stats is NULL");
    std::lock_guard<std::mutex> lock(s->m);
    *stats = s->st;
    stats->bytes_in_use = s->bytes_in_use;
    return BFI_OK;
}

bfi_status bfi_submit(bfi_server *s, const bfi_lattice *lattice, int64_t nsub, const double *lo, const double *hi,
                      const uint64_t *samples, uint32_t seed, uint32_t job_id, bfi_request **out) {
    if (!s || !out) return bfi::set_error(BFI_E_INVALID, "server and out must be non-NULL");
    *out = nullptr;
    bfi_status st = bfi::validate_lattice(lattice);
    if (st != BFI_OK) return st;
    if (nsub < 1 || !lo || !hi || !samples) return bfi::set_error(BFI_E_INVALID, "need nsub >= 1, lo, hi, samples");
    if (!bfi::find_shape(lattice->nx, lattice->nt)) return bfi::set_error(BFI_E_UNSUPPORTED, "lattice shape");
    for (int64_t k = 0; k < nsub; ++k)
        if (samples[k] >= (1ull << 48)) return bfi::set_error(BFI_E_INVALID, "a sample budget is >= 2^48");
    auto r = std::make_shared<Request>();
    r->lat = *lattice;
    r->seed = seed;
    r->job_id = job_id;
    r->d = lattice->nx * lattice->nt;
    r->R = lattice->nx / 2 + 1;
    r->SL = 5 + 3 * r->R;
    r->TL = 4 + 2 * r->R;
    r->nsub_initial = nsub;
    r->leaf_cap = 16 * nsub;
    r->next_sid = static_cast<uint32_t>(nsub);
    r->t_submit = Clock::now();
    auto p = make_pass(r, s->cfg.precision);
    p->lo.assign(lo, lo + nsub * r->d);
    p->hi.assign(hi, hi + nsub * r->d);
    p->samples.assign(samples, samples + nsub);
    p->sid.resize(nsub);
    for (int64_t k = 0; k < nsub; ++k) p->sid[k] = static_cast<uint32_t>(k);
    finalize_pass(*p, s->cfg.precision);
    auto *h = new (std::nothrow) bfi_request();
    if (!h) return bfi::set_error(BFI_E_NOMEM, "host allocation failed");
    h->r = r;
    h->srv = s;
    {
        std::lock_guard<std::mutex> lock(s->m);
        if (s->stopping || s->broken) {
            delete h;
            return bfi::set_error(BFI_E_BUSY, s->broken ? "the server's scheduler has stopped" : "server is stopping");
        }
        s->queue.push_back(p);
        s->st.submitted++;
        s->st.queued++;
        s->cv.notify_all();
    }
    *out = h;
    return BFI_OK;
}

bfi_status bfi_poll(bfi_request *h, int32_t *done) {
    if (!h || !done) return bfi::set_error(BFI_E_INVALID, "request or done is NULL");
    std::lock_guard<std::mutex> lock(h->r->m);
    *done = h->r->state >= 2;
    return BFI_OK;
}

bfi_status bfi_wait(bfi_request *h, int64_t timeout_ms) {
    if (!h) return bfi::set_error(BFI_E_INVALID, "request is NULL");
    Request &r = *h->r;
    std::unique_lock<std::mutex> lk(r.m);
    auto ended = [&] { return r.state >= 2; };
    if (timeout_ms < 0)
        r.cv.wait(lk, ended);
    else if (!r.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ended))
        return bfi::set_error(BFI_E_TIMEOUT, "request not finished within the timeout");
    if (r.state == 2) return BFI_OK;
    if (r.state == 3) return bfi::set_error(BFI_E_CANCELLED, "request was cancelled");
    return fail_msg(r.status, r.message);
}

bfi_status bfi_cancel(bfi_request *h) {
    if (!h) return bfi::set_error(BFI_E_INVALID, "request is NULL");
    h->r->cancel.store(true);
    std::lock_guard<std::mutex> lock(h->srv->m);
    h->srv->cv.notify_all();
    return BFI_OK;
}

bfi_status bfi_request_get_info(bfi_request *h, bfi_request_info *info) {
    if (!h || !info) return bfi::set_error(BFI_E_INVALID, "request or info is NULL");
    Request &r = *h->r;
    std::lock_guard<std::mutex> lock(r.m);
    info->state = r.state;
    info->status = r.status;
    info->nsub_final = static_cast<int64_t>(r.leaf_sid.size());
    info->passes = r.passes;
    info->samples = r.samples;
    info->queued_ms = r.started ? ms_between(r.t_submit, r.t_start) : -1.0;
    info->latency_ms = r.state >= 2 ? ms_between(r.t_submit, r.t_done) : -1.0;
    return BFI_OK;
}

bfi_status bfi_request_get_result(bfi_request *h, double *totals, double *slots, double *lo, double *hi,
                                  uint32_t *sub_id) {
    if (!h) return bfi::set_error(BFI_E_INVALID, "request is NULL");
    Request &r = *h->r;
    std::lock_guard<std::mutex> lock(r.m);
    if (r.state < 2) return bfi::set_error(BFI_E_BUSY, "request not finished");
    if (r.state == 3) return bfi::set_error(BFI_E_CANCELLED, "request was cancelled");
    if (r.state == 4) return fail_msg(r.status, r.message);
    if (totals) std::memcpy(totals, r.totals.data(), sizeof(double) * r.totals.size());
    if (slots) std::memcpy(slots, r.leaf_slots.data(), sizeof(double) * r.leaf_slots.size());
    if (lo) std::memcpy(lo, r.leaf_lo.data(), sizeof(double) * r.leaf_lo.size());
    if (hi) std::memcpy(hi, r.leaf_hi.data(), sizeof(double) * r.leaf_hi.size());
    if (sub_id) std::memcpy(sub_id, r.leaf_sid.data(), sizeof(uint32_t) * r.leaf_sid.size());
    return BFI_OK;
}

bfi_status bfi_request_get_work(bfi_request *h, bfi_work *work) {
    if (!h || !work) return bfi::set_error(BFI_E_INVALID, "request or work is NULL");
    std::lock_guard<std::mutex> lock(h->r->m);
    *work = h->r->work;
    return BFI_OK;
}

bfi_status bfi_request_release(bfi_request *h) {
    if (!h) return BFI_OK;
    bool finished;
    {
        std::lock_guard<std::mutex> lock(h->r->m);
        finished = h->r->state >= 2;
    }
    if (!finished) bfi_cancel(h);
    delete h;
    return BFI_OK;
}

}  // extern "C"
