// batch.cu -- many uneven integration jobs in one CUDA graph, and the
// autotuner of the persistent grid.  Built on the public plan calls: a batch is
// one plan per job (so each job's chunking, and therefore its result, is that
// of the job alone), whose kernels are captured into a single graph with the
// jobs spread over forked streams; replaying the graph costs one launch.
#include "bfi.h"
#include "bfi_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace {

bfi_status cuda_fail(const char *what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s failed: %s", what, cudaGetErrorString(e));
    return bfi::set_error(BFI_E_CUDA, msg);
}

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, int32_t> g_tuned;  // (nx, nt, precision, device) -> CTAs per SM

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int device) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != device) cudaSetDevice(device);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct bfi_batch {
    int device = 0;
    std::vector<bfi_plan *> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

bfi_status bfi_autotune_grid(const bfi_lattice *lattice, bfi_precision precision, int device, int32_t *ctas_per_sm) {
    bfi_status st = bfi::validate_lattice(lattice);
    if (st != BFI_OK) return st;
    if (!ctas_per_sm) return bfi::set_error(BFI_E_INVALID, "ctas_per_sm is NULL");
    const auto key = std::make_tuple(lattice->nx, lattice->nt, static_cast<int>(precision), device);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *ctas_per_sm = it->second;
            return BFI_OK;
        }
    }
    DeviceScope scope(device);
    // synthetic job: 64 subvolumes of [-5,5]^d with ~2^28 samples in total
    // (fewer for big lattices), a few milliseconds of work
    const int d = lattice->nx * lattice->nt;
    const int64_t nsub = 64;
    const uint64_t per_sub = std::max<uint64_t>(4096, (uint64_t(1) << 22) * 20 / std::max(d, 20));
    std::vector<uint64_t> samples(nsub, per_sub);
    std::vector<double> lo(nsub * d, -5.0), hi(nsub * d, 5.0);
    const int R = lattice->nx / 2 + 1;
    double *dbuf = nullptr;
    const size_t n_box = static_cast<size_t>(nsub) * d;
    const size_t n_out = static_cast<size_t>(nsub) * (5 + 3 * R) + (4 + 2 * R);
    cudaError_t e = cudaMalloc(&dbuf, sizeof(double) * (2 * n_box + n_out));
    if (e != cudaSuccess) return cuda_fail("autotune allocation", e);
    double *d_lo = dbuf, *d_hi = dbuf + n_box, *d_slots = dbuf + 2 * n_box, *d_tot = d_slots + nsub * (5 + 3 * R);
    e = cudaMemcpy(d_lo, lo.data(), sizeof(double) * n_box, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_hi, hi.data(), sizeof(double) * n_box, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dbuf);
        return cuda_fail("autotune copy", e);
    }
    bfi_plan *plan = nullptr;
    st = bfi_plan_create(&plan, lattice, nsub, samples.data(), precision, device);
    if (st != BFI_OK) {
        cudaFree(dbuf);
        return st;
    }
    bfi_plan_info info;
    bfi_plan_get_info(plan, &info);
    const int max_per_sm = std::max(1, static_cast<int>(info.ctas_per_sm_max));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // From the occupancy limit down: a smaller grid is chosen only when it wins
    // by 2%.  Measured on GB300, the batching workload ran 0.8% faster with
    // every job at its occupancy limit than with grids an earlier tuner picked
    // from the smallest grid up (ties and timing noise favoured small grids).
    int best = max_per_sm;
    float best_ms = INFINITY;
    for (int c = max_per_sm; c >= 1 && st == BFI_OK; --c) {
        if ((st = bfi_plan_set_grid(plan, c)) != BFI_OK) break;
        st = bfi_plan_execute(plan, d_lo, d_hi, nullptr, 1u, 0u, d_slots, d_tot, nullptr);  // warm-up
        std::vector<float> t;
        for (int rep = 0; rep < 5 && st == BFI_OK; ++rep) {
            cudaEventRecord(a, nullptr);
            st = bfi_plan_execute(plan, d_lo, d_hi, nullptr, 1u, 0u, d_slots, d_tot, nullptr);
            cudaEventRecord(b, nullptr);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            t.push_back(ms);
        }
        if (st != BFI_OK) break;
        std::sort(t.begin(), t.end());
        if (best_ms == INFINITY || t[2] < best_ms * 0.98f) {
            best_ms = t[2];
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    bfi_plan_destroy(plan);
    cudaFree(dbuf);
    if (st != BFI_OK) return st;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("autotune", e);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[key] = best;
    }
    *ctas_per_sm = best;
    return BFI_OK;
}

bfi_status bfi_batch_destroy(bfi_batch *batch) {
    if (!batch) return BFI_OK;
    {
        DeviceScope scope(batch->device);
        if (batch->exec) cudaGraphExecDestroy(batch->exec);
        if (batch->graph) cudaGraphDestroy(batch->graph);
        for (auto p : batch->plans) bfi_plan_destroy(p);
        for (auto s : batch->streams) cudaStreamDestroy(s);
        for (auto ev : batch->events) cudaEventDestroy(ev);
    }
    delete batch;
    return BFI_OK;
}

bfi_status bfi_batch_create(bfi_batch **out, const bfi_job *jobs, int32_t njobs, bfi_precision precision, int device,
                            int32_t nstreams, int32_t autotune) {
    if (!out || !jobs || njobs < 1) return bfi::set_error(BFI_E_INVALID, "need out, jobs and njobs >= 1");
    *out = nullptr;
    if (nstreams < 1) nstreams = 1;
    for (int32_t i = 0; i < njobs; ++i)
        if (!jobs[i].lo || !jobs[i].hi || !jobs[i].slots || !jobs[i].totals || !jobs[i].samples)
            return bfi::set_error(BFI_E_INVALID, "a job has a NULL array");
    DeviceScope scope(device);
    bfi_batch *b = new (std::nothrow) bfi_batch();
    if (!b) return bfi::set_error(BFI_E_NOMEM, "host allocation failed");
    b->device = device;
    bfi_status st = BFI_OK;
    for (int32_t i = 0; i < njobs && st == BFI_OK; ++i) {
        bfi_plan *p = nullptr;
        st = bfi_plan_create(&p, &jobs[i].lattice, jobs[i].nsub, jobs[i].samples, precision, device);
        if (st != BFI_OK) break;
        b->plans.push_back(p);
        if (autotune) {
            int32_t c = 0;
            st = bfi_autotune_grid(&jobs[i].lattice, precision, device, &c);
            if (st == BFI_OK) st = bfi_plan_set_grid(p, c);
        }
    }
    cudaError_t e = cudaSuccess;
    for (int32_t k = 0; k < nstreams && st == BFI_OK; ++k) {
        cudaStream_t s;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
            st = cuda_fail("cudaStreamCreate", e);
            break;
        }
        b->streams.push_back(s);
    }
    for (int32_t k = 0; k < nstreams + 1 && st == BFI_OK; ++k) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            st = cuda_fail("cudaEventCreate", e);
            break;
        }
        b->events.push_back(ev);
    }
    // one plain pass (sets kernel attributes outside capture, checks every job)
    for (int32_t i = 0; i < njobs && st == BFI_OK; ++i)
        st = bfi_plan_execute(b->plans[i], jobs[i].lo, jobs[i].hi, jobs[i].sub_id, jobs[i].seed, jobs[i].job_id,
                              jobs[i].slots, jobs[i].totals, b->streams[i % nstreams]);
    for (int32_t k = 0; k < nstreams && st == BFI_OK; ++k)
        if ((e = cudaStreamSynchronize(b->streams[k])) != cudaSuccess) st = cuda_fail("batch warm-up", e);
    // capture: fork from stream 0 to the others, one job per stream in turn, join back
    if (st == BFI_OK) {
        cudaStream_t origin = b->streams[0];
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail("cudaStreamBeginCapture", e);
        if (st == BFI_OK) {
            cudaEventRecord(b->events[nstreams], origin);
            for (int32_t k = 1; k < nstreams; ++k) cudaStreamWaitEvent(b->streams[k], b->events[nstreams], 0);
            for (int32_t i = 0; i < njobs && st == BFI_OK; ++i)
                st = bfi_plan_execute(b->plans[i], jobs[i].lo, jobs[i].hi, jobs[i].sub_id, jobs[i].seed,
                                      jobs[i].job_id, jobs[i].slots, jobs[i].totals, b->streams[i % nstreams]);
            for (int32_t k = 1; k < nstreams; ++k) {
                cudaEventRecord(b->events[k], b->streams[k]);
                cudaStreamWaitEvent(origin, b->events[k], 0);
            }
            const cudaError_t e2 = cudaStreamEndCapture(origin, &b->graph);
            if (st == BFI_OK && e2 != cudaSuccess) st = cuda_fail("cudaStreamEndCapture", e2);
        }
        if (st == BFI_OK && (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
            st = cuda_fail("cudaGraphInstantiate", e);
    }
    if (st != BFI_OK) {
        cudaGetLastError();
        bfi_batch_destroy(b);
        return st;
    }
    *out = b;
    return BFI_OK;
}

bfi_status bfi_batch_get_work(bfi_batch *batch, int32_t job, bfi_work *work) {
    if (!batch || job < 0 || job >= static_cast<int32_t>(batch->plans.size()))
        return bfi::set_error(BFI_E_INVALID, "batch is NULL or job out of range");
    return bfi_plan_get_work(batch->plans[job], work);
}

bfi_status bfi_batch_launch(bfi_batch *batch, void *stream) {
    if (!batch || !batch->exec) return bfi::set_error(BFI_E_INVALID, "batch is NULL");
    DeviceScope scope(batch->device);
    const cudaError_t e = cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail("cudaGraphLaunch", e);
    return BFI_OK;
}

}  // extern "C"
