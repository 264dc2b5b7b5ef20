// api.cu -- the C ABI declared in include/bfi.h: argument checks, plans
// (chunking of the sample budgets and the device scratch), the one-call
// host-buffer path, the host FP64 merge and the single-step entry points.
#include "bfi.h"
#include "bfi_device.cuh"
#include "bfi_host.h"
#include "bfi_kernels.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_last_error;

bfi_status fail(bfi_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define BFI_CUDA(expr)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (expr);                                                                         \
        if (e_ != cudaSuccess) return fail(BFI_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Makes 'device' current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int device) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != device) err = cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bfi_status check_lattice(const bfi_lattice *L) {
    if (!L) return fail(BFI_E_INVALID, "lattice is NULL");
    if (L->nx < 2 || L->nt < 1) return fail(BFI_E_INVALID, "lattice %dx%d: need nx >= 2, nt >= 1", L->nx, L->nt);
    if (static_cast<int64_t>(L->nx) * L->nt > bfi::kMaxD)
        return fail(BFI_E_INVALID, "lattice %dx%d: d = nx*nt must be <= %d", L->nx, L->nt, bfi::kMaxD);
    if (!finite_pos(L->D) || !finite_pos(L->a) || !finite_pos(L->tau))
        return fail(BFI_E_INVALID, "D, a and tau must be finite and > 0");
    if (!std::isfinite(L->nu) || L->nu < 0.0) return fail(BFI_E_INVALID, "nu must be finite and >= 0");
    if (!std::isfinite(L->nonlinear)) return fail(BFI_E_INVALID, "nonlinear must be finite");
    if (!std::isfinite(L->mass2) || L->mass2 < 0.0) return fail(BFI_E_INVALID, "mass2 must be finite and >= 0");
    return BFI_OK;
}

bfi::LatticeParams to_params(const bfi_lattice *L) {
    return bfi::LatticeParams{L->nx, L->nt, L->nu, L->D, L->a, L->tau, L->nonlinear, L->mass2};
}

int num_r(int nx) { return nx / 2 + 1; }

// Samples per chunk: a multiple of the block size, chosen from the job alone
// (never from the device or from other jobs) so that a job's rounding is the
// same wherever and with whatever else it runs.  At least 2048 chunks and up
// to 512 rows per thread; from there the rows double, up to 2048, while the
// job keeps at least 4096 chunks.  Longer chunks screen fewer points: a
// chunk's running reference starts at the subvolume's hint and falls as the
// chunk finds lower actions, so the screen passes more points early in every
// chunk, and each chunk ends with a queue drain and a record.  4096 chunks
// keep the end of the launch, where CTAs run out of chunks, short.
int64_t choose_chunk_samples(uint64_t total) {
    const uint64_t block = static_cast<uint64_t>(bfi::kBlock);
    uint64_t per_thread = total / (block * 2048u);
    uint64_t spt = 4;
    while (spt * 2 <= per_thread && spt < 512) spt *= 2;
    while (spt >= 512 && spt < 2048 && total / (block * spt * 2) >= 4096u) spt *= 2;
    return static_cast<int64_t>(spt) * bfi::kBlock;
}

// Samples whose action exceeds the subvolume's smallest by more than this
// are left out of the sums: the n <= n_max of them change any sum by less than
// n_max e^-window = e^-c relative, c = 34 in FP64 (below its 1e-12
// agreement with an FP64 reference by 1e-3) and 20 in FP32.
float negligible_window(bfi_precision precision, uint64_t n_max) {
    const double c = precision == BFI_FP64 ? 34.0 : 20.0;
    return static_cast<float>(c + std::log(static_cast<double>(n_max)));
}

}  // namespace

namespace bfi {
bfi_status set_error(bfi_status status, const char *message) {
    g_last_error = message;
    return status;
}
bfi_status validate_lattice(const bfi_lattice *lattice) { return check_lattice(lattice); }
// The chunks a CTA takes last are the shortest.  Once the chunks run out, each
// CTA still finishes the chunk it holds, and an SM stops only when its last
// CTA does; the slowest of the SMs sets the end of the launch, which comes
// about a third of a chunk's duration after the average SM would finish.  So
// the last subvolumes, the longest suffix holding at most an eighth of the
// samples and at most 512 full chunks' worth, are cut into chunks a quarter
// as long (never below 256 rows per thread, where the two-stage screen
// stops); chunks are handed out in index order, so these come last.
ChunkLayout plan_chunk_layout(const uint64_t *samples, int64_t nsub) {
    uint64_t total = 0;
    for (int64_t s = 0; s < nsub; ++s) total += samples[s];
    ChunkLayout L;
    L.chunk_samples = choose_chunk_samples(total);
    L.tail_chunk_samples = L.chunk_samples;
    L.tail_sub = nsub;
    const int64_t min_tail = static_cast<int64_t>(kTwoStageMinRows) * kBlock;
    if (L.chunk_samples > min_tail) {
        const uint64_t limit = std::min<uint64_t>(total / 8, 512u * static_cast<uint64_t>(L.chunk_samples));
        uint64_t tail = 0;
        int64_t s = nsub;
        while (s > 0 && tail + samples[s - 1] <= limit) tail += samples[--s];
        if (s < nsub && tail > 0) {
            L.tail_sub = s;
            L.tail_chunk_samples = std::max<int64_t>(L.chunk_samples / 4, min_tail);
        }
    }
    return L;
}
float plan_negligible_window(bfi_precision precision, uint64_t n_max) { return negligible_window(precision, n_max); }
}  // namespace bfi

struct bfi_plan {
    int device = 0;
    bfi::LatticeParams lat{};
    bfi_precision precision = BFI_FP64;
    const bfi::ShapeKernels *shape = nullptr;
    int64_t nsub = 0, nchunks = 0, chunk_samples = 0, total = 0;
    bfi::ChunkLayout layout;
    int grid = 1;
    int sms = 1, per_sm_max = 1, per_sm = 1;
    int R = 0, K = 0, d = 0;
    std::vector<uint64_t> samples;
    int64_t *d_chunk_off = nullptr;
    uint64_t *d_samples = nullptr;
    double *d_partials = nullptr;
    float *d_hint = nullptr;
    unsigned long long *d_stats = nullptr;
    double *d_fbuf = nullptr;
    float skip_window = 0.f;
    size_t scratch_bytes = 0;
    bool timing = false, timed = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int32_t sampler = BFI_SAMPLE_BOX;
    double *d_map = nullptr;  // Gaussian sampler: mean [d], then factor [d * d]
    double log_norm = 0.0;    // Gaussian sampler: (d/2) ln 2 pi + ln |det F|
    bool map_upper = false;   // Gaussian sampler: F is upper triangular
};

extern "C" {

int32_t bfi_num_r(int32_t nx) { return nx / 2 + 1; }
int32_t bfi_slot_len(int32_t nx) { return 5 + 3 * (nx / 2 + 1); }
int32_t bfi_totals_len(int32_t nx) { return 4 + 2 * (nx / 2 + 1); }
const char *bfi_last_error(void) { return g_last_error.c_str(); }

bfi_status bfi_plan_destroy(bfi_plan *plan) {
    if (!plan) return BFI_OK;
    {
        DeviceGuard g(plan->device);
        cudaFree(plan->d_chunk_off);
        cudaFree(plan->d_samples);
        cudaFree(plan->d_partials);
        cudaFree(plan->d_hint);
        cudaFree(plan->d_stats);
        cudaFree(plan->d_fbuf);
        cudaFree(plan->d_map);
        for (auto &e : plan->ev)
            if (e) cudaEventDestroy(e);
    }
    delete plan;
    return BFI_OK;
}

bfi_status bfi_plan_create(bfi_plan **out, const bfi_lattice *lattice, int64_t nsub, const uint64_t *samples,
                           bfi_precision precision, int device) {
    if (!out) return fail(BFI_E_INVALID, "out is NULL");
    *out = nullptr;
    bfi_status st = check_lattice(lattice);
    if (st != BFI_OK) return st;
    if (nsub < 1) return fail(BFI_E_INVALID, "nsub must be >= 1 (got %lld)", static_cast<long long>(nsub));
    if (!samples) return fail(BFI_E_INVALID, "samples is NULL");
    if (precision != BFI_FP64 && precision != BFI_FP32) return fail(BFI_E_INVALID, "unknown precision %d", precision);
    const bfi::ShapeKernels *shape = bfi::find_shape(lattice->nx, lattice->nt);
    if (!shape)
        return fail(BFI_E_UNSUPPORTED, "lattice %dx%d has no compiled kernel in this library", lattice->nx,
                    lattice->nt);
    uint64_t total = 0;
    for (int64_t s = 0; s < nsub; ++s) {
        if (samples[s] >= (1ull << 48))
            return fail(BFI_E_INVALID, "samples[%lld] = %llu must be < 2^48", static_cast<long long>(s),
                        static_cast<unsigned long long>(samples[s]));
        total += samples[s];
    }
    if (total >= (1ull << 62)) return fail(BFI_E_INVALID, "total sample budget too large");

    DeviceGuard g(device);
    if (g.err != cudaSuccess) return fail(BFI_E_CUDA, "cannot select device %d: %s", device, cudaGetErrorString(g.err));

    bfi_plan *p = new (std::nothrow) bfi_plan();
    if (!p) return fail(BFI_E_NOMEM, "host allocation failed");
    p->device = device;
    p->lat = to_params(lattice);
    p->precision = precision;
    p->shape = shape;
    p->nsub = nsub;
    p->R = num_r(lattice->nx);
    p->K = bfi::sum_count(p->R);
    p->d = lattice->nx * lattice->nt;
    p->total = static_cast<int64_t>(total);
    p->samples.assign(samples, samples + nsub);
    p->layout = bfi::plan_chunk_layout(samples, nsub);
    p->chunk_samples = p->layout.chunk_samples;
    uint64_t n_max = 1;
    for (int64_t s = 0; s < nsub; ++s) n_max = std::max<uint64_t>(n_max, samples[s]);
    p->skip_window = negligible_window(precision, n_max);
    std::vector<int64_t> off(nsub + 1, 0);
    for (int64_t s = 0; s < nsub; ++s)
        off[s + 1] = off[s] + p->layout.chunks_of(s, samples[s]);
    p->nchunks = off[nsub];

    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = shape->occupancy[precision](lattice->nx, lattice->nt, &per_sm);
    if (e != cudaSuccess) {
        delete p;
        return fail(BFI_E_CUDA, "device query failed: %s", cudaGetErrorString(e));
    }
    p->sms = sms;
    p->per_sm_max = per_sm > 0 ? per_sm : 1;
    p->per_sm = p->per_sm_max;
    const int64_t resident = static_cast<int64_t>(sms) * p->per_sm_max;
    p->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p->nchunks, resident)));

    const size_t off_bytes = sizeof(int64_t) * (nsub + 1);
    const size_t smp_bytes = sizeof(uint64_t) * nsub;
    const size_t par_bytes = sizeof(double) * static_cast<size_t>(std::max<int64_t>(p->nchunks, 1)) * (p->K + 2);
    const size_t hint_bytes = sizeof(float) * nsub;
    p->scratch_bytes = off_bytes + smp_bytes + par_bytes + hint_bytes + 4 * sizeof(unsigned long long) + sizeof(double) * 2 * nsub;
    if (cudaMalloc(&p->d_chunk_off, off_bytes) != cudaSuccess || cudaMalloc(&p->d_samples, smp_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_partials, par_bytes) != cudaSuccess || cudaMalloc(&p->d_hint, hint_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_stats, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&p->d_fbuf, sizeof(double) * 2 * nsub) != cudaSuccess) {
        cudaGetLastError();
        bfi_plan_destroy(p);
        return fail(BFI_E_NOMEM, "device allocation of %zu bytes failed", p->scratch_bytes);
    }
    e = cudaMemcpy(p->d_chunk_off, off.data(), off_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_samples, samples, smp_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        bfi_plan_destroy(p);
        return fail(BFI_E_CUDA, "copy of the chunk table failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return BFI_OK;
}

bfi_status bfi_chunking_of(int64_t nsub, const uint64_t *samples, bfi_chunking *out) {
    if (!out || !samples) return fail(BFI_E_INVALID, "samples or out is NULL");
    if (nsub < 1) return fail(BFI_E_INVALID, "nsub must be >= 1 (got %lld)", static_cast<long long>(nsub));
    uint64_t total = 0;
    for (int64_t s = 0; s < nsub; ++s) {
        if (samples[s] >= (1ull << 48))
            return fail(BFI_E_INVALID, "samples[%lld] = %llu must be < 2^48", static_cast<long long>(s),
                        static_cast<unsigned long long>(samples[s]));
        total += samples[s];
    }
    if (total >= (1ull << 62)) return fail(BFI_E_INVALID, "total sample budget too large");
    const bfi::ChunkLayout L = bfi::plan_chunk_layout(samples, nsub);
    out->chunk_samples = L.chunk_samples;
    out->tail_subvolume = L.tail_sub;
    out->tail_chunk_samples = L.tail_chunk_samples;
    out->chunks = 0;
    for (int64_t s = 0; s < nsub; ++s) out->chunks += L.chunks_of(s, samples[s]);
    return BFI_OK;
}

bfi_status bfi_plan_get_info(const bfi_plan *plan, bfi_plan_info *info) {
    if (!plan || !info) return fail(BFI_E_INVALID, "plan or info is NULL");
    info->nsub = plan->nsub;
    info->chunks = plan->nchunks;
    info->chunk_samples = plan->chunk_samples;
    info->tail_subvolume = plan->layout.tail_sub;
    info->tail_chunk_samples = plan->layout.tail_chunk_samples;
    info->total_samples = plan->total;
    info->grid = plan->grid;
    info->block = bfi::kBlock;
    info->kernel = plan->shape->kernel;
    info->slot_len = 5 + 3 * plan->R;
    info->totals_len = 4 + 2 * plan->R;
    info->scratch_bytes = plan->scratch_bytes;
    info->ctas_per_sm_max = plan->per_sm_max;
    info->ctas_per_sm = plan->per_sm;
    return BFI_OK;
}

bfi_status bfi_plan_execute(bfi_plan *plan, const double *lo, const double *hi, const uint32_t *sub_id, uint32_t seed,
                            uint32_t job_id, double *slots, double *totals, void *stream) {
    if (!plan) return fail(BFI_E_INVALID, "plan is NULL");
    if (!lo || !hi || !slots || !totals) return fail(BFI_E_INVALID, "lo, hi, slots and totals must be non-NULL");
    DeviceGuard g(plan->device);
    if (g.err != cudaSuccess) return fail(BFI_E_CUDA, "cannot select device: %s", cudaGetErrorString(g.err));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plan->timing) BFI_CUDA(cudaEventRecord(plan->ev[0], st));
    BFI_CUDA(cudaMemsetAsync(plan->d_stats, 0, 4 * sizeof(unsigned long long), st));
    if (plan->nchunks > 0) {
        bfi::IntegrandArgs a{lo,           hi,           sub_id,        plan->d_samples,     plan->d_chunk_off,
                             plan->d_partials, plan->d_hint, plan->d_stats, plan->nsub, plan->nchunks,
                             plan->chunk_samples, plan->skip_window, plan->d_stats + 1, plan->d_stats + 2,
                             plan->d_stats + 3, plan->layout.tail_sub, plan->layout.tail_chunk_samples};
        if (plan->sampler == BFI_SAMPLE_BOX) {
            BFI_CUDA(plan->shape->integrand[plan->precision](a, plan->lat, seed, job_id, plan->grid, st));
        } else if (plan->sampler == BFI_SAMPLE_TRANSFORM && plan->shape->transform) {
            BFI_CUDA(plan->shape->transform(a, plan->lat, seed, job_id, plan->grid, st));
        } else {
            const bfi::MapArgs mp{plan->sampler, plan->d_map, plan->d_map ? plan->d_map + plan->d : nullptr};
            if (plan->sampler == BFI_SAMPLE_GAUSSIAN && plan->shape->gaussian)
                BFI_CUDA(plan->shape->gaussian(a, plan->lat, mp, plan->map_upper, seed, job_id, plan->grid, st));
            else
                BFI_CUDA(bfi::launch_mapped(a, plan->lat, mp, seed, job_id, plan->grid, st));
        }
    }
    if (plan->timing) BFI_CUDA(cudaEventRecord(plan->ev[1], st));
    bfi::MergeArgs m{lo, hi, plan->d_chunk_off, plan->d_partials, slots, plan->nsub, plan->R, plan->d,
                     plan->sampler == BFI_SAMPLE_GAUSSIAN ? 1 : 0, plan->log_norm};
    bfi::TotalsArgs t{slots, totals, plan->d_fbuf, plan->nsub, plan->R};
    BFI_CUDA(bfi::launch_merges(m, t, st));
    if (plan->timing) {
        BFI_CUDA(cudaEventRecord(plan->ev[2], st));
        plan->timed = true;
    }
    return BFI_OK;
}

bfi_status bfi_plan_set_grid(bfi_plan *plan, int32_t ctas_per_sm) {
    if (!plan) return fail(BFI_E_INVALID, "plan is NULL");
    if (ctas_per_sm < 0 || ctas_per_sm > plan->per_sm_max)
        return fail(BFI_E_INVALID, "ctas_per_sm = %d outside 0..%d", ctas_per_sm, plan->per_sm_max);
    const int per_sm = ctas_per_sm == 0 ? plan->per_sm_max : ctas_per_sm;
    plan->per_sm = per_sm;
    const int64_t resident = static_cast<int64_t>(plan->sms) * per_sm;
    plan->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(plan->nchunks, resident)));
    return BFI_OK;
}

bfi_status bfi_plan_set_sampler(bfi_plan *plan, const bfi_sampler *sampler) {
    if (!plan || !sampler) return fail(BFI_E_INVALID, "plan or sampler is NULL");
    const int kind = sampler->kind;
    if (kind != BFI_SAMPLE_BOX && kind != BFI_SAMPLE_TRANSFORM && kind != BFI_SAMPLE_GAUSSIAN)
        return fail(BFI_E_INVALID, "unknown sampler kind %d", kind);
    if (kind != BFI_SAMPLE_BOX && plan->precision != BFI_FP64)
        return fail(BFI_E_UNSUPPORTED, "the transform and Gaussian samplers run in FP64 only");
    const int d = plan->d;
    double log_norm = 0.0;
    if (kind == BFI_SAMPLE_GAUSSIAN) {
        if (d > bfi::kMaxGaussD)
            return fail(BFI_E_UNSUPPORTED, "the Gaussian sampler supports d <= %d (d = %d)", bfi::kMaxGaussD, d);
        if (!sampler->factor) return fail(BFI_E_INVALID, "the Gaussian sampler needs a factor");
        for (int k = 0; k < d * d; ++k)
            if (!std::isfinite(sampler->factor[k])) return fail(BFI_E_INVALID, "the factor has a non-finite entry");
        if (sampler->mean)
            for (int k = 0; k < d; ++k)
                if (!std::isfinite(sampler->mean[k])) return fail(BFI_E_INVALID, "the mean has a non-finite entry");
        // ln |det F| by Gaussian elimination with partial pivoting
        std::vector<double> a(sampler->factor, sampler->factor + d * d);
        double log_det = 0.0;
        for (int col = 0; col < d; ++col) {
            int piv = col;
            for (int r = col + 1; r < d; ++r)
                if (std::fabs(a[r * d + col]) > std::fabs(a[piv * d + col])) piv = r;
            const double pv = a[piv * d + col];
            if (pv == 0.0) return fail(BFI_E_INVALID, "the factor is singular");
            if (piv != col)
                for (int k = 0; k < d; ++k) std::swap(a[piv * d + k], a[col * d + k]);
            log_det += std::log(std::fabs(pv));
            for (int r = col + 1; r < d; ++r) {
                const double f = a[r * d + col] / pv;
                for (int k = col; k < d; ++k) a[r * d + k] -= f * a[col * d + k];
            }
        }
        log_norm = 0.5 * d * std::log(2.0 * M_PI) + log_det;
    }
    DeviceGuard g(plan->device);
    if (g.err != cudaSuccess) return fail(BFI_E_CUDA, "cannot select device: %s", cudaGetErrorString(g.err));
    int per_sm = 0;
    cudaError_t e;
    if (kind == BFI_SAMPLE_BOX)
        e = plan->shape->occupancy[plan->precision](plan->lat.nx, plan->lat.nt, &per_sm);
    else if (kind == BFI_SAMPLE_TRANSFORM && plan->shape->transform_occupancy)
        e = plan->shape->transform_occupancy(plan->lat.nx, plan->lat.nt, &per_sm);
    else if (kind == BFI_SAMPLE_GAUSSIAN && plan->shape->gaussian_occupancy)
        e = plan->shape->gaussian_occupancy(plan->lat.nx, plan->lat.nt, &per_sm);
    else
        e = bfi::occupancy_mapped(plan->lat.nx, plan->lat.nt, kind, &per_sm);
    if (e != cudaSuccess) return fail(BFI_E_CUDA, "occupancy query failed: %s", cudaGetErrorString(e));
    if (kind == BFI_SAMPLE_GAUSSIAN) {
        if (!plan->d_map && cudaMalloc(&plan->d_map, sizeof(double) * (d + d * d)) != cudaSuccess) {
            cudaGetLastError();
            plan->d_map = nullptr;
            return fail(BFI_E_NOMEM, "device allocation of the sampler failed");
        }
        std::vector<double> host(d + d * d, 0.0);
        if (sampler->mean) std::copy(sampler->mean, sampler->mean + d, host.begin());
        std::copy(sampler->factor, sampler->factor + d * d, host.begin() + d);
        BFI_CUDA(cudaMemcpy(plan->d_map, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice));
    }
    plan->sampler = kind;
    plan->log_norm = log_norm;
    plan->map_upper = false;
    if (kind == BFI_SAMPLE_GAUSSIAN) {
        bool upper = true;
        for (int r = 1; r < d && upper; ++r)
            for (int j = 0; j < r; ++j)
                if (sampler->factor[r * d + j] != 0.0) {
                    upper = false;
                    break;
                }
        plan->map_upper = upper;
    }
    plan->per_sm_max = per_sm > 0 ? per_sm : 1;
    plan->per_sm = plan->per_sm_max;
    const int64_t resident = static_cast<int64_t>(plan->sms) * plan->per_sm_max;
    plan->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(plan->nchunks, resident)));
    return BFI_OK;
}

bfi_status bfi_gaussian_proposal(const bfi_lattice *lattice, double zero_mode_sigma, double *factor) {
    bfi_status st = check_lattice(lattice);
    if (st != BFI_OK) return st;
    if (!factor) return fail(BFI_E_INVALID, "factor is NULL");
    if (!(zero_mode_sigma > 0.0)) return fail(BFI_E_INVALID, "zero_mode_sigma must be > 0 (inf: no regulator)");
    const int nx = lattice->nx, nt = lattice->nt, d = nx * nt;
    if (d > bfi::kMaxGaussD) return fail(BFI_E_UNSUPPORTED, "the Gaussian sampler supports d <= %d", bfi::kMaxGaussD);
    // B: the residual of Eq. (Gen2) without the advection term,
    // (B v)_j = v_next(j) - v_j + c_dif (2 v_j - v_right(j) - v_left(j))
    const double c_dif = lattice->nu * lattice->tau / (lattice->a * lattice->a);
    std::vector<double> B(static_cast<size_t>(d) * d, 0.0), A(static_cast<size_t>(d) * d, 0.0);
    for (int j = 0; j < d; ++j) {
        const int l = j % nt;
        const int nxt = l + 1 < nt ? j + 1 : j + 1 - nt;
        const int right = (j + nt) % d, left = (j - nt + d) % d;
        B[j * d + nxt] += 1.0;
        B[j * d + j] += 2.0 * c_dif - 1.0;
        B[j * d + right] -= c_dif;
        B[j * d + left] -= c_dif;
    }
    // A = B^T B / (D tau) + (mass2 + 1/sigma0^2) I, the quadratic form of the
    // linear-limit action S = v^T A v / 2 plus the regulator
    const double diag = lattice->mass2 + (std::isinf(zero_mode_sigma) ? 0.0 : 1.0 / (zero_mode_sigma * zero_mode_sigma));
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) acc += B[k * d + r] * B[k * d + c];
            A[r * d + c] = acc / (lattice->D * lattice->tau) + (r == c ? diag : 0.0);
        }
    // Cholesky A = L L^T, then F = L^-T (upper triangular): F F^T = A^-1
    std::vector<double> Lc(static_cast<size_t>(d) * d, 0.0);
    for (int j = 0; j < d; ++j) {
        double s2 = A[j * d + j];
        for (int k = 0; k < j; ++k) s2 -= Lc[j * d + k] * Lc[j * d + k];
        if (!(s2 > 0.0))
            return fail(BFI_E_INVALID, "the linear-limit action has a zero mode: give a finite zero_mode_sigma");
        const double ljj = std::sqrt(s2);
        Lc[j * d + j] = ljj;
        for (int i = j + 1; i < d; ++i) {
            double t = A[i * d + j];
            for (int k = 0; k < j; ++k) t -= Lc[i * d + k] * Lc[j * d + k];
            Lc[i * d + j] = t / ljj;
        }
    }
    // solve L^T F = I column by column (back substitution)
    for (int c = 0; c < d; ++c)
        for (int i = d - 1; i >= 0; --i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k < d; ++k) t -= Lc[k * d + i] * factor[k * d + c];
            factor[i * d + c] = t / Lc[i * d + i];
        }
    return BFI_OK;
}

bfi_status bfi_plan_set_timing(bfi_plan *plan, int enable) {
    if (!plan) return fail(BFI_E_INVALID, "plan is NULL");
    DeviceGuard g(plan->device);
    if (enable && !plan->ev[0])
        for (auto &e : plan->ev) BFI_CUDA(cudaEventCreate(&e));
    plan->timing = enable != 0;
    plan->timed = false;
    return BFI_OK;
}

bfi_status bfi_plan_get_stats(bfi_plan *plan, uint64_t *evaluated, float *skip_window) {
    if (!plan) return fail(BFI_E_INVALID, "plan is NULL");
    DeviceGuard g(plan->device);
    if (evaluated) {
        unsigned long long v = 0;
        BFI_CUDA(cudaMemcpy(&v, plan->d_stats, sizeof v, cudaMemcpyDeviceToHost));
        *evaluated = v;
    }
    if (skip_window) *skip_window = plan->skip_window;
    return BFI_OK;
}

// Counters of the last execution: [0] evaluated, [1] samples the full screen
// examined (kernels with the split compiled in), [2] samples of chunks that
// ran stage 1.
static bfi_status read_counters(bfi_plan *plan, unsigned long long (&c)[3]) {
    DeviceGuard g(plan->device);
    BFI_CUDA(cudaMemcpy(c, plan->d_stats, sizeof c, cudaMemcpyDeviceToHost));
    return BFI_OK;
}

bfi_status bfi_plan_get_screen_stats(bfi_plan *plan, uint64_t *screened, int32_t *two_stage) {
    if (!plan) return fail(BFI_E_INVALID, "plan is NULL");
    unsigned long long c[3] = {0, 0, 0};
    const bool box = plan->sampler == BFI_SAMPLE_BOX;
    if (box) {
        const bfi_status st = read_counters(plan, c);
        if (st != BFI_OK) return st;
    }
    const bool two = box && c[2] > 0;
    if (two_stage) *two_stage = two ? 1 : 0;
    if (screened) *screened = two ? static_cast<uint64_t>(c[1]) : static_cast<uint64_t>(plan->total);
    return BFI_OK;
}

bfi_status bfi_plan_get_work(bfi_plan *plan, bfi_work *work) {
    if (!plan || !work) return fail(BFI_E_INVALID, "plan or work is NULL");
    unsigned long long c[3] = {0, 0, 0};
    const bfi_status st = read_counters(plan, c);
    if (st != BFI_OK) return st;
    const uint64_t total = static_cast<uint64_t>(plan->total);
    work->samples = total;
    work->evaluated = c[0];
    if (plan->sampler != BFI_SAMPLE_BOX) {  // every sample evaluated, no screen
        work->stage1 = work->full_screen = work->survivors = 0;
    } else {
        work->stage1 = c[2];
        work->full_screen = total - c[2];
        work->survivors = plan->shape->two_stage ? c[1] - work->full_screen : 0;
    }
    work->two_stage_shape = plan->sampler == BFI_SAMPLE_BOX && plan->shape->two_stage ? 1 : 0;
    work->rest_screen = work->two_stage_shape && plan->lat.nt == 2 && plan->lat.nx % 2 == 0 &&
                        static_cast<float>(0.5 * plan->lat.mass2) == 0.f;
    return BFI_OK;
}

bfi_status bfi_plan_get_timing(bfi_plan *plan, float *ms) {
    if (!plan || !ms) return fail(BFI_E_INVALID, "plan or ms is NULL");
    if (!plan->timed) return fail(BFI_E_INVALID, "no timed execution yet");
    DeviceGuard g(plan->device);
    BFI_CUDA(cudaEventSynchronize(plan->ev[2]));
    BFI_CUDA(cudaEventElapsedTime(&ms[0], plan->ev[0], plan->ev[1]));
    BFI_CUDA(cudaEventElapsedTime(&ms[1], plan->ev[1], plan->ev[2]));
    return BFI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Context: one device, one stream, a cached plan and device buffers.
// ---------------------------------------------------------------------------
struct bfi_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::atomic<bool> busy{false};
    bfi_plan *plan = nullptr;
    bfi_lattice lat{};
    bfi_precision precision = BFI_FP64;
    double *d_lo = nullptr, *d_hi = nullptr, *d_slots = nullptr, *d_totals = nullptr;
    uint32_t *d_sid = nullptr;
    size_t cap_lo = 0, cap_hi = 0, cap_sid = 0, cap_slots = 0, cap_totals = 0;
    int32_t sampler = BFI_SAMPLE_BOX;         // applied to every plan the context makes
    std::vector<double> map_mean, map_factor;
};

namespace {

bool same_lattice(const bfi_lattice &a, const bfi_lattice &b) { return std::memcmp(&a, &b, sizeof a) == 0; }

template <typename T>
bfi_status grow(T *&ptr, size_t &cap, size_t need) {
    if (need <= cap) return BFI_OK;
    cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    if (cudaMalloc(&ptr, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(BFI_E_NOMEM, "device allocation of %zu bytes failed", need * sizeof(T));
    }
    cap = need;
    return BFI_OK;
}

struct BusyGuard {
    std::atomic<bool> &flag;
    bool ok;
    explicit BusyGuard(std::atomic<bool> &f) : flag(f) {
        bool expected = false;
        ok = flag.compare_exchange_strong(expected, true);
    }
    ~BusyGuard() {
        if (ok) flag.store(false);
    }
};

}  // namespace

extern "C" {

bfi_status bfi_ctx_create(bfi_ctx **out, int device) {
    if (!out) return fail(BFI_E_INVALID, "out is NULL");
    *out = nullptr;
    DeviceGuard g(device);
    if (g.err != cudaSuccess) return fail(BFI_E_CUDA, "cannot select device %d: %s", device, cudaGetErrorString(g.err));
    bfi_ctx *c = new (std::nothrow) bfi_ctx();
    if (!c) return fail(BFI_E_NOMEM, "host allocation failed");
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return fail(BFI_E_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return BFI_OK;
}

bfi_status bfi_ctx_destroy(bfi_ctx *ctx) {
    if (!ctx) return BFI_OK;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        bfi_plan_destroy(ctx->plan);
        cudaFree(ctx->d_lo);
        cudaFree(ctx->d_hi);
        cudaFree(ctx->d_sid);
        cudaFree(ctx->d_slots);
        cudaFree(ctx->d_totals);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
    return BFI_OK;
}

bfi_status bfi_ctx_set_sampler(bfi_ctx *ctx, const bfi_sampler *sampler, int32_t d) {
    if (!ctx || !sampler) return fail(BFI_E_INVALID, "ctx or sampler is NULL");
    BusyGuard busy(ctx->busy);
    if (!busy.ok) return fail(BFI_E_BUSY, "context is in use by another thread");
    const int kind = sampler->kind;
    if (kind != BFI_SAMPLE_BOX && kind != BFI_SAMPLE_TRANSFORM && kind != BFI_SAMPLE_GAUSSIAN)
        return fail(BFI_E_INVALID, "unknown sampler kind %d", kind);
    ctx->map_mean.clear();
    ctx->map_factor.clear();
    if (kind == BFI_SAMPLE_GAUSSIAN) {
        if (d < 1 || d > bfi::kMaxGaussD || !sampler->factor)
            return fail(BFI_E_INVALID, "the Gaussian sampler needs 1 <= d <= %d and a factor", bfi::kMaxGaussD);
        ctx->map_factor.assign(sampler->factor, sampler->factor + static_cast<size_t>(d) * d);
        if (sampler->mean) ctx->map_mean.assign(sampler->mean, sampler->mean + d);
    }
    ctx->sampler = kind;
    // the next integration re-plans with the sampler
    bfi_plan_destroy(ctx->plan);
    ctx->plan = nullptr;
    return BFI_OK;
}

bfi_status bfi_integrate(bfi_ctx *ctx, const bfi_lattice *lattice, int64_t nsub, const double *lo, const double *hi,
                         const uint64_t *samples, const uint32_t *sub_id, uint32_t seed, uint32_t job_id,
                         bfi_precision precision, double *slots, double *totals) {
    if (!ctx) return fail(BFI_E_INVALID, "ctx is NULL");
    BusyGuard busy(ctx->busy);
    if (!busy.ok) return fail(BFI_E_BUSY, "context is in use by another thread");
    bfi_status st = check_lattice(lattice);
    if (st != BFI_OK) return st;
    if (!lo || !hi || !samples || !totals) return fail(BFI_E_INVALID, "lo, hi, samples and totals must be non-NULL");
    if (nsub < 1) return fail(BFI_E_INVALID, "nsub must be >= 1");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return fail(BFI_E_CUDA, "cannot select device: %s", cudaGetErrorString(g.err));

    bool replan = !ctx->plan || !same_lattice(ctx->lat, *lattice) || ctx->precision != precision ||
                  ctx->plan->nsub != nsub ||
                  std::memcmp(ctx->plan->samples.data(), samples, sizeof(uint64_t) * nsub) != 0;
    if (replan) {
        bfi_plan_destroy(ctx->plan);
        ctx->plan = nullptr;
        st = bfi_plan_create(&ctx->plan, lattice, nsub, samples, precision, ctx->device);
        if (st != BFI_OK) return st;
        ctx->lat = *lattice;
        ctx->precision = precision;
        if (ctx->sampler != BFI_SAMPLE_BOX) {
            const bool gauss = ctx->sampler == BFI_SAMPLE_GAUSSIAN;
            if (gauss && ctx->map_factor.size() != static_cast<size_t>(ctx->plan->d) * ctx->plan->d) {
                bfi_plan_destroy(ctx->plan);
                ctx->plan = nullptr;
                return fail(BFI_E_INVALID, "the context's Gaussian sampler was set for another dimension");
            }
            const bfi_sampler smp{ctx->sampler, gauss && !ctx->map_mean.empty() ? ctx->map_mean.data() : nullptr,
                                  gauss ? ctx->map_factor.data() : nullptr};
            st = bfi_plan_set_sampler(ctx->plan, &smp);
            if (st != BFI_OK) {
                bfi_plan_destroy(ctx->plan);
                ctx->plan = nullptr;
                return st;
            }
        }
    }
    const int d = lattice->nx * lattice->nt;
    const size_t nbox = static_cast<size_t>(nsub) * d;
    const size_t nslot = static_cast<size_t>(nsub) * bfi_slot_len(lattice->nx);
    if ((st = grow(ctx->d_lo, ctx->cap_lo, nbox)) != BFI_OK) return st;
    if ((st = grow(ctx->d_hi, ctx->cap_hi, nbox)) != BFI_OK) return st;
    if (sub_id && (st = grow(ctx->d_sid, ctx->cap_sid, static_cast<size_t>(nsub))) != BFI_OK) return st;
    if ((st = grow(ctx->d_slots, ctx->cap_slots, nslot)) != BFI_OK) return st;
    if ((st = grow(ctx->d_totals, ctx->cap_totals, static_cast<size_t>(bfi_totals_len(lattice->nx)))) != BFI_OK)
        return st;

    cudaStream_t s = ctx->stream;
    BFI_CUDA(cudaMemcpyAsync(ctx->d_lo, lo, nbox * sizeof(double), cudaMemcpyHostToDevice, s));
    BFI_CUDA(cudaMemcpyAsync(ctx->d_hi, hi, nbox * sizeof(double), cudaMemcpyHostToDevice, s));
    if (sub_id) BFI_CUDA(cudaMemcpyAsync(ctx->d_sid, sub_id, nsub * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    st = bfi_plan_execute(ctx->plan, ctx->d_lo, ctx->d_hi, sub_id ? ctx->d_sid : nullptr, seed, job_id, ctx->d_slots,
                          ctx->d_totals, s);
    if (st != BFI_OK) return st;
    if (slots) BFI_CUDA(cudaMemcpyAsync(slots, ctx->d_slots, nslot * sizeof(double), cudaMemcpyDeviceToHost, s));
    BFI_CUDA(cudaMemcpyAsync(totals, ctx->d_totals, bfi_totals_len(lattice->nx) * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    BFI_CUDA(cudaStreamSynchronize(s));
    return BFI_OK;
}

// ---------------------------------------------------------------------------
// Host FP64 merge: the same definitions as the device merge (merge_totals).
// ---------------------------------------------------------------------------
bfi_status bfi_merge_host(int32_t nx, int64_t nsub, const double *slots, double *totals) {
    if (nx < 2 || nsub < 0 || !slots || !totals) return fail(BFI_E_INVALID, "bad arguments to bfi_merge_host");
    const int R = num_r(nx), SL = 5 + 3 * R;
    auto usable = [&](const double *q) { return q[0] > 0.0 && q[3] > 0.0; };
    double L = -INFINITY, n_tot = 0.0, used = 0.0;
    bool inf_err = false;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (q[0] <= 0.0) continue;
        n_tot += q[0];
        used += 1.0;
        if (q[3] > 0.0) L = std::fmax(L, q[2] - std::log(q[0]) - q[1]);
    }
    // f_s and g_s = f_s^2 / (n_s - 1), the factor of every variance term (the
    // same arithmetic as the device merge)
    std::vector<double> f(static_cast<size_t>(nsub), 0.0), g(static_cast<size_t>(nsub), 0.0);
    double Z = 0.0, VZ = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (!usable(q)) continue;
        const double n = q[0];
        f[s] = std::exp(q[2] - std::log(n) - q[1] - L);
        Z += f[s] * q[3];
        if (n < 2.0) {
            inf_err = true;
            continue;
        }
        g[s] = f[s] * f[s] / (n - 1.0);
        VZ += g[s] * (n * q[4] - q[3] * q[3]);
    }
    totals[0] = L + std::log(Z);
    totals[1] = inf_err ? INFINITY : std::sqrt(VZ > 0.0 ? VZ : 0.0) / Z;
    totals[2] = n_tot;
    totals[3] = used;
    for (int r = 0; r < R; ++r) {
        double N = 0.0;
        for (int64_t s = 0; s < nsub; ++s)
            if (usable(slots + s * SL)) N += f[s] * slots[s * SL + 5 + r];
        const double C = N / Z;
        double V = 0.0;
        for (int64_t s = 0; s < nsub; ++s) {
            if (g[s] == 0.0) continue;
            const double *q = slots + s * SL;
            const double n = q[0];
            const double vN = n * q[5 + 2 * R + r] - q[5 + r] * q[5 + r];
            const double cov = n * q[5 + R + r] - q[3] * q[5 + r];
            const double vZ = n * q[4] - q[3] * q[3];
            V += g[s] * (vN - 2.0 * C * cov + C * C * vZ);
        }
        totals[4 + r] = C;
        totals[4 + R + r] = inf_err ? INFINITY : std::sqrt(V > 0.0 ? V : 0.0) / Z;
    }
    return BFI_OK;
}

// ---------------------------------------------------------------------------
// Stated arithmetic error of a result (box sampler).  Every step an evaluated
// sample goes through has a rounding bound; their first-order sum bounds how
// far the library's Z and C(r) can lie from the same estimator evaluated in
// exact arithmetic on the same points (FP32 mode: the same float points), to
// which the negligible-weight truncation adds at most e^-c.  u is the unit
// roundoff (2^-24 in FP32, 2^-53 in FP64).  With T a bound on the magnitude
// of each of the three terms of a residual (from vmax and the lattice
// constants), inv = 1/(2 D tau), and S_hi a bound on the action of a sample
// that can carry weight (the records' largest shift plus the window W):
//   action   |dS| <= 2 k u_a T sqrt(d S_hi inv) + (d + 1) u_a S_hi, with k
//            operations per residual of relative error u_a each (FP32: the
//            compensated action, k = 8, u_a = 2^-46; FP64: k = 4, u_a = u),
//            plus (d + 1) u_a times the mass term
//   weight   exp's error (CUDA documents expf at 2 ulp and exp at 1 ulp) plus
//            the argument's rounding (FP32: the split a_h + a_l is exact and
//            the first-order correction one fma, u (1 + 2^-18); FP64:
//            u |m - S| <= u (W + 17)) plus |dS|
//   products FP32: Dot2 kept as hi + lo, 2 (d u)^2 Q_0, then w Q_r =
//            fma(w, hi, w lo), one rounding; FP64: the FMA chain, gamma_d Q_0
//            (|Q_r| <= Q_0 by Cauchy-Schwarz), then w Q_r, one rounding
//   sums     per thread (at most N_t terms per chunk): FP32 Kahan 2u + N_t u^2,
//            FP64 plain (N_t - 1) u; then the FP64 merges of threads, chunks
//            and subvolumes, 2^-53 (64 + 4 chunks + 4 nsub); in FP32 the
//            chunk record first adds each lane's 8 threads in double-float
//            (16 exactly scaled terms), 2^-42 more
//   dropped  e^-c of Z (c = 20 in FP32, 34 in FP64); of N(r), e^-c vmax^2 Z,
//            since |P_r| <= vmax^2
// Z: b_Z = weight + sums + merges + e^-c.  N(r) relative to N(0): b_N =
// weight + products + sums + merges + e^-c vmax^2 / C(0).  C(r) = N(r)/Z
// relative to C(0): b_N (1 + b_Z) + b_Z (1 + b_Z).
// ---------------------------------------------------------------------------
bfi_status bfi_error_bound(const bfi_lattice *lattice, bfi_precision precision, int64_t nsub, const double *slots,
                           double vmax, double *bound) {
    bfi_status st = check_lattice(lattice);
    if (st != BFI_OK) return st;
    if (precision != BFI_FP64 && precision != BFI_FP32) return fail(BFI_E_INVALID, "unknown precision %d", precision);
    if (nsub < 1 || !slots || !bound) return fail(BFI_E_INVALID, "nsub must be >= 1 and slots, bound non-NULL");
    if (!std::isfinite(vmax) || vmax <= 0.0) return fail(BFI_E_INVALID, "vmax must be finite and > 0");
    const int nx = lattice->nx, R = num_r(nx), SL = 5 + 3 * R;
    const double d = static_cast<double>(nx) * lattice->nt;
    std::vector<double> tot(static_cast<size_t>(4 + 2 * R));
    if ((st = bfi_merge_host(nx, nsub, slots, tot.data())) != BFI_OK) return st;
    double m_hi = -INFINITY, n_max = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (q[0] <= 0.0) continue;
        n_max = std::fmax(n_max, q[0]);
        if (q[3] > 0.0) m_hi = std::fmax(m_hi, q[1]);
    }
    const double C0 = tot[4];
    if (!std::isfinite(m_hi) || !(C0 > 0.0)) return fail(BFI_E_INVALID, "the records carry no weight");
    const bfi::ShapeKernels *shape = bfi::find_shape(nx, lattice->nt);
    const bool f32 = precision == BFI_FP32;
    const double u = f32 ? 0x1p-24 : 0x1p-53;
    const double c_adv = lattice->nonlinear * lattice->tau / (2.0 * lattice->a);
    const double c_dif = lattice->nu * lattice->tau / (lattice->a * lattice->a);
    const double k1 = 2.0 * c_dif - 1.0, inv = 1.0 / (2.0 * lattice->D * lattice->tau);
    const double T = vmax * (1.0 + std::fabs(k1) + 2.0 * std::fabs(c_adv) * vmax) + 2.0 * std::fabs(c_dif) * vmax;
    const double c = f32 ? 20.0 : 34.0;
    const double W = c + std::log(std::fmax(n_max, 1.0));
    const double S_hi = 1.001 * (std::fmax(m_hi, 0.0) + 1.0) + W + 2.0;
    const double ua = f32 ? 0x1p-46 : u, k = f32 ? 8.0 : 4.0;
    double dS = 2.0 * k * ua * T * std::sqrt(d * S_hi * inv) + (d + 1.0) * ua * S_hi;
    if (lattice->mass2 > 0.0) dS += (d + 1.0) * ua * 0.5 * lattice->mass2 * d * vmax * vmax;
    const double e_w = (f32 ? 0x1p-22 : 0x1p-52) + (f32 ? u * (1.0 + 0x1p-18) : u * (W + 17.0)) + dS;
    const double e_q = (f32 ? 2.0 * (d * u) * (d * u) : d * u / (1.0 - d * u)) + u;
    // terms per per-thread (per-warp in the warp-per-sample kernel) sum in one
    // chunk: at most 2048 rows per thread
    const double n_t = shape && shape->kernel == 0 ? 2048.0 : 2048.0 * bfi::kBlock / 4.0;
    const double e_sum = f32 ? 2.0 * u + n_t * u * u : (n_t - 1.0) * u;
    const double e_merge = 0x1p-53 * (64.0 + 4.0 * std::ceil(n_max / 1024.0) + 4.0 * static_cast<double>(nsub)) +
                           (f32 ? 0x1p-42 : 0.0);
    const double drop = std::exp(-c);
    const double bz = e_w + e_sum + e_merge + drop;
    const double bn = e_w + e_q + e_sum + e_merge + drop * vmax * vmax / C0;
    bound[0] = bz;
    for (int r = 0; r < R; ++r) bound[1 + r] = bn * (1.0 + bz) + bz * (1.0 + bz);
    return BFI_OK;
}

// ---------------------------------------------------------------------------
// Single steps.
// ---------------------------------------------------------------------------
bfi_status bfi_points(int32_t d, const double *lo, const double *hi, uint32_t sub_id, uint32_t seed, uint32_t job_id,
                      uint64_t first, int64_t count, bfi_precision precision, double *y, void *stream) {
    if (d < 1 || d > bfi::kMaxD || count < 0 || !lo || !hi || (count > 0 && !y))
        return fail(BFI_E_INVALID, "bad arguments to bfi_points");
    if (precision != BFI_FP64 && precision != BFI_FP32) return fail(BFI_E_INVALID, "unknown precision");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bfi::PointsArgs a{lo, hi, y, first, count, d, sub_id};
    BFI_CUDA(bfi::launch_points(a, precision == BFI_FP32, seed, job_id, st));
    BFI_CUDA(cudaStreamSynchronize(st));
    return BFI_OK;
}

bfi_status bfi_eval(const bfi_lattice *lattice, int64_t npts, const double *y, bfi_precision precision, double *S,
                    double *P, void *stream) {
    bfi_status st = check_lattice(lattice);
    if (st != BFI_OK) return st;
    if (npts < 0 || (npts > 0 && (!y || !S || !P))) return fail(BFI_E_INVALID, "bad arguments to bfi_eval");
    if (precision != BFI_FP64 && precision != BFI_FP32 && precision != BFI_FP32_COMPENSATED)
        return fail(BFI_E_INVALID, "unknown precision");
    const bfi::ShapeKernels *shape = bfi::find_shape(lattice->nx, lattice->nt);
    if (!shape)
        return fail(BFI_E_UNSUPPORTED, "lattice %dx%d has no compiled kernel in this library", lattice->nx,
                    lattice->nt);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    bfi::EvalArgs a{y, S, P, npts};
    BFI_CUDA(shape->eval(a, to_params(lattice), static_cast<int>(precision), cs));
    BFI_CUDA(cudaStreamSynchronize(cs));
    return BFI_OK;
}

}  // extern "C"
