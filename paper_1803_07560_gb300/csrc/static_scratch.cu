// static_scratch.cu -- bfi_integrate_static_scratch: the whole integration
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host
// application whose memory manager owns the device heap and forbids other
// allocations, or a latency-critical loop where an allocation (and the device
// synchronisation it may imply) is not allowed after start-up.  For them this
// file keeps the scratch the integration needs (chunk table, per-chunk partial
// records, per-subvolume hints and merge factors, the evaluated-samples
// counter) in one
// file-scope device array of fixed size, so a call allocates nothing; the
// caller still passes its own inputs and outputs.  The kernels are the same
// ones bfi_plan_execute runs.
#include "bfi.h"
#include "bfi_host.h"
#include "bfi_kernels.h"

#include <cstdio>
#include <mutex>

namespace {

// The scratch: 16 MiB on every device that loads the library, held until the
// process exits.  In host code 'g_scratch' is only a stand-in for the device
// array, never a device address: kernels get the address obtained from
// cudaGetSymbolAddress on that device (scratch_address below).
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_address[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (the first call on a device does this set-up) and kept for the
// process: a cudaDeviceReset of that device (which unloads the module holding
// the array) invalidates it, so the entry point must not be used across one.
bfi_status scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return bfi::set_error(BFI_E_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_address[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch failed: %s",
                          cudaGetErrorString(e));
            return bfi::set_error(BFI_E_CUDA, msg);
        }
        g_address[device] = p;
    }
    *out = g_address[device];
    return BFI_OK;
}

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

// Chunk table from the budgets already copied into the scratch: subvolume s
// owns chunks [off[s], off[s+1]), ceil(n_s / chunk_samples) of them.  One
// CTA: each thread sums a contiguous range, thread 0 scans the partials in
// order, then every thread writes its range.
constexpr int kScanThreads = 256;

__global__ void __launch_bounds__(kScanThreads) chunk_table(const uint64_t *samples, int64_t nsub,
                                                            bfi::ChunkLayout layout, int64_t *off) {
    __shared__ int64_t part[kScanThreads];
    const int t = threadIdx.x;
    const int64_t per = (nsub + kScanThreads - 1) / kScanThreads;
    const int64_t b = min(nsub, t * per), e = min(nsub, b + per);
    auto chunks_of = [&](int64_t s) {
        const uint64_t c = static_cast<uint64_t>(s >= layout.tail_sub ? layout.tail_chunk_samples : layout.chunk_samples);
        return static_cast<int64_t>((samples[s] + c - 1) / c);
    };
    int64_t sum = 0;
    for (int64_t s = b; s < e; ++s) sum += chunks_of(s);
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < kScanThreads; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        off[nsub] = run;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t s = b; s < e; ++s) {
        off[s] = run;
        run += chunks_of(s);
    }
}

bfi_status cuda_fail(const char *what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s failed: %s", what, cudaGetErrorString(e));
    return bfi::set_error(BFI_E_CUDA, msg);
}

}  // namespace

extern "C" bfi_status bfi_integrate_static_scratch(const bfi_lattice *lattice, int64_t nsub, const uint64_t *samples,
                                                   const double *lo, const double *hi, const uint32_t *sub_id,
                                                   uint32_t seed, uint32_t job_id, bfi_precision precision,
                                                   double *slots, double *totals, void *stream) {
    bfi_status st = bfi::validate_lattice(lattice);
    if (st != BFI_OK) return st;
    if (nsub < 1 || !samples || !lo || !hi || !slots || !totals)
        return bfi::set_error(BFI_E_INVALID, "nsub must be >= 1 and samples, lo, hi, slots, totals non-NULL");
    if (precision != BFI_FP64 && precision != BFI_FP32) return bfi::set_error(BFI_E_INVALID, "unknown precision");
    const bfi::ShapeKernels *shape = bfi::find_shape(lattice->nx, lattice->nt);
    if (!shape) return bfi::set_error(BFI_E_UNSUPPORTED, "lattice shape has no compiled kernel in this library");

    // Sizes, checked against the fixed scratch before anything touches the device.
    uint64_t total = 0, n_max = 1;
    for (int64_t s = 0; s < nsub; ++s) {
        if (samples[s] >= (1ull << 48)) return bfi::set_error(BFI_E_INVALID, "a sample budget is >= 2^48");
        total += samples[s];
        n_max = samples[s] > n_max ? samples[s] : n_max;
    }
    if (total >= (1ull << 62)) return bfi::set_error(BFI_E_INVALID, "total sample budget too large");
    const int R = lattice->nx / 2 + 1, K = 2 + 3 * R, d = lattice->nx * lattice->nt;
    const bfi::ChunkLayout layout = bfi::plan_chunk_layout(samples, nsub);
    int64_t nchunks = 0;
    for (int64_t s = 0; s < nsub; ++s) nchunks += layout.chunks_of(s, samples[s]);
    const size_t off_bytes = round_up(sizeof(int64_t) * (nsub + 1));
    const size_t smp_bytes = round_up(sizeof(uint64_t) * nsub);
    const size_t hint_bytes = round_up(sizeof(float) * nsub);
    const size_t stat_bytes = round_up(2 * sizeof(unsigned long long));  // evaluated, next chunk
    const size_t fbuf_bytes = round_up(sizeof(double) * 2 * nsub);
    const size_t par_bytes = round_up(sizeof(double) * static_cast<size_t>(nchunks > 0 ? nchunks : 1) * (K + 2));
    const size_t need = off_bytes + smp_bytes + hint_bytes + stat_bytes + fbuf_bytes + par_bytes;
    if (need > kStaticScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "job needs %zu bytes of scratch (%lld chunk records); the static scratch holds %zu bytes",
                      need, static_cast<long long>(nchunks), kStaticScratchBytes);
        return bfi::set_error(BFI_E_INVALID, msg);
    }

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    void *base = nullptr;
    if ((st = scratch_address(device, &base)) != BFI_OK) return st;
    unsigned char *p = static_cast<unsigned char *>(base);
    int64_t *d_off = reinterpret_cast<int64_t *>(p);
    uint64_t *d_samples = reinterpret_cast<uint64_t *>(p + off_bytes);
    float *d_hint = reinterpret_cast<float *>(p + off_bytes + smp_bytes);
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(p + off_bytes + smp_bytes + hint_bytes);
    double *d_fbuf = reinterpret_cast<double *>(p + off_bytes + smp_bytes + hint_bytes + stat_bytes);
    double *d_partials = reinterpret_cast<double *>(p + off_bytes + smp_bytes + hint_bytes + stat_bytes + fbuf_bytes);

    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return cuda_fail("cudaDeviceGetAttribute", e);
    if ((e = shape->occupancy[precision](lattice->nx, lattice->nt, &per_sm)) != cudaSuccess) return cuda_fail("occupancy query", e);
    int64_t grid = static_cast<int64_t>(sms) * (per_sm > 0 ? per_sm : 1);
    grid = grid < nchunks ? grid : (nchunks > 0 ? nchunks : 1);

    // Everything below is ordered on 'stream'.  The two counters must start
    // at zero; every other scratch word is written before it is read.
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(d_samples, samples, sizeof(uint64_t) * nsub, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
        return cuda_fail("copy of the budgets", e);
    if ((e = cudaMemsetAsync(d_stats, 0, 2 * sizeof(unsigned long long), cs)) != cudaSuccess)
        return cuda_fail("clearing the counters", e);
    chunk_table<<<1, kScanThreads, 0, cs>>>(d_samples, nsub, layout, d_off);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("chunk table launch", e);
    const bfi::LatticeParams lp{lattice->nx, lattice->nt, lattice->nu, lattice->D,
                                lattice->a,  lattice->tau, lattice->nonlinear, lattice->mass2};
    if (nchunks > 0) {
        bfi::IntegrandArgs a{lo,         hi,     sub_id, d_samples, d_off,         d_partials,
                             d_hint,     d_stats, nsub,  nchunks,   layout.chunk_samples, bfi::plan_negligible_window(precision, n_max),
                             nullptr,    nullptr, d_stats + 1, layout.tail_sub, layout.tail_chunk_samples};
        if ((e = shape->integrand[precision](a, lp, seed, job_id, static_cast<int>(grid), cs)) != cudaSuccess)
            return cuda_fail("integrand launch", e);
    }
    const bfi::MergeArgs m{lo, hi, d_off, d_partials, slots, nsub, R, d, 0, 0.0};
    const bfi::TotalsArgs t{slots, totals, d_fbuf, nsub, R};
    if ((e = bfi::launch_merges(m, t, cs)) != cudaSuccess) return cuda_fail("merge launch", e);
    return BFI_OK;
}
