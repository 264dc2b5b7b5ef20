// nsphere.cu -- the test integrand of Sec. 3 (Listings 1-2) on the GPU:
// f(x) = sqrt(max(0, 1 - |x|^2)) over a box, plain Monte Carlo with the same
// Philox points as the lattice integrand (FP64 points), result V mean f, error
// V sigma / sqrt(n), and the split suggestion of the line protocol: the
// coordinate j with the largest |sum_{x_j < mid} f - sum_{x_j >= mid} f|.
#include "bfi.h"
#include "bfi_device.cuh"
#include "bfi_host.h"

#include <cmath>
#include <cstdio>

namespace {

constexpr int kNsBlock = 128;
constexpr int kNsMaxDims = 32;

struct NsArgs {
    double lo[kNsMaxDims], w[kNsMaxDims], mid[kNsMaxDims];
    uint64_t n;
    int dims;
    uint32_t sub_id;
};

// Per block: [sum f, sum f^2, sum_{x_j < mid} f for each j] in FP64, reduced
// in a fixed order into out[block * (2 + dims)].
__global__ void __launch_bounds__(kNsBlock) nsphere_kernel(const NsArgs a, const bfi::RoundKeys rk, double *out) {
    __shared__ double s[(2 + kNsMaxDims) * kNsBlock];
    const int t = threadIdx.x;
    const int W = 2 + a.dims;
    for (int k = 0; k < W; ++k) s[k * kNsBlock + t] = 0.0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kNsBlock;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(kNsBlock) + t; i < a.n; i += stride) {
        // |x|^2 in coordinate order with separate rounding, and a bit per
        // coordinate for the half of the box the point falls in
        double r2 = 0.0;
        uint32_t below = 0u;
        for (int q = 0; 4 * q < a.dims; ++q) {
            const uint4 b = bfi::philox4x32_10(
                make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), a.sub_id), rk);
            const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 4 * q + u;
                if (j < a.dims) {
                    const double x = bfi::Coord<double>::map(w4[u], a.lo[j], a.w[j]);
                    r2 = __dadd_rn(r2, __dmul_rn(x, x));
                    below |= static_cast<uint32_t>(x < a.mid[j]) << j;
                }
            }
        }
        const double f = r2 < 1.0 ? sqrt(1.0 - r2) : 0.0;
        s[t] += f;
        s[kNsBlock + t] += f * f;
        for (; below; below &= below - 1u) s[(2 + __ffs(below) - 1) * kNsBlock + t] += f;
    }
    __syncthreads();
    for (int off = kNsBlock / 2; off > 0; off >>= 1) {
        if (t < off)
            for (int k = 0; k < W; ++k) s[k * kNsBlock + t] += s[k * kNsBlock + t + off];
        __syncthreads();
    }
    if (t < W) out[blockIdx.x * W + t] = s[t * kNsBlock];
}

// Sums the block records in block order.
__global__ void nsphere_sum(const double *in, int blocks, int W, double *out) {
    const int k = threadIdx.x;
    if (k >= W) return;
    double v = 0.0;
    for (int b = 0; b < blocks; ++b) v += in[b * W + k];
    out[k] = v;
}

bfi_status cuda_fail(const char *what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s failed: %s", what, cudaGetErrorString(e));
    return bfi::set_error(BFI_E_CUDA, msg);
}

}  // namespace

extern "C" bfi_status bfi_nsphere(int32_t dims, const double *lo, const double *hi, uint64_t n, uint32_t seed,
                                  uint32_t job_id, uint32_t sub_id, double *result, double *abs_err,
                                  int32_t *split_dim, int device) {
    if (dims < 1 || dims > kNsMaxDims || !lo || !hi || !result || !abs_err || n < 2)
        return bfi::set_error(BFI_E_INVALID, "need 1 <= dims <= 32, n >= 2 and non-NULL arrays");
    NsArgs a{};
    a.n = n;
    a.dims = dims;
    a.sub_id = sub_id;
    double vol = 1.0;
    for (int j = 0; j < dims; ++j) {
        if (!(hi[j] > lo[j])) return bfi::set_error(BFI_E_INVALID, "need lo < hi in every coordinate");
        a.lo[j] = lo[j];
        a.w[j] = hi[j] - lo[j];
        a.mid[j] = 0.5 * (lo[j] + hi[j]);
        vol *= a.w[j];
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nsphere_kernel, kNsBlock, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int blocks = sms * per_sm, W = 2 + dims;  // one resident wave
    double *buf = nullptr;
    e = cudaMalloc(&buf, sizeof(double) * (static_cast<size_t>(blocks) * W + W));
    if (e != cudaSuccess) {
        if (prev >= 0) cudaSetDevice(prev);
        return cuda_fail("cudaMalloc", e);
    }
    nsphere_kernel<<<blocks, kNsBlock>>>(a, bfi::make_round_keys(seed, job_id), buf);
    nsphere_sum<<<1, 64>>>(buf, blocks, W, buf + static_cast<size_t>(blocks) * W);
    double sums[2 + kNsMaxDims];
    e = cudaMemcpy(sums, buf + static_cast<size_t>(blocks) * W, sizeof(double) * W, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail("nsphere", e);
    const double nn = static_cast<double>(n), sf = sums[0], sf2 = sums[1];
    *result = vol * sf / nn;
    *abs_err = vol * std::sqrt((sf2 - sf * sf / nn) / (nn - 1.0) / nn);
    if (split_dim) {
        int best = 0;
        double gap_best = -1.0;
        for (int j = 0; j < dims; ++j) {
            const double gap = std::fabs(sums[2 + j] - (sf - sums[2 + j]));
            if (gap > gap_best) {
                gap_best = gap;
                best = j;
            }
        }
        *split_dim = best;
    }
    return BFI_OK;
}
