// nsphere.cu -- the test integrand of Sec. 3 (Listings 1-2) on the GPU:
// f(x) = sqrt(max(0, 1 - |x|^2)) over boxes, plain Monte Carlo with the same
// Philox points as the lattice integrand (FP64 points), result V mean f, error
// V sigma / sqrt(n), and the split suggestion of the line protocol: the
// coordinate j with the largest |sum_{x_j < mid} f - sum_{x_j >= mid} f|.
// Many boxes go in one launch (a round of the adaptive driver); bfi_nsphere is
// a batch of one.
#include "bfi.h"
#include "bfi_device.cuh"
#include "bfi_host.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

namespace {

constexpr int kNsBlock = 128;
constexpr int kNsMaxDims = 32;

struct NsBoxes {
    const double *lo, *w, *mid;  // [nbox][dims]
    const uint64_t *n;           // [nbox]
    const uint32_t *sub_id;      // [nbox]
    int dims;
    int gx;                      // blocks per box
};

// Block (box, bx) of box*gx + bx sums [f, f^2, f over x_j < mid_j for each j]
// over samples bx*128 + t, stepping by gx*128, in FP64, and reduces them in a
// fixed order into partial[(box*gx + bx) * (2 + dims)].
__global__ void __launch_bounds__(kNsBlock) nsphere_kernel(const NsBoxes b, const bfi::RoundKeys rk, double *partial) {
    __shared__ double s[(2 + kNsMaxDims) * kNsBlock];
    __shared__ double s_lo[kNsMaxDims], s_w[kNsMaxDims], s_mid[kNsMaxDims];
    const int t = threadIdx.x;
    const int W = 2 + b.dims;
    const int box = blockIdx.x / b.gx, bx = blockIdx.x % b.gx;
    if (t < b.dims) {
        s_lo[t] = b.lo[box * b.dims + t];
        s_w[t] = b.w[box * b.dims + t];
        s_mid[t] = b.mid[box * b.dims + t];
    }
    for (int k = 0; k < W; ++k) s[k * kNsBlock + t] = 0.0;
    __syncthreads();
    const uint64_t n = b.n[box];
    const uint32_t sub = b.sub_id[box];
    const uint64_t stride = static_cast<uint64_t>(b.gx) * kNsBlock;
    for (uint64_t i = static_cast<uint64_t>(bx) * kNsBlock + t; i < n; i += stride) {
        // |x|^2 in coordinate order with separate rounding, and a bit per
        // coordinate for the half of the box the point falls in
        double r2 = 0.0;
        uint32_t below = 0u;
        for (int q = 0; 4 * q < b.dims; ++q) {
            const uint4 c = bfi::philox4x32_10(
                make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), sub), rk);
            const uint32_t w4[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 4 * q + u;
                if (j < b.dims) {
                    const double x = bfi::Coord<double>::map(w4[u], s_lo[j], s_w[j]);
                    r2 = __dadd_rn(r2, __dmul_rn(x, x));
                    below |= static_cast<uint32_t>(x < s_mid[j]) << j;
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
    if (t < W) partial[static_cast<size_t>(blockIdx.x) * W + t] = s[t * kNsBlock];
}

// out[box][k] = sum over bx in order of partial[box][bx][k].
__global__ void nsphere_sum(const double *partial, int nbox, int gx, int W, double *out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nbox * W) return;
    const int box = idx / W, k = idx % W;
    double v = 0.0;
    for (int bx = 0; bx < gx; ++bx) v += partial[(static_cast<size_t>(box) * gx + bx) * W + k];
    out[idx] = v;
}

bfi_status cuda_fail(const char *what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s failed: %s", what, cudaGetErrorString(e));
    return bfi::set_error(BFI_E_CUDA, msg);
}

}  // namespace

namespace bfi {

bfi_status nsphere_batch(int dims, int64_t nbox, const double *lo, const double *hi, const uint64_t *n,
                         const uint32_t *sub_id, uint32_t seed, uint32_t job_id, int device, double *sums) {
    if (dims < 1 || dims > kNsMaxDims || nbox < 1 || nbox > (int64_t(1) << 24) || !lo || !hi || !n || !sub_id || !sums)
        return set_error(BFI_E_INVALID, "need 1 <= dims <= 32, 1 <= boxes <= 2^24 and non-NULL arrays");
    const size_t nd = static_cast<size_t>(nbox) * dims;
    std::vector<double> w(nd), mid(nd);
    for (size_t i = 0; i < nd; ++i) {
        if (!(hi[i] > lo[i])) return set_error(BFI_E_INVALID, "need lo < hi in every coordinate");
        w[i] = hi[i] - lo[i];
        mid[i] = 0.5 * (lo[i] + hi[i]);
    }
    for (int64_t k = 0; k < nbox; ++k)
        if (n[k] >= (uint64_t(1) << 48)) return set_error(BFI_E_INVALID, "a sample count is >= 2^48");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
    struct Restore {
        int prev;
        ~Restore() {
            if (prev >= 0) cudaSetDevice(prev);
        }
    } restore{prev};
    int sms = 1, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nsphere_kernel, kNsBlock, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // about one resident wave in total, at least one block per box
    const int64_t wave = static_cast<int64_t>(sms) * per_sm;
    const int gx = static_cast<int>(std::max<int64_t>(1, (wave + nbox - 1) / nbox));
    const int W = 2 + dims;
    const size_t n_part = static_cast<size_t>(nbox) * gx * W, n_out = static_cast<size_t>(nbox) * W;
    unsigned char *buf = nullptr;
    const size_t bytes = sizeof(double) * (3 * nd + n_part + n_out) + sizeof(uint64_t) * nbox + sizeof(uint32_t) * nbox;
    e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) return cuda_fail("cudaMalloc", e);
    double *d_lo = reinterpret_cast<double *>(buf), *d_w = d_lo + nd, *d_mid = d_w + nd, *d_part = d_mid + nd,
           *d_out = d_part + n_part;
    uint64_t *d_n = reinterpret_cast<uint64_t *>(d_out + n_out);
    uint32_t *d_sub = reinterpret_cast<uint32_t *>(d_n + nbox);
    e = cudaMemcpy(d_lo, lo, sizeof(double) * nd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_w, w.data(), sizeof(double) * nd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_mid, mid.data(), sizeof(double) * nd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_n, n, sizeof(uint64_t) * nbox, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_sub, sub_id, sizeof(uint32_t) * nbox, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const NsBoxes b{d_lo, d_w, d_mid, d_n, d_sub, dims, gx};
        nsphere_kernel<<<static_cast<unsigned>(nbox * gx), kNsBlock>>>(b, make_round_keys(seed, job_id), d_part);
        const int threads = 256, blocks = static_cast<int>((n_out + threads - 1) / threads);
        nsphere_sum<<<blocks, threads>>>(d_part, static_cast<int>(nbox), gx, W, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(sums, d_out, sizeof(double) * n_out, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail("nsphere", e);
    return BFI_OK;
}

void nsphere_finish(int dims, const double *lo, const double *hi, uint64_t n, const double *sums, double *result,
                    double *abs_err, int32_t *split_dim) {
    double vol = 1.0;
    for (int j = 0; j < dims; ++j) vol *= hi[j] - lo[j];
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
}

}  // namespace bfi

extern "C" bfi_status bfi_nsphere(int32_t dims, const double *lo, const double *hi, uint64_t n, uint32_t seed,
                                  uint32_t job_id, uint32_t sub_id, double *result, double *abs_err,
                                  int32_t *split_dim, int device) {
    if (!result || !abs_err || n < 2) return bfi::set_error(BFI_E_INVALID, "need n >= 2 and non-NULL outputs");
    double sums[2 + kNsMaxDims];
    const bfi_status st = bfi::nsphere_batch(dims, 1, lo, hi, &n, &sub_id, seed, job_id, device, sums);
    if (st != BFI_OK) return st;
    bfi::nsphere_finish(dims, lo, hi, n, sums, result, abs_err, split_dim);
    return BFI_OK;
}
