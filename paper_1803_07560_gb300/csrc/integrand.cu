// integrand.cu -- the hot path of the Monte Carlo evaluation of the lattice
// Burgers functional integral (Honkonen & Honkonen, arXiv:1803.07560,
// Eq. (Gen2), Sec. 3 and Sec. 4) as sm_103a kernels:
//
//   integrand_f64 / integrand_f32
//                  persistent, thread-per-sample: Philox points -> action ->
//                  shifted weight -> products -> per-thread sums; then a
//                  warp / block merge of shifted records into one partial
//                  record per chunk of samples
//   hint_f32       per-subvolume reference action (the smallest FP32 action
//                  of the first samples), the starting point of both kernels
//   merge_subvolumes   FP64 merge of each subvolume's chunk records, in chunk
//                      order, into its slot
//   merge_totals       FP64 merge of all slots into Z, C(r) and errors
//
// Every reduction has a fixed order, so results are bitwise reproducible and do
// not depend on what else runs on the device.
#include "integrand_kernels.cuh"

#include <cmath>

namespace bfi {
// ---------------------------------------------------------------------------
// Per-subvolume FP64 merge of chunk records, in chunk order.  One warp per
// subvolume: lane t merges sums t, t + 32, ... (each in chunk order, so every
// sum is the same as a sequential merge gives), and the reads of a chunk
// record are coalesced.  Also scales the unscaled products Q_r = d P_r back to
// P_r and records log V_s (the per-lane sums of log widths combined in a fixed
// butterfly).
// ---------------------------------------------------------------------------
__global__ void merge_subvolumes(const MergeArgs a) {
    const int64_t s = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= a.nsub) return;  // warp-uniform
    const int R = a.R, K = 2 + 3 * R, SL = 5 + 3 * R;
    double *slot = a.slots + s * SL;
    double n = 0.0, m = INFINITY;
    for (int k = lane; k < K; k += 32) slot[3 + k] = 0.0;
    for (int64_t c = a.chunk_off[s]; c < a.chunk_off[s + 1]; ++c) {
        const double *p = a.partials + c * (K + 2);
        n += p[0];
        const double mb = p[1];
        if (mb == INFINITY) continue;  // no evaluated samples in the chunk
        if (mb == m) {
            for (int k = lane; k < K; k += 32) slot[3 + k] = __dadd_rn(slot[3 + k], p[2 + k]);
            continue;
        }
        const double mn = fmin(m, mb);
        const double fa = (m == INFINITY) ? 0.0 : exp(mn - m);
        const double fb = exp(mn - mb);
        for (int k = lane; k < K; k += 32) {
            const bool sq = (k == 1) || (k >= 2 + R);
            slot[3 + k] = __dadd_rn(__dmul_rn(slot[3 + k], sq ? fa * fa : fa), __dmul_rn(p[2 + k], sq ? fb * fb : fb));
        }
        m = mn;
    }
    const double inv_d = 1.0 / static_cast<double>(a.d);
    for (int r = lane; r < R; r += 32) {
        slot[5 + r] *= inv_d;
        slot[5 + R + r] *= inv_d;
        slot[5 + 2 * R + r] *= inv_d * inv_d;
    }
    double log_vol = 0.0;
    for (int j = lane; j < a.d; j += 32) log_vol += log(a.hi[s * a.d + j] - a.lo[s * a.d + j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) log_vol += __shfl_xor_sync(0xffffffffu, log_vol, off);
    if (lane == 0) {
        slot[0] = n;
        slot[1] = m;
        slot[2] = a.log_norm_set ? a.log_norm : log_vol;
    }
}

// ---------------------------------------------------------------------------
// Cross-subvolume FP64 merge (one CTA of 256 threads, fixed-order trees).
//   ls_s = log V_s - log n_s - m_s,  L = max ls_s,  f_s = exp(ls_s - L)
//   Z' = sum f_s sum w,  N'(r) = sum f_s sum w P_r,  C = N'/Z'
//   Var Z' = sum f_s^2 (n sum w^2 - (sum w)^2)/(n-1)
//   Var C  = sum f_s^2 [V_N - 2 C Cov + C^2 V_Z] / Z'^2   (delta method)
// ---------------------------------------------------------------------------
constexpr int kTotThreads = 256;

// Block-wide sum / max: an XOR butterfly in each warp, then every thread adds
// the kTotThreads/32 warp results in warp order (fixed order: reproducible).
__device__ double block_sum(double v, double *sh) {
    const int t = threadIdx.x;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int w = 0; w < kTotThreads / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double *sh) {
    const int t = threadIdx.x;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double r = sh[0];
#pragma unroll
    for (int w = 1; w < kTotThreads / 32; ++w) r = fmax(r, sh[w]);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kTotThreads) merge_totals(const TotalsArgs a) {
    double *f_buf = a.f_buf;
    __shared__ double sh[kTotThreads];
    const int t = threadIdx.x;
    const int R = a.R, SL = 5 + 3 * R;
    double lmax = -INFINITY, n_tot = 0.0, used = 0.0;
    for (int64_t s = t; s < a.nsub; s += kTotThreads) {
        const double *q = a.slots + s * SL;
        if (q[0] <= 0.0) continue;
        n_tot += q[0];
        used += 1.0;
        if (!(q[3] > 0.0)) continue;
        lmax = fmax(lmax, q[2] - log(q[0]) - q[1]);
    }
    const double L = block_max(lmax, sh);
    n_tot = block_sum(n_tot, sh);
    used = block_sum(used, sh);

    // f_s = exp(ls_s - L) once per subvolume (0 for subvolumes without weight),
    // and g_s = f_s^2 / (n_s - 1), the factor of every variance term (one
    // division per subvolume instead of one per term)
    double z = 0.0, vz = 0.0, bad = 0.0;
    for (int64_t s = t; s < a.nsub; s += kTotThreads) {
        const double *q = a.slots + s * SL;
        double f = 0.0, gs = 0.0;
        if (q[0] > 0.0 && q[3] > 0.0) {
            const double n = q[0];
            f = exp(q[2] - log(n) - q[1] - L);
            z += f * q[3];
            if (n < 2.0) {
                bad = 1.0;
            } else {
                gs = f * f / (n - 1.0);
                vz += gs * (n * q[4] - q[3] * q[3]);
            }
        }
        f_buf[s] = f;
        f_buf[a.nsub + s] = gs;
    }
    const double Z = block_sum(z, sh);
    const double VZ = block_sum(vz, sh);
    const bool inf_err = block_max(bad, sh) > 0.0;
    if (t == 0) {
        a.totals[0] = L + log(Z);
        a.totals[1] = inf_err ? INFINITY : sqrt(VZ > 0.0 ? VZ : 0.0) / Z;
        a.totals[2] = n_tot;
        a.totals[3] = used;
    }
    for (int r = 0; r < R; ++r) {
        double nr = 0.0;
        for (int64_t s = t; s < a.nsub; s += kTotThreads) nr += f_buf[s] * a.slots[s * SL + 5 + r];
        const double C = block_sum(nr, sh) / Z;
        double var = 0.0;
        for (int64_t s = t; s < a.nsub; s += kTotThreads) {
            const double gs = f_buf[a.nsub + s];
            if (gs == 0.0) continue;
            const double *q = a.slots + s * SL;
            const double n = q[0];
            const double vN = n * q[5 + 2 * R + r] - q[5 + r] * q[5 + r];
            const double cov = n * q[5 + R + r] - q[3] * q[5 + r];
            const double vZ = n * q[4] - q[3] * q[3];
            var += gs * (vN - 2.0 * C * cov + C * C * vZ);
        }
        const double V = block_sum(var, sh);
        if (t == 0) {
            a.totals[4 + r] = C;
            a.totals[4 + R + r] = inf_err ? INFINITY : sqrt(V > 0.0 ? V : 0.0) / Z;
        }
    }
}

// ---------------------------------------------------------------------------
// Single-step kernels for step-by-step checks.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void points_kernel(const PointsArgs a, const RoundKeys rk) {
    const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int nq = (a.d + 3) / 4;
    if (idx >= a.count * nq) return;
    const int64_t k = idx / nq;
    const int q = static_cast<int>(idx % nq);
    const uint64_t i = a.first + static_cast<uint64_t>(k);
    const uint4 wd = philox4x32_10(
        make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), a.sub_id), rk);
    const uint32_t w4[4] = {wd.x, wd.y, wd.z, wd.w};
    for (int t = 0; t < 4; ++t) {
        const int j = 4 * q + t;
        if (j >= a.d) break;
        Real b, w;
        BoxPair<Real>::load(a.lo, a.hi, j, b, w);
        a.y[k * a.d + j] = static_cast<double>(Coord<Real>::map(w4[t], b, w));
    }
}

const ShapeKernels *find_shape(int nx, int nt) {
    for (auto table : {shapes_small, shapes_config_a, shapes_config_b, shapes_config_c, shapes_config_d}) {
        int n = 0;
        const ShapeKernels *t = table(&n);
        for (int i = 0; i < n; ++i)
            if (t[i].nx == nx && t[i].nt == nt) return &t[i];
    }
    return generic_shape(nx, nt);
}

cudaError_t launch_merges(const MergeArgs &m, const TotalsArgs &t, cudaStream_t st) {
    const int threads = 256;  // 8 subvolumes (one warp each) per block
    const int64_t blocks = (m.nsub * 32 + threads - 1) / threads;
    merge_subvolumes<<<static_cast<unsigned>(blocks), threads, 0, st>>>(m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    merge_totals<<<1, kTotThreads, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_points(const PointsArgs &a, bool fp32, uint32_t seed, uint32_t job, cudaStream_t st) {
    const int threads = 128;
    const int64_t work = a.count * ((a.d + 3) / 4);
    const int64_t blocks = (work + threads - 1) / threads;
    if (blocks == 0) return cudaSuccess;
    if (fp32)
        points_kernel<float><<<static_cast<unsigned>(blocks), threads, 0, st>>>(a, make_round_keys(seed, job));
    else
        points_kernel<double><<<static_cast<unsigned>(blocks), threads, 0, st>>>(a, make_round_keys(seed, job));
    return cudaGetLastError();
}

}  // namespace bfi
