// mapped_kernels.cuh -- the range map of Sec. 4 (the infinite range of every
// coordinate taken to (-1, 1)) and Gaussian importance sampling as
// thread-per-sample FP64 kernels over the compiled lattice shapes, with their
// launchers.  Included by the shapes_*.cu files next to the box-sampler
// kernels.
//
//   transform_f64  persistent, thread per sample: Philox point y in the box,
//                  v_j = y_j / (1 - y_j^2), S_eff = S(v) - ln J with
//                  ln J = sum_j ln[(1 + y_j^2) / (1 - y_j^2)^2], weight,
//                  products and per-thread sums -> one FP64 record per chunk
//   gaussian_f64   the same with v = mean + F z, z standard normal from the
//                  unit point by the Box-Muller transform, S_eff = S(v) -
//                  |z|^2 / 2 and weight 0 outside the box (d <= 40)
//
// There is no FP32 screen: the map stretches the coordinates without bound
// near y = +-1, so no fixed margin covers the FP32 action's error there, and
// inside a subvolume S_eff varies far less than it does over a box of the
// plain field (most samples carry weight).  Every sample is evaluated in FP64;
// the kernel is bound by GB300's FP64 pipe, so its FP64 work per sample is
// kept small: one reciprocal per coordinate by Newton's iteration instead of
// a division, and one logarithm per sample for all of ln J.
#pragma once

#include "integrand_kernels.cuh"

namespace bfi {

// 1/x within about an ulp: Newton's iteration for f(r) = 1/r - x,
// r <- r + r (1 - x r), which squares the relative error at each step, from
// the hardware's approximate reciprocal (PTX rcp.approx.ftz.f64).  Two steps
// take an error below 2^-20 to the rounding level.  x must be a positive
// normal number (here 1 - y^2 >= 2^-53); 0 gives NaN.
__device__ __forceinline__ double recip_newton(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = __fma_rn(-x, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-x, r, 1.0);
    return __fma_rn(r, e, r);
}

// ln of a product of factors >= 1, kept as p * 2^e with p brought back to
// [1, 2) by integer operations on its exponent field (no FP64 work), so that
// one logarithm serves the whole product.  renorm() after at most four
// factors below 2^255 each keeps p finite; an infinite or NaN p is left alone
// (its logarithm is then +inf or NaN, as the sum of the logarithms would be).
struct LogProduct {
    double p = 1.0;
    int e = 0;
    __device__ __forceinline__ void mul(double x) { p *= x; }
    __device__ __forceinline__ void renorm() {
        const int hi = __double2hiint(p);
        const int ex = (hi >> 20) & 0x7ff;
        if (ex != 0x7ff) {
            e += ex - 1023;
            p = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(p));
        }
    }
    __device__ __forceinline__ double log_value() const {
        return fma(static_cast<double>(e), 0.6931471805599453, log(p));  // e ln 2 + ln p
    }
};

// Compiled for one resident CTA per SM (all 255 registers a thread may
// have): the FP64 pipe (two lanes per SM and clock) takes a warp instruction
// every 64 cycles per scheduler, which two warps per scheduler keep busy, so
// occupancy buys nothing and spilling the d FP64 coordinates would cost.

// ---------------------------------------------------------------------------
// One CTA processes chunk blockIdx.x, then the chunks next_chunk hands it; thread t
// evaluates samples first + t, first + t + B, ... of the chunk.  The Philox
// words, the point y = lo + (hi - lo) u (the FP64 point of the box sampler)
// and 1 - y^2 = (1 - y)(1 + y) are those of the definition; v_j = y_j r_j
// with r_j = 1 / (1 - y_j^2), and J_j = (1 + y_j^2) r_j^2 joins the running
// product.  Each thread's shift starts above every action and drops to its
// first sample's S_eff, then moves down only when beaten by more than
// kRescaleMargin (as in the box kernels); the chunk record merges the
// threads at the smallest shift.  A chunk with no finite S_eff records
// m = +inf and zero sums.
// ---------------------------------------------------------------------------
template <int NX, int NT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) transform_f64(const IntegrandArgs args, const LatticeConst<double> lc,
                                                          const RoundKeys rk) {
    constexpr int D = NX * NT;
    constexpr int R = NX / 2 + 1;
    constexpr int K = sum_count(R);
    constexpr int NQ = (D + 3) / 4;
    __shared__ ChunkShared<BLOCK> sh;
    __shared__ double s_lo[D], s_w[D];
    __shared__ PhiloxPrefix s_pre[NQ];
    __shared__ double s_sums[K * BLOCK];
    const int tid = threadIdx.x;
    SmemSums<double, K, BLOCK> acc{s_sums + tid};

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, &sh.next)) {
        const ChunkView v = chunk_view(args, c, D);
        if (tid < D) {
            s_lo[tid] = v.lo[tid];
            s_w[tid] = v.hi[tid] - v.lo[tid];
        }
        chunk_prefixes<D>(v, rk, s_pre);
        if (tid == 0) sh.evaluated = 0u;
        acc.zero();
        __syncthreads();

        double m_acc = INFINITY;
        unsigned n_eval = 0;
        for (uint64_t k = tid; k < v.cnt; k += BLOCK) {
            const uint32_t x = static_cast<uint32_t>(v.first + k);
            double u[D];
            LogProduct jac;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const uint4 b = philox_from_prefix(x, s_pre[q], rk);
                const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = 4 * q + t;
                    if (j < D) {
                        const double y = Coord<double>::map(w4[t], s_lo[j], s_w[j]);
                        const double r = recip_newton((1.0 - y) * (1.0 + y));
                        u[j] = y * r;
                        jac.mul(fma(y, y, 1.0) * r * r);
                        if (j % 2 == 1 || j == D - 1) jac.renorm();
                    }
                }
            }
            const double S = action<NX, NT, double>(u, lc) - jac.log_value();
            double Q[R];
            products<NX, NT, double>(u, Q);
            if (S < m_acc - kRescaleMargin) {  // the first sample, then rarely
                rescale<double, K, R, BLOCK>(acc, exp(S - m_acc));
                m_acc = S;
            }
            accumulate<double, K, R, BLOCK>(acc, exp(m_acc - S), Q);
            ++n_eval;
        }
        add_evaluated(args.stats, n_eval, &sh.evaluated);
        chunk_record<double, K, R, BLOCK>(acc, m_acc, sh.f, &sh.mb, args.partials + c * (K + 2), v.cnt);
    }
}

// ---------------------------------------------------------------------------
// Gaussian importance sampling, thread per sample (d <= kGaussThreadMaxD):
// z_{2p}, z_{2p+1} = box_muller(u_{2p}, u_{2p+1}) for the unit point u (the
// box plays no part in drawing; for odd d the pair of z_{d-1} takes word d of
// the last Philox block), v = mean + F z, S_eff = S(v) - |z|^2 / 2, and
// weight 0 outside the box
// [lo, hi).  The rest of 1/q (the record's log-volume (d/2) ln 2 pi +
// ln |det F|) is set by the merge.  F, held transposed in shared memory
// (column j of F contiguous, every thread reading the same word), is applied
// column by column as each z_j is drawn, so z is never stored; for an upper
// triangular F (TRI, the proposal bfi_gaussian_proposal returns) column j
// stops at row j.  Samples outside the box are counted in n and skip the
// action; the kernel counts the evaluated (inside) samples in stats.
// ---------------------------------------------------------------------------
constexpr int kGaussThreadMaxD = 40;

template <int NX, int NT, int BLOCK, bool TRI>
__global__ void __launch_bounds__(BLOCK, 1) gaussian_f64(const IntegrandArgs args, const LatticeConst<double> lc,
                                                         const RoundKeys rk, const double *mean,
                                                         const double *factor) {
    constexpr int D = NX * NT;
    constexpr int R = NX / 2 + 1;
    constexpr int K = sum_count(R);
    constexpr int NQ = (D + 3) / 4;
    static_assert(D <= kGaussThreadMaxD, "the thread-per-sample Gaussian kernel holds v in registers");
    __shared__ ChunkShared<BLOCK> sh;
    __shared__ double s_ft[D * D];  // s_ft[j D + r] = F[r][j]
    __shared__ double s_mean[D], s_lo[D], s_hi[D];
    __shared__ PhiloxPrefix s_pre[NQ];
    __shared__ double s_sums[K * BLOCK];
    const int tid = threadIdx.x;
    SmemSums<double, K, BLOCK> acc{s_sums + tid};
    for (int k = tid; k < D * D; k += BLOCK) s_ft[(k % D) * D + k / D] = factor[k];
    for (int k = tid; k < D; k += BLOCK) s_mean[k] = mean ? mean[k] : 0.0;

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, &sh.next)) {
        const ChunkView v = chunk_view(args, c, D);
        if (tid < D) {
            s_lo[tid] = v.lo[tid];
            s_hi[tid] = v.hi[tid];
        }
        chunk_prefixes<D>(v, rk, s_pre);
        if (tid == 0) sh.evaluated = 0u;
        acc.zero();
        __syncthreads();

        double m_acc = INFINITY;
        unsigned n_eval = 0;
        for (uint64_t k = tid; k < v.cnt; k += BLOCK) {
            const uint32_t x = static_cast<uint32_t>(v.first + k);
            double u[D];
#pragma unroll
            for (int r = 0; r < D; ++r) u[r] = s_mean[r];
            double zz = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const uint4 b = philox_from_prefix(x, s_pre[q], rk);
                const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int t = 0; t < 4; t += 2) {
                    const int j = 4 * q + t;
                    if (j < D) {
                        double zp[2];
                        box_muller(unit_f64(w4[t]), unit_f64(w4[t + 1]), zp[0], zp[1]);
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            if (j + e < D) {
                                const double z = zp[e];
                                zz = fma(z, z, zz);
#pragma unroll
                                for (int r = 0; r < (TRI ? j + e + 1 : D); ++r)
                                    u[r] = fma(s_ft[(j + e) * D + r], z, u[r]);
                            }
                        }
                    }
                }
            }
            bool inside = true;
#pragma unroll
            for (int r = 0; r < D; ++r) inside = inside && u[r] >= s_lo[r] && u[r] < s_hi[r];
            if (!inside) continue;  // weight 0
            const double S = action<NX, NT, double>(u, lc) - 0.5 * zz;
            double Q[R];
            products<NX, NT, double>(u, Q);
            if (S < m_acc - kRescaleMargin) {
                rescale<double, K, R, BLOCK>(acc, exp(S - m_acc));
                m_acc = S;
            }
            accumulate<double, K, R, BLOCK>(acc, exp(m_acc - S), Q);
            ++n_eval;
        }
        add_evaluated(args.stats, n_eval, &sh.evaluated);
        chunk_record<double, K, R, BLOCK>(acc, m_acc, sh.f, &sh.mb, args.partials + c * (K + 2), v.cnt);
    }
}

template <int NX, int NT>
cudaError_t launch_gaussian(const IntegrandArgs &args, const LatticeParams &p, const MapArgs &m, bool upper,
                            uint32_t seed, uint32_t job, int grid, cudaStream_t st) {
    const RoundKeys rk = make_round_keys(seed, job);
    if (upper)
        gaussian_f64<NX, NT, kBlock, true><<<grid, kBlock, 0, st>>>(args, make_const<double>(p), rk, m.mean, m.factor);
    else
        gaussian_f64<NX, NT, kBlock, false><<<grid, kBlock, 0, st>>>(args, make_const<double>(p), rk, m.mean, m.factor);
    return cudaGetLastError();
}

template <int NX, int NT>
cudaError_t occupancy_gaussian(int, int, int *blocks_per_sm) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, gaussian_f64<NX, NT, kBlock, true>, kBlock, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gaussian_f64<NX, NT, kBlock, false>, kBlock, 0);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

// The Gaussian entries of the shape table: null above kGaussThreadMaxD (those
// shapes use generic_mapped<2>).
template <int NX, int NT>
constexpr GaussLauncher gaussian_entry() {
    if constexpr (NX * NT <= kGaussThreadMaxD) return launch_gaussian<NX, NT>;
    else return nullptr;
}
template <int NX, int NT>
constexpr OccupancyQuery gaussian_occupancy_entry() {
    if constexpr (NX * NT <= kGaussThreadMaxD) return occupancy_gaussian<NX, NT>;
    else return nullptr;
}

template <int NX, int NT>
cudaError_t launch_transform(const IntegrandArgs &args, const LatticeParams &p, uint32_t seed, uint32_t job, int grid,
                             cudaStream_t st) {
    transform_f64<NX, NT, kBlock><<<grid, kBlock, 0, st>>>(args, make_const<double>(p), make_round_keys(seed, job));
    return cudaGetLastError();
}

template <int NX, int NT>
cudaError_t occupancy_transform(int, int, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transform_f64<NX, NT, kBlock>, kBlock, 0);
}

}  // namespace bfi
