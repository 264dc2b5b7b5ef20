// integrand_kernels.cuh -- the integrand kernels of the lattice Burgers
// functional integral (Honkonen & Honkonen, arXiv:1803.07560, Eq. (Gen2),
// Sec. 3 and Sec. 4) as templates over the lattice shape, with their host
// launchers.  Each shape is instantiated in one of the shapes_*.cu files so
// that the shapes compile in parallel.
//
//   integrand_f64 / integrand_f32
//                  persistent, thread-per-sample: Philox points -> FP32 screen
//                  -> (queued, 32 at a time) full evaluation -> per-thread
//                  sums -> one FP64 record per chunk of samples
//   hint_f32       per-subvolume reference action (the smallest FP32 action
//                  of the first samples), the starting point of both kernels
//   eval_kernel    action and products at given points (single-step checks)
#pragma once

#include "bfi_device.cuh"
#include "bfi_kernels.h"

#include <cmath>
#include <type_traits>

// Resident CTAs per SM the integrand kernels are compiled for; 0 (default)
// picks it from the lattice size (registers grow with d, shared memory with R).
#ifndef BFI_INTEGRAND_MIN_BLOCKS
#define BFI_INTEGRAND_MIN_BLOCKS 0
#endif

namespace bfi {

// Shared memory of integrand_f64 per CTA (the larger of the two kernels).
template <int NX, int NT>
constexpr int integrand_smem_bytes() {
    return 8 * (kBlock + 2) + 24 * NX * NT + 8 * (2 + 3 * (NX / 2 + 1)) * kBlock + 4 * (kBlock / 32) * 64;
}

template <int NX, int NT>
constexpr int min_blocks() {
    constexpr int d = NX * NT;
    constexpr int by_regs = d <= 32 ? 4 : (d <= 48 ? 3 : 2);
    constexpr int by_smem = (227 * 1024) / integrand_smem_bytes<NX, NT>();
    constexpr int b = by_regs < by_smem ? by_regs : by_smem;
    return BFI_INTEGRAND_MIN_BLOCKS > 0 ? BFI_INTEGRAND_MIN_BLOCKS : (b > 0 ? b : 1);
}


// ---------------------------------------------------------------------------
// Chunk lookup: chunks of subvolume s are [chunk_off[s], chunk_off[s+1]).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t find_subvolume(const int64_t *chunk_off, int64_t nsub, int64_t c) {
    int64_t lo = 0, hi = nsub;  // invariant: chunk_off[lo] <= c < chunk_off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (chunk_off[mid] <= c) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename Real>
struct BoxPair;
template <>
struct BoxPair<float> {
    __device__ __forceinline__ static void load(const double *lo, const double *hi, int j, float &b, float &w) {
        b = __double2float_rn(lo[j]);
        w = __double2float_rn(hi[j] - lo[j]);
    }
};
template <>
struct BoxPair<double> {
    __device__ __forceinline__ static void load(const double *lo, const double *hi, int j, double &b, double &w) {
        b = lo[j];
        w = hi[j] - lo[j];
    }
};

// ---------------------------------------------------------------------------
// Chunk set-up shared by the integrand kernels.
// ---------------------------------------------------------------------------
struct ChunkView {
    int64_t s;          // subvolume
    uint64_t first;     // first sample index of the chunk
    uint64_t cnt;       // samples in the chunk
    uint32_t sid;       // Philox counter word 3
    const double *lo, *hi;
};

__device__ __forceinline__ ChunkView chunk_view(const IntegrandArgs &args, int64_t c, int d) {
    ChunkView v;
    v.s = find_subvolume(args.chunk_off, args.nsub, c);
    const uint64_t n_s = args.samples[v.s];
    const uint64_t cs = static_cast<uint64_t>(
        args.tail_chunk_samples > 0 && v.s >= args.tail_sub ? args.tail_chunk_samples : args.chunk_samples);
    v.first = static_cast<uint64_t>(c - args.chunk_off[v.s]) * cs;
    v.cnt = min(cs, n_s - v.first);
    v.sid = args.sub_id ? args.sub_id[v.s] : static_cast<uint32_t>(v.s);
    v.lo = args.lo + v.s * d;
    v.hi = args.hi + v.s * d;
    return v;
}

// S of Eq. (Gen2): the residual sum of squares plus the optional mass term.
template <int NX, int NT, typename Real>
__device__ __forceinline__ Real action(const Real (&u)[NX * NT], const LatticeConst<Real> &c) {
    Real S = residual_sq_sum<NX, NT, Real>(u, c) * c.inv_2Dtau;
    if (c.half_mass2 != Real(0)) {
        Real s2 = Real(0);
#pragma unroll
        for (int j = 0; j < NX * NT; ++j) s2 = fma(u[j], u[j], s2);
        S = fma(c.half_mass2, s2, S);
    }
    return S;
}

// Raw Philox words of sample i: block q = (q, i lo, i hi, sid), word j%4.
template <int D>
__device__ __forceinline__ void sample_words(uint64_t i, uint32_t sid, const RoundKeys &rk, uint32_t (&w)[D]) {
    constexpr int NQ = (D + 3) / 4;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 b = philox4x32_10(
            make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), sid), rk);
        const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * q + t < D) w[4 * q + t] = w4[t];
    }
}

// FP32 coordinates of sample i from the (lo, width) pairs in shared memory.
template <int D>
__device__ __forceinline__ void make_point_smem(uint64_t i, uint32_t sid, const RoundKeys &rk, const float2 *box,
                                                float (&u)[D]) {
    constexpr int NQ = (D + 3) / 4;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 b = philox4x32_10(
            make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), sid), rk);
        const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * q + t;
            if (j < D) {
                const float2 bw = box[j];
                u[j] = Coord<float>::map(w4[t], bw.x, bw.y);
            }
        }
    }
}

// The same two from the chunk's Philox prefixes (one per block q, in shared
// memory): x is the low word of the sample index.
template <int D>
__device__ __forceinline__ void sample_words_pre(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                                 uint32_t (&w)[D]) {
    constexpr int NQ = (D + 3) / 4;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 b = philox_from_prefix(x, pre[q], rk);
        const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * q + t < D) w[4 * q + t] = w4[t];
    }
}

template <int D>
__device__ __forceinline__ void make_point_pre(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                               const float2 *box, float (&u)[D]) {
    constexpr int NQ = (D + 3) / 4;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 b = philox_from_prefix(x, pre[q], rk);
        const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * q + t;
            if (j < D) {
                const float2 bw = box[j];
                u[j] = Coord<float>::map(w4[t], bw.x, bw.y);
            }
        }
    }
}

// Prefixes of the chunk's blocks q = 0 .. NQ-1 (threads 0 .. NQ-1; the
// caller synchronises before use).
template <int D>
__device__ __forceinline__ void chunk_prefixes(const ChunkView &v, const RoundKeys &rk, PhiloxPrefix *pre) {
    constexpr int NQ = (D + 3) / 4;
    if (threadIdx.x < NQ) pre[threadIdx.x] = philox_prefix(threadIdx.x, static_cast<uint32_t>(v.first >> 32), v.sid, rk);
}

// ---------------------------------------------------------------------------
// Packed FP32 screen for even NX.  Site m is paired with site m + NX/2:
// P[h NT + l] = (u[h NT + l], u[(h + NX/2) NT + l]), h < NX/2.  The next-slice,
// right and left neighbours of a pair are pairs too, except across the seam
// (right of h = NX/2 - 1, left of h = 0) where the partner's halves come
// swapped; so the residuals of two sites go through one f32x2 instruction
// each.  Every component is rounded as the scalar residual rounds it (right -
// left as one FMA with -1); only the order of the final sum differs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

template <int NX, int NT>
__device__ __forceinline__ float action_pairs(const float2 (&P)[(NX / 2) * NT], const LatticeConst<float> &c) {
    constexpr int H = NX / 2;
    const float2 cadv = make_float2(c.c_adv, c.c_adv), k1 = make_float2(c.k1, c.k1);
    const float2 ncd = make_float2(c.neg_c_dif, c.neg_c_dif), m1 = make_float2(-1.f, -1.f);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < H; ++h) {
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            const float2 here = P[h * NT + l];
            const float2 next = P[h * NT + (l + 1) % NT];
            const float2 right = h + 1 < H ? P[(h + 1) * NT + l] : swap2(P[l]);
            const float2 left = h > 0 ? P[(h - 1) * NT + l] : swap2(P[(H - 1) * NT + l]);
            const float2 t = __ffma2_rn(cadv, __ffma2_rn(m1, left, right), k1);
            float2 R = __ffma2_rn(here, t, next);
            R = __ffma2_rn(ncd, __fadd2_rn(right, left), R);
            acc = __ffma2_rn(R, R, acc);
        }
    }
    float S = (acc.x + acc.y) * c.inv_2Dtau;
    if (c.half_mass2 != 0.f) {
        float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < H * NT; ++k) s2 = __ffma2_rn(P[k], P[k], s2);
        S = fmaf(c.half_mass2, s2.x + s2.y, S);
    }
    return S;
}

// Points of sample x in that pair layout; Map(word, box[j]) -> coordinate.
template <int NX, int NT, typename Map>
__device__ __forceinline__ void make_pairs_pre(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                               const float2 *box, Map map, float2 (&P)[(NX / 2) * NT]) {
    constexpr int D = NX * NT, NQ = (D + 3) / 4, H = NX / 2;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 b = philox_from_prefix(x, pre[q], rk);
        const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * q + t;
            if (j < D) {
                const int m = j / NT, l = j % NT;
                const float val = map(w4[t], box[j]);
                if (m < H) P[m * NT + l].x = val;
                else P[(m - H) * NT + l].y = val;
            }
        }
    }
}

// The screen point of both kernels: y = fmaf(1.m, w, lo') with 1.m the
// word's top 23 bits as a float in [1,2) and lo' = lo - (1 - 2^-24) w folded
// per chunk into the screen's box table, one operation fewer per coordinate
// than the exact FP32 point (Coord<float>::map, which the FP32 evaluation
// uses); it differs from that point by the rounding of lo' (under 1e-6 here),
// which the screen's margin covers.
struct MapScreen {
    __device__ __forceinline__ float operator()(uint32_t w, float2 bw) const {
        return __fmaf_rn(__uint_as_float(0x3f800000u | (w >> 9)), bw.y, bw.x);
    }
};

// FP32 screen action of sample x: packed for even NX, scalar otherwise.
template <int NX, int NT, typename Map>
__device__ __forceinline__ float screen_action(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                               const float2 *box, const LatticeConst<float> &c) {
    if constexpr (NX % 2 == 0) {
        float2 P[(NX / 2) * NT];
        make_pairs_pre<NX, NT>(x, pre, rk, box, Map{}, P);
        return action_pairs<NX, NT>(P, c);
    } else {
        constexpr int D = NX * NT, NQ = (D + 3) / 4;
        float u[D];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint4 b = philox_from_prefix(x, pre[q], rk);
            const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (4 * q + t < D) u[4 * q + t] = Map{}(w4[t], box[4 * q + t]);
        }
        return action<NX, NT, float>(u, c);
    }
}

// ---------------------------------------------------------------------------
// Two-stage screen.  Stage 1 draws only the first BP Philox blocks, which
// hold the coordinates of the complete sites 0 .. MC-1, and sums the squared
// residuals of sites 1 .. MC-2 (every slice): a partial action P <= S,
// computed like the full FP32 action on a subset of its non-negative terms,
// so the screen's bound |S_f32 - S| <= 1 + 0.1% S holds for it too.  A sample
// whose P already exceeds the threshold is rejected; the few that survive
// (about a fifth at 10x2 over the box) are queued and screened 32 at a time
// by stage 2: for NT = 2 the rest of the action added to P (rest_action),
// otherwise the full screen.  BP is about 0.6 of the blocks.
//
// The split is used where the lattice has 3 or more blocks and stage 1 covers
// at least 35% of the residual sites, but not all: measured on GB300, 4x4
// (25%) and 6x2 (33%) ran 5-16% slower with it and 6x4 (33%) no faster,
// while 8x4 (37.5%) and 10x2 (40%) ran 5-15% faster.
//
// Chunks with fewer than kTwoStageMinRows rows per thread screen in one
// stage: the survivor queue's final drain costs about one full-screen row per
// warp, and the smaller jobs that get short chunks have less selective
// references.  On the batching workload (256 jobs of 2^20-2^28 samples) a
// threshold of 16 rows cost 4% against one stage, 64 rows 2%, 256 rows
// nothing.  A per-warp switch back to one stage when too many samples
// survive was measured and rejected: early in a chunk the reference action
// is still high, and the switch fired on the 10x2 workload too.
// (kTwoStageMinRows, in bfi_kernels.h, where the host's chunking reads it.)
// ---------------------------------------------------------------------------

template <int NX, int NT>
struct PartialScreen {
    static constexpr int D = NX * NT;
    static constexpr int NQ = (D + 3) / 4;
    static constexpr int BP = (3 * NQ + 4) / 5;
    static constexpr int MC = (4 * BP) / NT < NX ? (4 * BP) / NT : NX;
    static constexpr int DW = MC * NT;  // coordinates stage 1 maps
#ifdef BFI_NO_PARTIAL_SCREEN
    static constexpr bool enabled = false;
#else
    static constexpr bool enabled = NQ >= 3 && MC < NX && 20 * (MC - 2) >= 7 * NX;
#endif
};

// Stage 1 on packed f32x2 pairs of time slices (h, h + NT/2) of one site:
// the next slice of pair h is pair h + 1, and the swapped pair 0 for the last
// one (NT is even wherever the split is used).  Each component rounds as the
// scalar residual does.
template <int NX, int NT, typename Map>
__device__ __forceinline__ float partial_action(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                                const float2 *box, const LatticeConst<float> &c) {
    using PS = PartialScreen<NX, NT>;
    static_assert(!PS::enabled || NT % 2 == 0, "the partial screen pairs time slices");
    if constexpr (!PS::enabled) {
        return 0.f;  // never called: the kernels take the one-stage path
    } else {
        constexpr int H = NT / 2;
        float2 P[PS::MC * H];
#pragma unroll
        for (int q = 0; q < PS::BP; ++q) {
            const uint4 b = philox_from_prefix(x, pre[q], rk);
            const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = 4 * q + t;
                if (j < PS::DW) {
                    const int m = j / NT, l = j % NT;
                    const float val = Map{}(w4[t], box[j]);
                    if (l < H) P[m * H + l].x = val;
                    else P[m * H + l - H].y = val;
                }
            }
        }
        const float2 cadv = make_float2(c.c_adv, c.c_adv), k1 = make_float2(c.k1, c.k1);
        const float2 ncd = make_float2(c.neg_c_dif, c.neg_c_dif), m1 = make_float2(-1.f, -1.f);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m + 1 < PS::MC; ++m) {
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float2 here = P[m * H + h];
                const float2 next = h + 1 < H ? P[m * H + h + 1] : swap2(P[m * H]);
                const float2 right = P[(m + 1) * H + h];
                const float2 left = P[(m - 1) * H + h];
                const float2 t = __ffma2_rn(cadv, __ffma2_rn(m1, left, right), k1);
                float2 R = __ffma2_rn(here, t, next);
                R = __ffma2_rn(ncd, __fadd2_rn(right, left), R);
                acc = __ffma2_rn(R, R, acc);
            }
        }
        return (acc.x + acc.y) * c.inv_2Dtau;
    }
}

// Stage 2 for NT = 2 without redrawing what stage 1 summed: a survivor's
// partial action P comes with it through the queue, and the rest of S is the
// residuals of sites 0 and MC-1 .. NX-1.  They need sites 0, 1 (block 0),
// MC-2, MC-1 (block BP-1) and MC .. NX-1 (blocks BP ..), so the blocks
// 1 .. BP-2 are not drawn again.  Slices 0 and 1 of a site form one f32x2
// pair (the next slice is the swapped pair).  The mass term needs every
// coordinate, so with mass2 != 0 the kernels screen survivors in full.
template <int NX, int NT>
struct RestScreen {
    using PS = PartialScreen<NX, NT>;
    static constexpr bool enabled = PS::enabled && NT == 2 && NX % 2 == 0 && PS::BP >= 2;  // whole blocks of sites
};

template <int NX, int NT, typename Map>
__device__ __forceinline__ float rest_action(uint32_t x, const PhiloxPrefix *pre, const RoundKeys &rk,
                                             const float2 *box, const LatticeConst<float> &c) {
    using PS = PartialScreen<NX, NT>;
    if constexpr (!RestScreen<NX, NT>::enabled) {
        return 0.f;  // never called: the kernels screen survivors in full
    } else {
        float2 P[NX];  // P[m] = (u[m, 0], u[m, 1]); only the sites drawn here are read
#pragma unroll
        for (int q = 0; q < PS::NQ; ++q) {
            if (q == 0 || q >= PS::BP - 1) {
                const uint4 b = philox_from_prefix(x, pre[q], rk);
                P[2 * q] = make_float2(Map{}(b.x, box[4 * q]), Map{}(b.y, box[4 * q + 1]));
                P[2 * q + 1] = make_float2(Map{}(b.z, box[4 * q + 2]), Map{}(b.w, box[4 * q + 3]));
            }
        }
        const float2 cadv = make_float2(c.c_adv, c.c_adv), k1 = make_float2(c.k1, c.k1);
        const float2 ncd = make_float2(c.neg_c_dif, c.neg_c_dif), m1 = make_float2(-1.f, -1.f);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < NX; ++m) {
            if (m == 0 || m >= PS::MC - 1) {
                const float2 here = P[m];
                const float2 right = P[(m + 1) % NX];
                const float2 left = P[(m + NX - 1) % NX];
                const float2 t = __ffma2_rn(cadv, __ffma2_rn(m1, left, right), k1);
                float2 R = __ffma2_rn(here, t, swap2(here));
                R = __ffma2_rn(ncd, __fadd2_rn(right, left), R);
                acc = __ffma2_rn(R, R, acc);
            }
        }
        return (acc.x + acc.y) * c.inv_2Dtau;
    }
}

// Running minimum shared across the CTA at fixed points of the sample loop:
// every thread contributes, then every thread reads the same value, so the
// decisions that depend on it do not depend on timing.  S >= 0, so the float
// order equals the order of the bit patterns as signed ints.
__device__ __forceinline__ void share_min(int *s_min, float &m_ref) {
    atomicMin(s_min, __float_as_int(m_ref));
    __syncthreads();
    m_ref = __int_as_float(*s_min);
    __syncthreads();
}

// Count of fully evaluated samples of the chunk, added to the plan's stats.
__device__ __forceinline__ void add_evaluated(unsigned long long *stats, unsigned n_eval, unsigned *s_cnt) {
    if (!stats) return;
    atomicAdd(s_cnt, n_eval);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(stats, static_cast<unsigned long long>(*s_cnt));
}

// The same for the samples the full screen examined (two-stage screens).
__device__ __forceinline__ void add_screened(unsigned long long *screened, unsigned n_full, unsigned *s_cnt) {
    if (!screened) return;
    atomicAdd(s_cnt, n_full);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(screened, static_cast<unsigned long long>(*s_cnt));
}

// The samples of a chunk that ran stage 1 of the two-stage screen.
__device__ __forceinline__ void add_stage1(unsigned long long *stage1, uint64_t cnt) {
    if (stage1 && threadIdx.x == 0) atomicAdd(stage1, static_cast<unsigned long long>(cnt));
}

// ---------------------------------------------------------------------------
// Negligible weights.  A sample whose action exceeds the subvolume's
// smallest action by more than args.skip_window has weight below
// e^-skip_window of the largest; with skip_window = c + ln(n_max) the n_s such
// samples of a subvolume change every sum by less than e^-c relative (the
// largest weight is 1).  Both kernels leave those samples out of the
// products, the weight and the sums.  The reference point m_ref is the
// per-subvolume hint (the smallest FP32 action among the first samples) and
// then the smallest action evaluated so far: shared across the warp after
// every row of samples and across the CTA every kShareRows rows, at fixed
// points, so every decision is reproducible.  m_ref is always the action of
// an evaluated sample (or within FP32 error of one), never far below the
// final shift.
//
// Shift.  Both kernels accumulate w = exp(m_acc - S) with m_acc starting at
// the hint and moving down only when a sample beats it by more than
// kRescaleMargin (FP64: to that sample's action; FP32: by whole multiples of
// ln 2, so the float sums rescale exactly), so the sums are rescaled a
// handful of times and the threads of a CTA mostly share one shift (cheap
// merges).  w <= e^16.
//
// Sums.  The per-thread sums live in shared memory ([k][thread], no bank
// conflicts); they are touched only by the few samples that pass the screen,
// which keeps the registers of the hot loop (Philox, point, FP32 action) low
// enough for four CTAs per SM at 10x2.
// ---------------------------------------------------------------------------
// Rows between the CTA's shares of its smallest action.  A share is a
// barrier: a warp that has just evaluated a queue batch in FP64 (hundreds of
// instructions on a pipe of 2 lanes per SM and clock) holds the CTA there, so
// sharing less often pays; measured on GB300 at 10x2, 128 rows ran the FP64
// step 0.7% faster than 64, and 256 let more samples through to evaluation.
constexpr int kShareRows = 128;
constexpr float kMarginInv = 1.0f / 0.999f;  // the screen's 0.1% margin folded into its threshold
constexpr float kRescaleMargin = 16.f;

__device__ __forceinline__ float warp_min(float x) {
    return __int_as_float(static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned>(__float_as_int(x)))));
}

// Per-thread sums in shared memory: element k of thread t at buf[k * BLOCK + t].
template <typename Real, int K, int BLOCK>
struct SmemSums;

template <int K, int BLOCK>
struct SmemSums<float, K, BLOCK> {  // first-order sums Kahan-compensated
    static constexpr int R = (K - 2) / 3;
    static constexpr int NC = 1 + R;
    static constexpr int WORDS = K + NC;
    float *b;
    __device__ __forceinline__ static bool compensated(int k) { return k == 0 || (k >= 2 && k < 2 + R); }
    __device__ __forceinline__ static int cidx(int k) { return K + (k == 0 ? 0 : k - 1); }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < WORDS; ++k) b[k * BLOCK] = 0.f;
    }
    __device__ __forceinline__ void add(int k, float x) {
        if (compensated(k)) {
            const float sk = b[k * BLOCK], ck = b[cidx(k) * BLOCK];
            const float y = x - ck;
            const float t = sk + y;
            b[cidx(k) * BLOCK] = (t - sk) - y;
            b[k * BLOCK] = t;
        } else {
            b[k * BLOCK] += x;
        }
    }
    __device__ __forceinline__ void scale(int k, float f) {
        b[k * BLOCK] *= f;
        if (compensated(k)) b[cidx(k) * BLOCK] *= f;
    }
    __device__ __forceinline__ double value(int k) const {
        return compensated(k) ? static_cast<double>(b[k * BLOCK]) - static_cast<double>(b[cidx(k) * BLOCK])
                              : static_cast<double>(b[k * BLOCK]);
    }
};

template <int K, int BLOCK>
struct SmemSums<double, K, BLOCK> {
    static constexpr int WORDS = K;
    double *b;
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < K; ++k) b[k * BLOCK] = 0.0;
    }
    __device__ __forceinline__ void add(int k, double x) { b[k * BLOCK] += x; }
    __device__ __forceinline__ void scale(int k, double f) { b[k * BLOCK] *= f; }
    __device__ __forceinline__ double value(int k) const { return b[k * BLOCK]; }
};

// The CTA's record of a chunk, [cnt, m, sums...], reduced straight from the
// shared-memory sums: the CTA shift m_b is the smallest thread shift; each
// thread's factor exp(m_b - m_t) (1 when equal, the common case) goes to
// s_f; then warp w sums elements k = w, w + WARPS, ... over all threads, lane
// l taking threads l, l + 32, ... in order and the lanes combining in a fixed
// butterfly.  Every order is fixed, so the record is reproducible.
// FP32 sums: every thread's shift is the hint moved down by whole steps of
// ln 2 (shift_steps), so m_t - m_b is n ln 2 up to the double roundings of
// those moves, far below half a step, and the factor is exactly 2^-n.  A lane
// then scales its threads' float sums exactly and adds them (and their Kahan
// compensations) in double-float on the FP32 pipe, 16 terms with a relative
// error below 2^-42 of their magnitudes; only its partial and the butterfly
// are double.  (In double the same took a multiply, an add and, per thread,
// an exp on the FP64 pipe, 2 lanes per SM and clock, for every short chunk.)
template <typename Real, int K, int R, int BLOCK>
__device__ __forceinline__ void chunk_record(const SmemSums<Real, K, BLOCK> &acc, double m_t, double *s_f,
                                             double *s_mb, double *out, uint64_t cnt) {
    constexpr int WARPS = BLOCK / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_f[tid] = m_t;
    __syncthreads();
    if (warp == 0) {
        double mn = INFINITY;
        for (int t = lane; t < BLOCK; t += 32) mn = fmin(mn, s_f[t]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        if (lane == 0) *s_mb = mn;
    }
    __syncthreads();
    const double mb = *s_mb;
    if constexpr (std::is_same<Real, float>::value) {
        const double n = (m_t - mb) * (1.0 / kLn2);  // >= 0; NaN or huge: no weight
        s_f[tid] = n < 1000.0 ? ldexp(1.0, -static_cast<int>(rint(n))) : 0.0;
    } else {
        s_f[tid] = (m_t == INFINITY) ? 0.0 : (m_t == mb ? 1.0 : exp(mb - m_t));
    }
    __syncthreads();
    const Real *base = acc.b - tid;  // element k of thread t: sums of thread t
    for (int k = warp; k < K; k += WARPS) {
        const bool sq = second_order(k, R);
        double part = 0.0;
        if constexpr (std::is_same<Real, float>::value) {
            using F32Sums = SmemSums<float, K, BLOCK>;
            DF p{0.f, 0.f};
            for (int t = lane; t < BLOCK; t += 32) {
                const double f = s_f[t];
                const float ff = static_cast<float>(sq ? f * f : f);
                p = df_add_f(p, __fmul_rn(base[k * BLOCK + t], ff));
                if (F32Sums::compensated(k)) p = df_add_f(p, -__fmul_rn(base[F32Sums::cidx(k) * BLOCK + t], ff));
            }
            part = static_cast<double>(p.h) + static_cast<double>(p.l);
        } else {
            for (int t = lane; t < BLOCK; t += 32) {
                SmemSums<Real, K, BLOCK> other{const_cast<Real *>(base) + t};
                const double f = s_f[t];
                part = __dadd_rn(part, __dmul_rn(other.value(k), sq ? f * f : f));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part = __dadd_rn(part, __shfl_xor_sync(0xffffffffu, part, off));
        if (lane == 0) out[2 + k] = part;
    }
    if (tid == 0) {
        out[0] = static_cast<double>(cnt);
        out[1] = mb;
    }
    __syncthreads();
}

template <typename Real, int K, int R, int BLOCK>
__device__ __forceinline__ void accumulate(SmemSums<Real, K, BLOCK> &acc, Real w, const Real (&Q)[R]) {
    acc.add(0, w);
    acc.add(1, w * w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const Real wq = w * Q[r];
        acc.add(2 + r, wq);
        acc.add(2 + R + r, w * wq);
        acc.add(2 + 2 * R + r, wq * wq);
    }
}

// The FP32 evaluation's sums with the products formed on the way: w Q_r =
// fma(w, hi, w lo) from the compensated Q_r = hi + lo, so w Q_r is rounded
// once; no array of products is held.
template <int NX, int NT, int K, int BLOCK>
__device__ __forceinline__ void accumulate_products_df(SmemSums<float, K, BLOCK> &acc, float w,
                                                       const float (&u)[NX * NT]) {
    constexpr int R = NX / 2 + 1;
    acc.add(0, w);
    acc.add(1, w * w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const DF q = product_df<NX, NT>(u, r);
        const float wq = __fmaf_rn(w, q.h, w * q.l);
        acc.add(2 + r, wq);
        acc.add(2 + R + r, w * wq);
        acc.add(2 + 2 * R + r, wq * wq);
    }
}

template <typename Real, int K, int R, int BLOCK>
__device__ __forceinline__ void rescale(SmemSums<Real, K, BLOCK> &acc, Real f) {
    const Real f2 = f * f;
#pragma unroll
    for (int k = 0; k < K; ++k) acc.scale(k, second_order(k, R) ? f2 : f);
}

// Shared state of one CTA for one chunk.
template <int BLOCK>
struct ChunkShared {
    double f[BLOCK];  // per-thread shift factors of the chunk record
    double mb;
    long long next;   // the chunk this CTA takes next
    int left[BLOCK / 32];  // each warp's candidates left at the end of the chunk
    int min_bits;
    unsigned evaluated;
    unsigned screened;
};

// The chunk a CTA takes after chunk c.  With a counter, chunks beyond the
// first grid go to CTAs in the order they finish, so the CTAs that drew
// cheaper chunks take more and the launch ends more evenly; a chunk's record
// depends on the chunk alone, so which CTA takes it changes no result.  Every
// thread of the CTA calls this at the end of the chunk; 'slot' is a
// shared-memory word that nothing else reads, and the next chunk's first
// barrier separates this read from the next write.
__device__ __forceinline__ int64_t next_chunk(const IntegrandArgs &args, int64_t c, long long *slot) {
    if (!args.next_chunk) return c + gridDim.x;
    if (threadIdx.x == 0) *slot = static_cast<long long>(gridDim.x + atomicAdd(args.next_chunk, 1ull));
    __syncthreads();
    return *slot;
}

// ---------------------------------------------------------------------------
// Candidate queues.  The few samples that pass the screen are not evaluated
// where they are found (one or two lanes of a warp, which on GB300's FP64
// pipe, 2 lanes per SM and clock, would hold the whole warp for the full
// warp-width cost of every FP64 instruction).  Each warp appends its
// candidates, in (row, lane) order, to its own queue in shared memory and
// evaluates them 32 at a time with every lane busy; the remainder is
// evaluated at the end of the chunk.  Lane l always takes queue entry l, so
// which lane accumulates which sample, and in what order, is fixed.
// ---------------------------------------------------------------------------
constexpr int kQueueCap = 64;

// Appends this lane's candidate (if any) to the warp's queue; returns the new
// count.  lt = the lanes below this one ((1 << lane) - 1, computed once per
// kernel).  Needs count < 32 on entry (then count < 64 = kQueueCap on exit).
__device__ __forceinline__ int enqueue(uint32_t *q, int count, bool cand, uint32_t k, unsigned lt) {
    const unsigned mask = __ballot_sync(0xffffffffu, cand);
    if (mask == 0u) return count;  // the common case: no candidate in the row (warp-uniform)
    if (cand) q[count + __popc(mask & lt)] = k;
    __syncwarp();
    return count + __popc(mask);
}

// Removes the first 32 entries after a full batch.
__device__ __forceinline__ int dequeue32(uint32_t *q, int count) {
    const int lane = threadIdx.x & 31;
    const uint32_t moved = (lane + 32 < count) ? q[lane + 32] : 0u;
    __syncwarp();
    if (lane + 32 < count) q[lane] = moved;
    __syncwarp();
    return count - 32;
}

// The same for a queue that carries a float beside each entry (a survivor
// and its partial action).
__device__ __forceinline__ int enqueue_pair(uint32_t *q, float *pq, int count, bool cand, uint32_t k, float p,
                                            unsigned lt) {
    const unsigned mask = __ballot_sync(0xffffffffu, cand);
    if (mask == 0u) return count;
    if (cand) {
        const int at = count + __popc(mask & lt);
        q[at] = k;
        pq[at] = p;
    }
    __syncwarp();
    return count + __popc(mask);
}

__device__ __forceinline__ int dequeue32_pair(uint32_t *q, float *pq, int count) {
    const int lane = threadIdx.x & 31;
    const bool mv = lane + 32 < count;
    const uint32_t moved = mv ? q[lane + 32] : 0u;
    const float pmoved = mv ? pq[lane + 32] : 0.f;
    __syncwarp();
    if (mv) {
        q[lane] = moved;
        pq[lane] = pmoved;
    }
    __syncwarp();
    return count - 32;
}

// ---------------------------------------------------------------------------
// FP64 integrand, thread per sample.  One CTA processes chunk blockIdx.x,
// then the chunks next_chunk hands it; within a chunk thread t screens samples
// first + t, first + t + B, ... with the FP32 action of the screen point
// (fast pipes; two stages where the split is compiled, see PartialScreen).  Samples that may carry weight (within skip_window of m_ref, plus
// a margin of 1 + 0.1% of S) go to the warp's
// queue and are evaluated in FP64: Philox words drawn again, FP64 point,
// action, products and weight.  The margin bounds |S_f32(y_f32) - S(y_f64)|:
// the FP32 rounding of the action (~(d + 10) eps_32 S) plus the point
// difference (|y_f32 - y_f64| <= ~1.8e-6 for the screen point, times
// sum_j |dS/dy_j| <= ~52 sqrt(2 d S) for unit parameters: 0.007 at 10x2).
// ---------------------------------------------------------------------------
template <int NX, int NT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, min_blocks<NX, NT>()) integrand_f64(const IntegrandArgs args,
                                                                                 const LatticeConst<double> lc,
                                                                                 const LatticeConst<float> lcf,
                                                                                 const RoundKeys rk) {
    constexpr int D = NX * NT;
    constexpr int R = NX / 2 + 1;
    constexpr int K = sum_count(R);
    constexpr int WARPS = BLOCK / 32;
    __shared__ ChunkShared<BLOCK> sh;
    __shared__ double s_lo[D], s_w[D];
    __shared__ __align__(16) float2 s_box[D];  // (lo', width) as floats for the FP32 screen (MapScreen)
    __shared__ PhiloxPrefix s_pre[(D + 3) / 4];
    __shared__ double s_sums[K * BLOCK];
    __shared__ uint32_t s_queue[WARPS][kQueueCap];
    __shared__ uint32_t s_squeue[PartialScreen<NX, NT>::enabled ? WARPS : 1][kQueueCap];
    __shared__ float s_pqueue[RestScreen<NX, NT>::enabled ? WARPS : 1][kQueueCap];  // survivors' partial actions
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;  // the lanes below this one
    uint32_t *queue = s_queue[tid >> 5];
    uint32_t *squeue = s_squeue[PartialScreen<NX, NT>::enabled ? tid >> 5 : 0];
    float *pqueue = s_pqueue[RestScreen<NX, NT>::enabled ? tid >> 5 : 0];
    SmemSums<double, K, BLOCK> acc{s_sums + tid};

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, &sh.next)) {
        const ChunkView v = chunk_view(args, c, D);
        if (tid < D) {
            s_lo[tid] = v.lo[tid];
            s_w[tid] = v.hi[tid] - v.lo[tid];
            float lo_f, w_f;
            BoxPair<float>::load(v.lo, v.hi, tid, lo_f, w_f);
            s_box[tid] = make_float2(__fmaf_rn(-0.99999994f, w_f, lo_f), w_f);
        }
        chunk_prefixes<D>(v, rk, s_pre);
        const float hint = args.hint[v.s];
        float m_ref = hint;
        // the thread's shift lives in its shared-memory slot (only evaluations touch it)
        double &m_acc = sh.f[tid];
        m_acc = static_cast<double>(hint);
        if (tid == 0) {
            sh.min_bits = __float_as_int(hint);
            sh.evaluated = 0u;
            sh.screened = 0u;
        }
        acc.zero();
        __syncthreads();

        unsigned n_eval = 0;
        int count = 0;
        // low index word of the chunk's first sample: sample offset k has word xb + k (chunks never cross 2^32)
        const uint32_t xb = static_cast<uint32_t>(v.first);
        // FP64 evaluation of queue entry 'lane' (a sample offset in the chunk)
        auto evaluate = [&](uint32_t k) {
            uint32_t w[D];
            sample_words_pre<D>(xb + k, s_pre, rk, w);
            double u[D];
#pragma unroll
            for (int j = 0; j < D; ++j) u[j] = Coord<double>::map(w[j], s_lo[j], s_w[j]);
            const double S = action<NX, NT, double>(u, lc);
            m_ref = fminf(m_ref, __double2float_rn(S));
            double Q[R];
            products<NX, NT, double>(u, Q);
            double m = m_acc;
            if (S < m - kRescaleMargin) {  // rare: move the shift down
                rescale<double, K, R, BLOCK>(acc, exp(S - m));
                m = S;
                m_acc = m;
            }
            accumulate<double, K, R, BLOCK>(acc, exp(m - S), Q);
            ++n_eval;
        };
        // m_ref changes only where the queue is evaluated (then made uniform
        // across the warp) and where the CTA shares it; thr follows it
        float thr = m_ref + args.skip_window + 1.0f;
        // x (1 - 1e-3) <= thr, the screen's 0.1% margin, as x <= thr / (1 - 1e-3)
        float thr_m = thr * kMarginInv;
        // full screen of sample offset k (valid lanes) and the candidate queue
        unsigned n_full = 0;
        // full screen of sample offset k (valid lanes), or with rest (warp-uniform) the survivor's partial
        // action P_f plus the rest of S, then the candidate queue
        const bool rest_ok = RestScreen<NX, NT>::enabled && lcf.half_mass2 == 0.f;
        auto screen = [&](uint32_t k, bool valid, bool rest, float P_f) {
            bool cand = false;
            if (valid) {
                ++n_full;
                const uint32_t x = xb + k;
                const float S_f = rest ? P_f + rest_action<NX, NT, MapScreen>(x, s_pre, rk, s_box, lcf)
                                       : screen_action<NX, NT, MapScreen>(x, s_pre, rk, s_box, lcf);
                cand = S_f <= thr_m;  // S_f <= m_ref + window + 1 + 0.1% of S_f
            }
            count = enqueue(queue, count, cand, k, lt);
            if (count >= 32) {
                evaluate(queue[lane]);
                count = dequeue32(queue, count);
                m_ref = warp_min(m_ref);
                thr = m_ref + args.skip_window + 1.0f;
                thr_m = thr * kMarginInv;
            }
        };
        int scount = 0;  // stage-1 survivors waiting for the full screen
        const uint32_t nrows = static_cast<uint32_t>((v.cnt + BLOCK - 1) / BLOCK);
        const uint32_t nfull = static_cast<uint32_t>(v.cnt / BLOCK);  // rows in which every thread has a sample
        const bool two_stage = PartialScreen<NX, NT>::enabled && nrows >= kTwoStageMinRows;
        // Stage 1 of one row: this thread's sample offset k ('valid' false past the chunk's end), its partial
        // action, the survivor queue.
        auto stage1_row = [&](uint32_t k, bool valid) {
            bool surv = false;
            float P_f = 0.f;
            if (valid) {
                P_f = partial_action<NX, NT, MapScreen>(xb + k, s_pre, rk, s_box, lcf);
                surv = P_f <= thr_m;
            }
            if constexpr (RestScreen<NX, NT>::enabled) {
                scount = enqueue_pair(squeue, pqueue, scount, surv, k, P_f, lt);
                if (scount >= 32) {
                    screen(squeue[lane], true, rest_ok, pqueue[lane]);
                    scount = dequeue32_pair(squeue, pqueue, scount);
                }
            } else {
                scount = enqueue(squeue, scount, surv, k, lt);
                if (scount >= 32) {
                    screen(squeue[lane], true, false, 0.f);
                    scount = dequeue32(squeue, scount);
                }
            }
        };
        auto one_stage_row = [&](uint32_t k, bool valid) { screen(k, valid, false, 0.f); };
        // The rows in blocks of kShareRows, the CTA sharing its smallest action between blocks; in each block the
        // full rows first (no bounds check), then the chunk's ragged last row if it falls there.
        auto rows = [&](auto step) {
            for (uint32_t r0 = 0; r0 < nrows; r0 += kShareRows) {
                const uint32_t r1 = min(r0 + static_cast<uint32_t>(kShareRows), nrows), rf = min(r1, nfull);
                for (uint32_t row = r0; row < rf; ++row) step(row * BLOCK + tid, true);
                for (uint32_t row = rf; row < r1; ++row) step(row * BLOCK + tid, row * BLOCK + tid < v.cnt);
                if (r1 < nrows) {
                    share_min(&sh.min_bits, m_ref);
                    thr = m_ref + args.skip_window + 1.0f;
                    thr_m = thr * kMarginInv;
                }
            }
        };
        if constexpr (PartialScreen<NX, NT>::enabled) {
            if (two_stage)
                rows(stage1_row);
            else
                rows(one_stage_row);
        } else {
            rows(one_stage_row);
        }
        if (scount > 0)  // survivors still queued
            screen(lane < scount ? squeue[lane] : 0u, lane < scount, rest_ok,
                   RestScreen<NX, NT>::enabled && lane < scount ? pqueue[lane] : 0.f);
        // The warps' leftover candidates (fewer than 32 each) are gathered into
        // one list in warp order and evaluated in as few warps as possible:
        // an FP64 evaluation costs its warp the full width of every FP64
        // instruction however few lanes are busy, and at the end of a short
        // chunk every warp would otherwise pay that for one or two candidates
        // at the same time as the others.
        {
            uint32_t *flat = &s_queue[0][0];
            const uint32_t mine = lane < count ? queue[lane] : 0u;
            if (lane == 0) sh.left[warp] = count;
            __syncthreads();
            int off = 0, total = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const int c_w = sh.left[w];
                off += w < warp ? c_w : 0;
                total += c_w;
            }
            if (lane < count) flat[off + lane] = mine;
            __syncthreads();
            if (tid < total) evaluate(flat[tid]);
        }
        add_evaluated(args.stats, n_eval, &sh.evaluated);
        if (PartialScreen<NX, NT>::enabled) add_screened(args.screened, n_full, &sh.screened);
        if (two_stage) add_stage1(args.stage1, v.cnt);
        chunk_record<double, K, R, BLOCK>(acc, double(m_acc), sh.f, &sh.mb, args.partials + c * (K + 2), v.cnt);
    }
}

// ---------------------------------------------------------------------------
// FP32 integrand.  Points, screen, action, products and weights in float;
// per-thread Kahan sums; the log-weight shift and the merges in double.
// Candidates are queued as above and each is evaluated with the compensated
// FP32 action (action_df), the split-argument weight (weight_f32) and the
// compensated products (accumulate_products_df); the shift moves down by
// whole powers of two (shift_steps), so rescaling the sums is exact.  Every
// step of an evaluation then has a bound of a few float roundings, which is
// what the library's stated arithmetic error of a result adds up
// (bfi_error_bound).
// ---------------------------------------------------------------------------

template <int NX, int NT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, min_blocks<NX, NT>()) integrand_f32(const IntegrandArgs args,
                                                                                 const LatticeConst<float> lc,
                                                                                 const LatticeConstDF lcd,
                                                                                 const RoundKeys rk) {
    constexpr int D = NX * NT;
    constexpr int R = NX / 2 + 1;
    constexpr int K = sum_count(R);
    constexpr int WARPS = BLOCK / 32;
    using Sums = SmemSums<float, K, BLOCK>;
    __shared__ ChunkShared<BLOCK> sh;
    __shared__ __align__(16) float2 s_box[D];  // (lo, width) as floats: the evaluation's exact points
    __shared__ __align__(16) float2 s_scr[D];  // (lo', width): the screen's points (MapScreen)
    __shared__ PhiloxPrefix s_pre[(D + 3) / 4];
    __shared__ float s_sums[Sums::WORDS * BLOCK];
    __shared__ uint32_t s_queue[WARPS][kQueueCap];
    __shared__ uint32_t s_squeue[PartialScreen<NX, NT>::enabled ? WARPS : 1][kQueueCap];
    __shared__ float s_pqueue[RestScreen<NX, NT>::enabled ? WARPS : 1][kQueueCap];  // survivors' partial actions
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;  // the lanes below this one
    uint32_t *queue = s_queue[tid >> 5];
    uint32_t *squeue = s_squeue[PartialScreen<NX, NT>::enabled ? tid >> 5 : 0];
    float *pqueue = s_pqueue[RestScreen<NX, NT>::enabled ? tid >> 5 : 0];
    Sums acc{s_sums + tid};

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, &sh.next)) {
        const ChunkView v = chunk_view(args, c, D);
        if (tid < D) {
            float lo_f, w_f;
            BoxPair<float>::load(v.lo, v.hi, tid, lo_f, w_f);
            s_box[tid] = make_float2(lo_f, w_f);
            s_scr[tid] = make_float2(__fmaf_rn(-0.99999994f, w_f, lo_f), w_f);
        }
        chunk_prefixes<D>(v, rk, s_pre);
        const float hint = args.hint[v.s];
        float m_ref = hint;
        // the thread's shift (double) lives in its shared-memory slot: only evaluations touch it
        double &m_acc = sh.f[tid];
        m_acc = static_cast<double>(hint);
        if (tid == 0) {
            sh.min_bits = __float_as_int(hint);
            sh.evaluated = 0u;
            sh.screened = 0u;
        }
        acc.zero();
        __syncthreads();

        unsigned n_eval = 0;
        int count = 0;
        // low index word of the chunk's first sample: sample offset k has word xb + k (chunks never cross 2^32)
        const uint32_t xb = static_cast<uint32_t>(v.first);
        auto evaluate = [&](uint32_t k) {
            float u[D];
            make_point_pre<D>(xb + k, s_pre, rk, s_box, u);
            const DF S = action_df<NX, NT>(u, lcd);
            m_ref = fminf(m_ref, S.h);
            const double S_d = static_cast<double>(S.h) + static_cast<double>(S.l);
            double m = m_acc;
            if (S_d < m - kRescaleMargin) {  // rare: move the shift down by whole powers of two
                const int steps = shift_steps(m, S_d);
                rescale<float, K, R, BLOCK>(acc, pow2_neg(steps));
                m -= steps * kLn2;
                m_acc = m;
            }
            accumulate_products_df<NX, NT, K, BLOCK>(acc, weight_f32(m, S), u);
            ++n_eval;
        };
        // m_ref changes only where the queue is evaluated (then made uniform
        // across the warp) and where the CTA shares it; thr follows it.  The
        // screen keeps a sample when its screen action, less 0.1%, is within
        // the window plus 1 of m_ref: that margin bounds the screen's error
        // against the evaluation's exact float action (its own rounding,
        // ~(d + 10) 2^-24 S, and the folded point, |dy| < 2^-22 |y|), so no
        // sample within the window is dropped.
        float thr = m_ref + args.skip_window + 1.0f;
        float thr_m = thr * kMarginInv;
        unsigned n_full = 0;
        const bool rest_ok = RestScreen<NX, NT>::enabled && lc.half_mass2 == 0.f;
        auto screen = [&](uint32_t k, bool valid, bool rest, float P_f) {
            n_full += valid ? 1u : 0u;
            bool cand = false;
            if (valid) {
                const uint32_t x = xb + k;
                cand = (rest ? P_f + rest_action<NX, NT, MapScreen>(x, s_pre, rk, s_scr, lc)
                             : screen_action<NX, NT, MapScreen>(x, s_pre, rk, s_scr, lc)) <= thr_m;
            }
            count = enqueue(queue, count, cand, k, lt);
            if (count >= 32) {
                evaluate(queue[lane]);
                count = dequeue32(queue, count);
                m_ref = warp_min(m_ref);
                thr = m_ref + args.skip_window + 1.0f;
                thr_m = thr * kMarginInv;
            }
        };
        int scount = 0;  // stage-1 survivors waiting for the full screen
        const uint32_t nrows = static_cast<uint32_t>((v.cnt + BLOCK - 1) / BLOCK);
        const uint32_t nfull = static_cast<uint32_t>(v.cnt / BLOCK);  // rows in which every thread has a sample
        const bool two_stage = PartialScreen<NX, NT>::enabled && nrows >= kTwoStageMinRows;
        // Stage 1 of one row: this thread's sample offset k ('valid' false past the chunk's end), its partial
        // action, the survivor queue.
        auto stage1_row = [&](uint32_t k, bool valid) {
            bool surv = false;
            float P_f = 0.f;
            if (valid) {
                P_f = partial_action<NX, NT, MapScreen>(xb + k, s_pre, rk, s_scr, lc);
                surv = P_f <= thr_m;
            }
            if constexpr (RestScreen<NX, NT>::enabled) {
                scount = enqueue_pair(squeue, pqueue, scount, surv, k, P_f, lt);
                if (scount >= 32) {
                    screen(squeue[lane], true, rest_ok, pqueue[lane]);
                    scount = dequeue32_pair(squeue, pqueue, scount);
                }
            } else {
                scount = enqueue(squeue, scount, surv, k, lt);
                if (scount >= 32) {
                    screen(squeue[lane], true, false, 0.f);
                    scount = dequeue32(squeue, scount);
                }
            }
        };
        auto one_stage_row = [&](uint32_t k, bool valid) { screen(k, valid, false, 0.f); };
        // The rows in blocks of kShareRows, the CTA sharing its smallest action between blocks; in each block the
        // full rows first (no bounds check), then the chunk's ragged last row if it falls there.
        auto rows = [&](auto step) {
            for (uint32_t r0 = 0; r0 < nrows; r0 += kShareRows) {
                const uint32_t r1 = min(r0 + static_cast<uint32_t>(kShareRows), nrows), rf = min(r1, nfull);
                for (uint32_t row = r0; row < rf; ++row) step(row * BLOCK + tid, true);
                for (uint32_t row = rf; row < r1; ++row) step(row * BLOCK + tid, row * BLOCK + tid < v.cnt);
                if (r1 < nrows) {
                    share_min(&sh.min_bits, m_ref);
                    thr = m_ref + args.skip_window + 1.0f;
                    thr_m = thr * kMarginInv;
                }
            }
        };
        if constexpr (PartialScreen<NX, NT>::enabled) {
            if (two_stage)
                rows(stage1_row);
            else
                rows(one_stage_row);
        } else {
            rows(one_stage_row);
        }
        if (scount > 0)  // survivors still queued
            screen(lane < scount ? squeue[lane] : 0u, lane < scount, rest_ok,
                   RestScreen<NX, NT>::enabled && lane < scount ? pqueue[lane] : 0.f);
        if (lane < count) evaluate(queue[lane]);
        add_evaluated(args.stats, n_eval, &sh.evaluated);
        if (PartialScreen<NX, NT>::enabled) add_screened(args.screened, n_full, &sh.screened);
        if (two_stage) add_stage1(args.stage1, v.cnt);
        chunk_record<float, K, R, BLOCK>(acc, double(m_acc), sh.f, &sh.mb, args.partials + c * (K + 2), v.cnt);
    }
}

// Per-subvolume hint: the smallest FP32 action among the subvolume's first
// hint_samples(n_s) samples (n_s/32, at least 256 and at most 4096: a few
// percent of the work at most).  One CTA per subvolume.
__host__ __device__ constexpr uint64_t hint_samples(uint64_t n) {
    return n < 256 ? n : (n / 32 < 256 ? 256 : (n / 32 > 4096 ? 4096 : n / 32));
}

template <int NX, int NT>
__global__ void __launch_bounds__(kBlock) hint_f32(const IntegrandArgs args, const LatticeConst<float> lc,
                                                   const RoundKeys rk) {
    constexpr int D = NX * NT;
    __shared__ int s_min;
    __shared__ __align__(16) float2 s_box[D];
    const int64_t s = blockIdx.x;
    if (threadIdx.x == 0) s_min = __float_as_int(INFINITY);
    if (threadIdx.x < D) BoxPair<float>::load(args.lo + s * D, args.hi + s * D, threadIdx.x, s_box[threadIdx.x].x,
                                              s_box[threadIdx.x].y);
    __syncthreads();
    const uint64_t n = hint_samples(args.samples[s]);
    const uint32_t sid = args.sub_id ? args.sub_id[s] : static_cast<uint32_t>(s);
    float mn = INFINITY;
    for (uint64_t k = threadIdx.x; k < n; k += blockDim.x) {
        float u[D];
        make_point_smem<D>(k, sid, rk, s_box, u);
        mn = fminf(mn, action<NX, NT, float>(u, lc));
    }
    atomicMin(&s_min, __float_as_int(mn));
    __syncthreads();
    if (threadIdx.x == 0) args.hint[s] = __int_as_float(s_min);
}

template <int NX, int NT, typename Real>
__global__ void eval_kernel(const EvalArgs a, const LatticeConst<Real> lc, const LatticeConstDF lcd, bool compensated) {
    constexpr int D = NX * NT;
    constexpr int R = NX / 2 + 1;
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= a.npts) return;
    Real u[D];
#pragma unroll
    for (int j = 0; j < D; ++j) u[j] = static_cast<Real>(a.y[i * D + j]);
    Real Q[R];
    products<NX, NT, Real>(u, Q);
    double S = static_cast<double>(action<NX, NT, Real>(u, lc));
    if constexpr (sizeof(Real) == 4) {
        if (compensated) {
            const DF Sd = action_df<NX, NT>(u, lcd);
            S = static_cast<double>(Sd.h) + static_cast<double>(Sd.l);
        }
    }
    a.S[i] = S;
#pragma unroll
    for (int r = 0; r < R; ++r) a.P[i * R + r] = static_cast<double>(Q[r]) / static_cast<double>(D);
}

// ---------------------------------------------------------------------------
// Host-side launchers and the table of compiled shapes.
// ---------------------------------------------------------------------------
template <typename Real>
inline LatticeConst<Real> make_const(const LatticeParams &p) {
    LatticeConst<Real> c;
    const double c_adv = p.nonlinear * p.tau / (2.0 * p.a);
    const double c_dif = p.nu * p.tau / (p.a * p.a);
    c.c_adv = static_cast<Real>(c_adv);
    c.k1 = static_cast<Real>(2.0 * c_dif - 1.0);
    c.neg_c_dif = static_cast<Real>(-c_dif);
    c.inv_2Dtau = static_cast<Real>(1.0 / (2.0 * p.D * p.tau));
    c.half_mass2 = static_cast<Real>(0.5 * p.mass2);
    return c;
}

inline LatticeConstDF make_const_df(const LatticeParams &p) {
    LatticeConstDF c;
    const double c_dif = p.nu * p.tau / (p.a * p.a);
    c.c_adv = split_df(p.nonlinear * p.tau / (2.0 * p.a));
    c.k1 = split_df(2.0 * c_dif - 1.0);
    c.c_dif = split_df(c_dif);
    c.inv_2Dtau = split_df(1.0 / (2.0 * p.D * p.tau));
    c.half_mass2 = split_df(0.5 * p.mass2);
    return c;
}

template <int NX, int NT, typename Real>
cudaError_t launch_integrand(const IntegrandArgs &args, const LatticeParams &p, uint32_t seed, uint32_t job,
                             int grid, cudaStream_t st) {
    const RoundKeys rk = make_round_keys(seed, job);
    hint_f32<NX, NT><<<static_cast<unsigned>(args.nsub), kBlock, 0, st>>>(args, make_const<float>(p), rk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(Real) == 8)
        integrand_f64<NX, NT, kBlock><<<grid, kBlock, 0, st>>>(args, make_const<double>(p), make_const<float>(p), rk);
    else
        integrand_f32<NX, NT, kBlock><<<grid, kBlock, 0, st>>>(args, make_const<float>(p), make_const_df(p), rk);
    return cudaGetLastError();
}

template <int NX, int NT, typename Real>
cudaError_t occupancy_integrand(int, int, int *blocks_per_sm) {
    if constexpr (sizeof(Real) == 8)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrand_f64<NX, NT, kBlock>, kBlock, 0);
    else
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrand_f32<NX, NT, kBlock>, kBlock, 0);
}

template <int NX, int NT>
cudaError_t launch_eval(const EvalArgs &a, const LatticeParams &p, int mode, cudaStream_t st) {
    const int threads = 128;
    const int64_t blocks = (a.npts + threads - 1) / threads;
    if (blocks == 0) return cudaSuccess;
    if (mode == 0)
        eval_kernel<NX, NT, double><<<static_cast<unsigned>(blocks), threads, 0, st>>>(a, make_const<double>(p),
                                                                                    make_const_df(p), false);
    else
        eval_kernel<NX, NT, float><<<static_cast<unsigned>(blocks), threads, 0, st>>>(a, make_const<float>(p),
                                                                                   make_const_df(p), mode == 2);
    return cudaGetLastError();
}

}  // namespace bfi
