// generic.cu -- warp-per-sample integrand for any lattice shape with
// d = Nx Nt <= kMaxD (Honkonen & Honkonen, arXiv:1803.07560, Eq. (Gen2),
// Sec. 3 and Sec. 4), used for the shapes without a compiled thread-per-sample
// kernel (large lattices such as 32x4 or 64x8, and any other shape).
//
// One warp evaluates one sample at a time: the lanes draw the Philox blocks
// of the sample in parallel and write the coordinates to the warp's slice of
// shared memory; each lane then takes sites j = lane, lane + 32, ... of the
// stencil (neighbours through a per-CTA table: next time slice, and j +- Nt
// for the spatial neighbours), and the lanes own the correlation distances
// r = lane, lane + 32, ...  Sums across lanes are XOR butterflies, which give
// every lane the bit-identical result, so every decision is warp-uniform and
// reproducible.  The same screen / full-evaluation / shifted-weight rules as
// the thread-per-sample kernels apply (integrand_kernels.cuh).
#include "integrand_kernels.cuh"

namespace bfi {
namespace {

constexpr int kGBlock = 128;
constexpr int kGWarps = kGBlock / 32;

struct GenShape {
    int nx, nt, d, R, K, nq;
    int dpad;  // per-warp stride of the point buffers: d rounded up to 4 (vector stores stay aligned)
};

GenShape gen_shape(int nx, int nt) {
    GenShape g;
    g.nx = nx;
    g.nt = nt;
    g.d = nx * nt;
    g.R = nx / 2 + 1;
    g.K = 2 + 3 * g.R;
    g.nq = (g.d + 3) / 4;
    g.dpad = 4 * g.nq;
    return g;
}

// Dynamic shared memory layout of one CTA (byte offsets, 16-aligned).
struct GenLayout {
    int next, box_f, lo_d, w_d, uf, ud, sums, mw, pre4, pre1, fac, mean, zb, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// 'mapped' (the sampler kind of the mapped kernel, 0 for the plain integrand)
// adds the per-warp y / z vectors, and for the Gaussian sampler (2) its
// factor and mean.
__host__ __device__ inline GenLayout gen_layout(const GenShape &g, int mapped = 0) {
    const bool gauss = mapped == 2;
    GenLayout L;
    int o = 0;
    L.next = o;  o = align16(o + 2 * g.d);                    // uint16 next-time-slice index per site
    L.box_f = o; o = align16(o + 8 * g.d);                    // float2 (lo, width)
    L.lo_d = o;  o = align16(o + 8 * g.d);                    // double lo
    L.w_d = o;   o = align16(o + 8 * g.d);                    // double width
    L.uf = o;    o = align16(o + 4 * g.dpad * kGWarps);       // float point per warp
    L.ud = o;    o = align16(o + 8 * g.dpad * kGWarps);       // double point per warp
    L.sums = o;  o = align16(o + 8 * (g.K + g.R + 1) * kGWarps);  // per-warp sums (FP64, or FP32 sums + comps)
    L.mw = o;    o = align16(o + 8 * kGWarps + 16);            // per-warp shift, counter, next chunk
    L.pre4 = o;  o = align16(o + 16 * g.nq);                   // Philox prefixes of the chunk (lane screen):
    L.pre1 = o;  o = align16(o + 4 * g.nq);                    //   words a, g, fk, h as uint4, then l3
    L.fac = o;   if (gauss) o = align16(o + 8 * g.d * g.d);   // factor F, row-major
    L.mean = o;  if (gauss) o = align16(o + 8 * g.d);         // mean
    L.zb = o;    if (mapped) o = align16(o + 8 * g.dpad * kGWarps);  // per warp: y of the range map, or u then z
    L.total = o;
    return L;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const DF o{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
        v = df_add(v, o);
    }
    return v;
}

__device__ __forceinline__ int wrap(int j, int d) { return j >= d ? j - d : (j < 0 ? j + d : j); }

// Four consecutive values at a 16-byte (float) or 32-byte (double) aligned
// address: the warp's slices are 16-aligned and j is a multiple of 4.
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double *p, double a, double b, double c, double d) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}

// S at the point u (shared memory), every lane gets the same value.
template <typename Real>
__device__ Real warp_action(const Real *u, const uint16_t *next, const GenShape &g, const LatticeConst<Real> &c) {
    const int lane = threadIdx.x & 31;
    Real acc = Real(0), s2 = Real(0);
    for (int j = lane; j < g.d; j += 32) {
        const Real here = u[j];
        const Real right = u[wrap(j + g.nt, g.d)];
        const Real left = u[wrap(j - g.nt, g.d)];
        const Real t = fma(c.c_adv, right - left, c.k1);
        Real R = fma(here, t, u[next[j]]);
        R = fma(c.neg_c_dif, right + left, R);
        acc = fma(R, R, acc);
        s2 = fma(here, here, s2);
    }
    acc = warp_sum(acc);
    Real S = acc * c.inv_2Dtau;
    if (c.half_mass2 != Real(0)) S = fma(c.half_mass2, warp_sum(s2), S);
    return S;
}

// The same in compensated FP32 (see action_df).
__device__ DF warp_action_df(const float *u, const uint16_t *next, const GenShape &g, const LatticeConstDF &c) {
    const int lane = threadIdx.x & 31;
    DF acc{0.f, 0.f}, mass{0.f, 0.f};
    for (int j = lane; j < g.d; j += 32) {
        const float here = u[j];
        const float right = u[wrap(j + g.nt, g.d)];
        const float left = u[wrap(j - g.nt, g.d)];
        const DF dx = two_sum(right, -left);
        const DF t = df_add(df_mul(c.c_adv, dx), c.k1);
        const DF q = df_add_f(df_mul_f(t, here), u[next[j]]);
        const DF lr = two_sum(right, left);
        const DF R = df_add(q, df_mul(c.c_dif, DF{-lr.h, -lr.l}));
        DF sq = two_prod(R.h, R.h);
        sq.l = __fmaf_rn(2.f * R.h, R.l, sq.l);
        acc = df_add(acc, sq);
        mass = df_add(mass, two_prod(here, here));
    }
    acc = warp_sum_df(acc);
    DF S = df_mul(acc, c.inv_2Dtau);
    if (c.half_mass2.h != 0.f) S = df_add(S, df_mul(warp_sum_df(mass), c.half_mass2));
    return S;
}

// Q_r = sum_j u_j u_{j + r Nt (mod d)} for the distances r this lane owns
// (r = lane + 32 i), handed to f(r, Q_r).  Each lane starts its sweep at
// j = lane, so at every step the lanes read consecutive words (no bank
// conflicts); the order is fixed per lane, so the result is reproducible.
// FP32 sums are compensated and handed over as hi + lo.
template <typename F>
__device__ __forceinline__ void lane_products(const double *u, const GenShape &g, F f) {
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < g.R; r += 32) {
        double q = 0.0;
        int j = lane % g.d, jr = wrap(j + r * g.nt, g.d);
        for (int t = 0; t < g.d; ++t) {
            q = fma(u[j], u[jr], q);
            j = (j + 1 == g.d) ? 0 : j + 1;
            jr = (jr + 1 == g.d) ? 0 : jr + 1;
        }
        f(r, q);
    }
}

template <typename F>
__device__ __forceinline__ void lane_products(const float *u, const GenShape &g, F f) {
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < g.R; r += 32) {
        DF q{0.f, 0.f};
        int j = lane % g.d, jr = wrap(j + r * g.nt, g.d);
        for (int t = 0; t < g.d; ++t) {
            q = df_add(q, two_prod(u[j], u[jr]));
            j = (j + 1 == g.d) ? 0 : j + 1;
            jr = (jr + 1 == g.d) ? 0 : jr + 1;
        }
        f(r, q);
    }
}

// Philox blocks q = lane, lane + 32, ... of sample i mapped into u; a full
// block is written with one vector store (conflict-free), the ragged last one
// word by word.
template <typename Real, typename Box>
__device__ __forceinline__ void warp_point(uint64_t i, uint32_t sid, const RoundKeys &rk, const GenShape &g, Box box,
                                           Real *u, int n = -1) {
    // coordinates 0 .. n - 1 (n <= 4 nq; default d)
    const int nd = n < 0 ? g.d : n;
    for (int q = threadIdx.x & 31; q < g.nq; q += 32) {
        const uint4 b = philox4x32_10(
            make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), sid), rk);
        const int j = 4 * q;
        if (j + 4 <= nd) {
            store4(u + j, box(j, b.x), box(j + 1, b.y), box(j + 2, b.z), box(j + 3, b.w));
        } else {
            const uint32_t w4[4] = {b.x, b.y, b.z, b.w};
            for (int t = 0; t < 4 && j + t < nd; ++t) u[j + t] = box(j + t, w4[t]);
        }
    }
    __syncwarp();
}

// Per-CTA set-up shared by the kernels: neighbour table (once) and box.
__device__ void load_box(unsigned char *sm, const GenLayout &L, const GenShape &g, const double *lo,
                         const double *hi) {
    float2 *bf = reinterpret_cast<float2 *>(sm + L.box_f);
    double *ld = reinterpret_cast<double *>(sm + L.lo_d);
    double *wd = reinterpret_cast<double *>(sm + L.w_d);
    for (int j = threadIdx.x; j < g.d; j += blockDim.x) {
        bf[j] = make_float2(__double2float_rn(lo[j]), __double2float_rn(hi[j] - lo[j]));
        ld[j] = lo[j];
        wd[j] = hi[j] - lo[j];
    }
}

__device__ void build_next(unsigned char *sm, const GenLayout &L, const GenShape &g) {
    uint16_t *next = reinterpret_cast<uint16_t *>(sm + L.next);
    for (int j = threadIdx.x; j < g.d; j += blockDim.x) {
        const int l = j % g.nt;
        next[j] = static_cast<uint16_t>(l + 1 < g.nt ? j + 1 : j + 1 - g.nt);
    }
}

struct GenArgs {
    IntegrandArgs a;
    GenShape g;
    GenLayout L;
    LatticeConst<float> cf;
    LatticeConst<double> cd;
    LatticeConstDF cdf;
    RoundKeys rk;
};

// ---------------------------------------------------------------------------
// Register-resident FP32 screen for Nx = G SPL.  A group of G lanes (the whole
// warp, or each half of it: two samples per warp) screens one sample, and its
// lane t owns the spatial sites [SPL t, SPL t + SPL) with all NT time slices:
// the coordinates [C t, C t + C), C = SPL NT, which are whole Philox blocks
// (C is a multiple of 4).  It draws its own blocks, keeps the field and the
// chunk's box in registers, and takes the one site of each spatial neighbour
// from lanes t - 1 and t + 1 of its group (2 NT shuffles), so the screen
// touches no shared memory.  For even NT the residuals of slices l and
// l + NT/2 run as one f32x2 pair.  The per-lane residual sums meet in an XOR
// butterfly within the group (bit-identical on its lanes).  Points and
// residuals round as the shared-memory screen's do; only the order of the sum
// differs.  Half-warp groups serve the shapes whose lanes would otherwise own
// a single Philox block (C = 4 at G = 32): the fixed costs of a sample (the
// neighbour shuffles, the butterfly, the screen's decision) then spread over
// twice the sites, and each lane runs two independent Philox chains.
// ---------------------------------------------------------------------------
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int SPL, int NT, int G = 32>
struct LaneScreen {
    static constexpr int C = SPL * NT;
    static_assert(C % 4 == 0, "a lane's coordinates must be whole Philox blocks");
    static_assert(G == 32 || G == 16, "a sample's group is a warp or half of one");
    float lo[C], w[C];

    __device__ __forceinline__ void load(const float2 *bf) {
        const int j0 = (threadIdx.x & (G - 1)) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            lo[c] = bf[j0 + c].x;
            w[c] = bf[j0 + c].y;
        }
    }

    // Where block q = t (C/4) + b of the chunk keeps its Philox prefix: at
    // b G + t, so that the lanes of a group read consecutive words (and the
    // two groups of a warp the same ones).
    __host__ __device__ static int prefix_slot(int q) { return (q % (C / 4)) * G + q / (C / 4); }

    // S of the group's own sample, whose index has low word i (the chunk's
    // prefixes hold the rest), on every lane of the group.
    __device__ __forceinline__ float action(uint32_t i, const uint4 *pre4, const uint32_t *pre1, const RoundKeys &rk,
                                            const LatticeConst<float> &cf) const {
        const int lane = threadIdx.x & 31, t = lane & (G - 1), base = lane - t;
        float X[C];  // X[s NT + l]
#pragma unroll
        for (int b = 0; b < C / 4; ++b) {
            const uint4 a = pre4[b * G + t];
            const PhiloxPrefix p{a.x, a.y, a.z, a.w, pre1[b * G + t], {0u, 0u, 0u}};
            const uint4 r = philox_from_prefix(i, p, rk);
            X[4 * b + 0] = Coord<float>::map(r.x, lo[4 * b + 0], w[4 * b + 0]);
            X[4 * b + 1] = Coord<float>::map(r.y, lo[4 * b + 1], w[4 * b + 1]);
            X[4 * b + 2] = Coord<float>::map(r.z, lo[4 * b + 2], w[4 * b + 2]);
            X[4 * b + 3] = Coord<float>::map(r.w, lo[4 * b + 3], w[4 * b + 3]);
        }
        float left[NT], right[NT];
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            left[l] = __shfl_sync(0xffffffffu, X[(SPL - 1) * NT + l], base + ((t + G - 1) & (G - 1)));
            right[l] = __shfl_sync(0xffffffffu, X[l], base + ((t + 1) & (G - 1)));
        }
        float acc;
        if constexpr (NT % 2 == 0) {
            // slices l and l + NT/2 of a site as one f32x2 pair: the next
            // slice of a pair is the following pair (swapped after the last)
            constexpr int HN = NT / 2;
            const float2 cadv = make_float2(cf.c_adv, cf.c_adv), k1 = make_float2(cf.k1, cf.k1);
            const float2 ncd = make_float2(cf.neg_c_dif, cf.neg_c_dif), m1 = make_float2(-1.f, -1.f);
            float2 a2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int sp = 0; sp < SPL; ++sp) {
#pragma unroll
                for (int l = 0; l < HN; ++l) {
                    const float2 here = make_float2(X[sp * NT + l], X[sp * NT + l + HN]);
                    const float2 nxt = l + 1 < HN ? make_float2(X[sp * NT + l + 1], X[sp * NT + l + 1 + HN])
                                                  : make_float2(X[sp * NT + HN], X[sp * NT]);
                    const float2 r = sp + 1 < SPL ? make_float2(X[(sp + 1) * NT + l], X[(sp + 1) * NT + l + HN])
                                                  : make_float2(right[l], right[l + HN]);
                    const float2 le = sp > 0 ? make_float2(X[(sp - 1) * NT + l], X[(sp - 1) * NT + l + HN])
                                             : make_float2(left[l], left[l + HN]);
                    const float2 t = __ffma2_rn(cadv, __ffma2_rn(m1, le, r), k1);
                    float2 R = __ffma2_rn(here, t, nxt);
                    R = __ffma2_rn(ncd, __fadd2_rn(r, le), R);
                    a2 = __ffma2_rn(R, R, a2);
                }
            }
            acc = a2.x + a2.y;
        } else {
            acc = 0.f;
#pragma unroll
            for (int sp = 0; sp < SPL; ++sp) {
#pragma unroll
                for (int l = 0; l < NT; ++l) {
                    const float here = X[sp * NT + l];
                    const float nxt = X[sp * NT + (l + 1) % NT];
                    const float r = sp + 1 < SPL ? X[(sp + 1) * NT + l] : right[l];
                    const float le = sp > 0 ? X[(sp - 1) * NT + l] : left[l];
                    const float t = fmaf(cf.c_adv, r - le, cf.k1);
                    float R = fmaf(here, t, nxt);
                    R = fmaf(cf.neg_c_dif, r + le, R);
                    acc = fmaf(R, R, acc);
                }
            }
        }
        float S = group_sum<G>(acc) * cf.inv_2Dtau;
        if (cf.half_mass2 != 0.f) {
            float s2 = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) s2 = fmaf(X[c], X[c], s2);
            S = fmaf(cf.half_mass2, group_sum<G>(s2), S);
        }
        return S;
    }
};

// Placeholder screen of the shared-memory path (SPL = 0).
struct NoLaneScreen {
    __device__ __forceinline__ void load(const float2 *) {}
    __host__ __device__ static int prefix_slot(int q) { return q; }
};
template <int SPL, int NT, int G>
struct ScreenOf {
    using type = LaneScreen<SPL, NT, G>;
};
template <int NT, int G>
struct ScreenOf<0, NT, G> {
    using type = NoLaneScreen;
};

// ---------------------------------------------------------------------------
// The integrand.  FP64 = true: FP32 screen, FP64 evaluation; false: FP32
// screen and evaluation with the compensated action near the minimum.  SPL > 0
// takes the register-resident screen (Nx = G SPL, NT time slices; with G = 16
// a warp screens two consecutive samples at once and evaluates the candidates
// among them in sample order); SPL = 0 the shared-memory one, for any shape.
// ---------------------------------------------------------------------------
// 16 coordinates a lane at SPL >= 2 (64x8, 128x4, 256x2, 512x1) compile to 96
// registers without spilling when asked for 5 CTAs per SM (4 otherwise); 32x16
// would spill.  0 asks for no minimum and leaves every other shape to the
// compiler's own allocation (an explicit 1 would let it take up to 255).
template <int SPL, int NT>
constexpr int lane_min_blocks() { return SPL * NT == 16 && SPL >= 2 ? 5 : 0; }

template <bool FP64, int SPL, int NT, int G = 32>
__global__ void __launch_bounds__(kGBlock, lane_min_blocks<SPL, NT>()) generic_integrand(const GenArgs ga) {
    constexpr int P = SPL > 0 ? 32 / G : 1;  // samples a warp screens at once
    extern __shared__ __align__(16) unsigned char sm[];
    const IntegrandArgs &args = ga.a;
    const GenShape &g = ga.g;
    const GenLayout &L = ga.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *next = reinterpret_cast<const uint16_t *>(sm + L.next);
    const float2 *bf = reinterpret_cast<const float2 *>(sm + L.box_f);
    const double *ld = reinterpret_cast<const double *>(sm + L.lo_d);
    const double *wd = reinterpret_cast<const double *>(sm + L.w_d);
    float *uf = reinterpret_cast<float *>(sm + L.uf) + warp * g.dpad;
    double *ud = reinterpret_cast<double *>(sm + L.ud) + warp * g.dpad;
    double *mw = reinterpret_cast<double *>(sm + L.mw);
    unsigned *cnt_all = reinterpret_cast<unsigned *>(mw + kGWarps);
    long long *next_slot = reinterpret_cast<long long *>(mw + kGWarps + 1);
    // per-warp sums: FP64 -> double[K]; FP32 -> float[K] then float comps[1 + R]
    double *sd = reinterpret_cast<double *>(sm + L.sums) + warp * (g.K + g.R + 1);
    float *sf = reinterpret_cast<float *>(sm + L.sums) + warp * 2 * (g.K + g.R + 1);
    float *cf = sf + g.K;
    build_next(sm, L, g);

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, next_slot)) {
        const ChunkView v = chunk_view(args, c, g.d);
        __syncthreads();  // the previous chunk's readers of box and sums are done
        load_box(sm, L, g, v.lo, v.hi);
        for (int k = lane; k < g.K + g.R + 1; k += 32) {
            if (FP64) sd[k] = 0.0; else { sf[2 * k] = 0.f; sf[2 * k + 1] = 0.f; }
        }
        if (tid == 0) *cnt_all = 0u;
        __syncthreads();
        typename ScreenOf<SPL, NT, G>::type scr;
        scr.load(bf);
        // the chunk's Philox prefixes: the sample index's high word and the sub_id are fixed within a chunk
        uint4 *pre4 = reinterpret_cast<uint4 *>(sm + L.pre4);
        uint32_t *pre1 = reinterpret_cast<uint32_t *>(sm + L.pre1);
        if constexpr (SPL > 0) {
            for (int q = tid; q < g.nq; q += kGBlock) {
                const PhiloxPrefix p = philox_prefix(static_cast<uint32_t>(q), static_cast<uint32_t>(v.first >> 32),
                                                     v.sid, ga.rk);
                const int at = decltype(scr)::prefix_slot(q);
                pre4[at] = make_uint4(p.a, p.g, p.fk, p.h);
                pre1[at] = p.l3;
            }
            __syncthreads();
        }
        const float hint = args.hint[v.s];
        float m_ref = hint;
        double m_acc = static_cast<double>(hint);
        unsigned n_eval = 0;
        // sample offsets in the chunk are 32-bit (a chunk never crosses a multiple of 2^32)
        const uint32_t cnt = static_cast<uint32_t>(v.cnt), xb = static_cast<uint32_t>(v.first);
        for (uint32_t k0 = static_cast<uint32_t>(warp) * P; k0 < cnt; k0 += kGWarps * P) {
            // the screen of samples k0 .. k0 + P - 1 (group p of the warp screens k0 + p)
            float S_group;
            if constexpr (SPL > 0) {
                S_group = scr.action(xb + k0 + (P > 1 ? lane / G : 0), pre4, pre1, ga.rk, ga.cf);
            } else {
                warp_point<float>(v.first + k0, v.sid, ga.rk, g, [&](int j, uint32_t w) { return Coord<float>::map(w, bf[j].x, bf[j].y); }, uf);
                S_group = warp_action<float>(uf, next, g, ga.cf);
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const uint32_t k = k0 + p;
                if (P > 1 && k >= cnt) break;  // the chunk's ragged end (warp-uniform)
                const uint64_t i = v.first + k;
                const float S_f = P > 1 ? __shfl_sync(0xffffffffu, S_group, p * G) : S_group;
                if (FP64) {
                    if (!(S_f <= m_ref + args.skip_window + 1.0f + 1e-3f * S_f)) continue;
                    warp_point<double>(i, v.sid, ga.rk, g, [&](int j, uint32_t w) { return Coord<double>::map(w, ld[j], wd[j]); }, ud);
                    const double S = warp_action<double>(ud, next, g, ga.cd);
                    m_ref = fminf(m_ref, __double2float_rn(S));
                    if (S < m_acc - kRescaleMargin) {
                        const double f = exp(S - m_acc), f2 = f * f;
                        for (int kk = lane; kk < g.K; kk += 32) sd[kk] *= second_order(kk, g.R) ? f2 : f;
                        m_acc = S;
                        __syncwarp();  // another lane owns some of the sums it rescaled
                    }
                    const double w = exp(m_acc - S);
                    if (lane == 0) {
                        sd[0] += w;
                        sd[1] += w * w;
                    }
                    lane_products(ud, g, [&](int r, double q) {
                        const double wq = w * q;
                        sd[2 + r] += wq;
                        sd[2 + g.R + r] += w * wq;
                        sd[2 + 2 * g.R + r] += wq * wq;
                    });
                } else {
                    // the screen's margin, as in FP64 mode: no sample within the window is dropped
                    if (!(S_f <= m_ref + args.skip_window + 1.0f + 1e-3f * S_f)) continue;
                    if constexpr (SPL > 0)  // the evaluation reads the point from shared memory
                        warp_point<float>(i, v.sid, ga.rk, g, [&](int j, uint32_t w) { return Coord<float>::map(w, bf[j].x, bf[j].y); }, uf);
                    // every candidate: compensated action, exact power-of-two shift moves, split-argument weight
                    const DF S = warp_action_df(uf, next, g, ga.cdf);
                    m_ref = fminf(m_ref, S.h);
                    const double S_d = static_cast<double>(S.h) + static_cast<double>(S.l);
                    if (S_d < m_acc - kRescaleMargin) {
                        const int steps = shift_steps(m_acc, S_d);
                        const float f = pow2_neg(steps), f2 = f * f;
                        for (int kk = lane; kk < g.K; kk += 32) sf[kk] *= second_order(kk, g.R) ? f2 : f;
                        for (int kk = lane; kk < 1 + g.R; kk += 32) cf[kk] *= f;
                        m_acc -= steps * kLn2;
                        __syncwarp();  // another lane owns some of the sums it rescaled
                    }
                    const float w = weight_f32(m_acc, S);
                    auto kahan = [&](int k, int ci, float x) {
                        const float y = x - cf[ci];
                        const float t = sf[k] + y;
                        cf[ci] = (t - sf[k]) - y;
                        sf[k] = t;
                    };
                    if (lane == 0) {
                        kahan(0, 0, w);
                        sf[1] += w * w;
                    }
                    lane_products(uf, g, [&](int r, DF q) {
                        const float wq = __fmaf_rn(w, q.h, w * q.l);  // w Q_r rounded once
                        kahan(2 + r, 1 + r, wq);
                        sf[2 + g.R + r] += w * wq;
                        sf[2 + 2 * g.R + r] += wq * wq;
                    });
                }
                ++n_eval;
                __syncwarp();
            }
        }
        if (lane == 0) {
            mw[warp] = m_acc;
            atomicAdd(cnt_all, n_eval);
        }
        __syncthreads();
        // chunk record: warps merged in order at the smallest warp shift
        double mb = mw[0];
        for (int w = 1; w < kGWarps; ++w) mb = fmin(mb, mw[w]);
        double *out = args.partials + c * (g.K + 2);
        for (int k = tid; k < g.K; k += kGBlock) {
            const bool sq = second_order(k, g.R);
            double acc = 0.0;
            for (int w = 0; w < kGWarps; ++w) {
                const double f = mw[w] == mb ? 1.0 : exp(mb - mw[w]);
                double val;
                if (FP64) {
                    val = reinterpret_cast<const double *>(sm + L.sums)[w * (g.K + g.R + 1) + k];
                } else {
                    const float *s = reinterpret_cast<const float *>(sm + L.sums) + w * 2 * (g.K + g.R + 1);
                    const bool comp = k == 0 || (k >= 2 && k < 2 + g.R);
                    val = static_cast<double>(s[k]);
                    if (comp) val -= static_cast<double>(s[g.K + (k == 0 ? 0 : k - 1)]);
                }
                acc = __dadd_rn(acc, __dmul_rn(val, sq ? f * f : f));
            }
            out[2 + k] = acc;
        }
        if (tid == 0) {
            out[0] = static_cast<double>(v.cnt);
            out[1] = mb;
            if (args.stats) atomicAdd(args.stats, static_cast<unsigned long long>(*cnt_all));
        }
    }
}

// ---------------------------------------------------------------------------
// Mapped samplers, FP64.  The unit point goes through a map to the field v
// and the log-Jacobian joins the action, S_eff = S(v) - ln J:
//   KIND 1 (the range map of Sec. 4): y uniform in the box (inside
//          [-1,1]^d), v_j = y_j / (1 - y_j^2), ln J = sum_j ln(1 + y_j^2)
//          - 2 ln(1 - y_j^2);
//   KIND 2 (Gaussian importance sampling): z standard normal from the unit
//          point in Box-Muller pairs (box_muller), v = mean + F z,
//          ln J = |z|^2 / 2 (the rest of 1/q goes into the record's
//          log-volume on the host); samples outside the box [lo, hi) have
//          weight 0.
// Every sample is evaluated in FP64: a map stretches the coordinates, so the
// FP32 screen's bound on |S_f32 - S| does not hold.  Each warp's shift starts
// above every action (kNoShift) and drops to the first sample's S_eff.
// ---------------------------------------------------------------------------
constexpr double kNoShift = 1e300;

template <int KIND>
__global__ void __launch_bounds__(kGBlock) generic_mapped(const GenArgs ga, const MapArgs mp) {
    extern __shared__ __align__(16) unsigned char sm[];
    const IntegrandArgs &args = ga.a;
    const GenShape &g = ga.g;
    const GenLayout &L = ga.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *next = reinterpret_cast<const uint16_t *>(sm + L.next);
    double *lo_s = reinterpret_cast<double *>(sm + L.lo_d);
    double *b_s = reinterpret_cast<double *>(sm + L.w_d);  // KIND 1: width; KIND 2: upper bound
    double *ud = reinterpret_cast<double *>(sm + L.ud) + warp * g.dpad;
    double *zb = reinterpret_cast<double *>(sm + L.zb) + warp * g.dpad;  // y (KIND 1) or u, then z (KIND 2)
    double *fac = reinterpret_cast<double *>(sm + L.fac);
    double *mean = reinterpret_cast<double *>(sm + L.mean);
    double *mw = reinterpret_cast<double *>(sm + L.mw);
    unsigned *cnt_all = reinterpret_cast<unsigned *>(mw + kGWarps);
    long long *next_slot = reinterpret_cast<long long *>(mw + kGWarps + 1);
    double *sd = reinterpret_cast<double *>(sm + L.sums) + warp * (g.K + g.R + 1);
    build_next(sm, L, g);
    if (KIND == 2) {  // the factor transposed (fac[j d + r] = F[r][j]): lane r reads consecutive words
        for (int k = tid; k < g.d * g.d; k += kGBlock) fac[(k % g.d) * g.d + k / g.d] = mp.factor[k];
        for (int k = tid; k < g.d; k += kGBlock) mean[k] = mp.mean ? mp.mean[k] : 0.0;
    }

    for (int64_t c = blockIdx.x; c < args.nchunks; c = next_chunk(args, c, next_slot)) {
        const ChunkView v = chunk_view(args, c, g.d);
        __syncthreads();  // the previous chunk's readers of box and sums are done
        for (int j = tid; j < g.d; j += kGBlock) {
            lo_s[j] = v.lo[j];
            b_s[j] = KIND == 1 ? v.hi[j] - v.lo[j] : v.hi[j];
        }
        for (int k = lane; k < g.K; k += 32) sd[k] = 0.0;
        if (tid == 0) *cnt_all = 0u;
        __syncthreads();
        double m_acc = kNoShift;
        unsigned n_eval = 0;
        for (uint64_t k = warp; k < v.cnt; k += kGWarps) {
            const uint64_t i = v.first + k;
            double part = 0.0;  // this lane's share of ln J
            bool inside = true;
            // the Philox blocks are drawn by lanes q = lane (4 words each); the
            // per-coordinate maps then run on lanes j = lane, lane + 32, ...
            if (KIND == 1) {
                warp_point<double>(i, v.sid, ga.rk, g, [&](int j, uint32_t w) {
                    return Coord<double>::map(w, lo_s[j], b_s[j]);
                }, zb);
                for (int j = lane; j < g.d; j += 32) {
                    const double y = zb[j];
                    const double one_m = (1.0 - y) * (1.0 + y);
                    part += log1p(y * y) - 2.0 * log(one_m);
                    ud[j] = y / one_m;
                }
            } else {
                // the unit point with one more coordinate for odd d (word d of
                // the last block), then z in Box-Muller pairs, one pair a lane
                warp_point<double>(i, v.sid, ga.rk, g, [&](int j, uint32_t w) { return unit_f64(w); }, zb,
                                   g.d + (g.d & 1));
                for (int j = 2 * lane; j < g.d; j += 64) {
                    double z0, z1;
                    box_muller(zb[j], zb[j + 1], z0, z1);
                    part += z0 * z0;
                    zb[j] = z0;
                    if (j + 1 < g.d) {
                        part += z1 * z1;
                        zb[j + 1] = z1;
                    }
                }
                part *= 0.5;
                __syncwarp();
                for (int r = lane; r < g.d; r += 32) {  // v = mean + F z, one row per lane
                    double acc = mean[r];
                    for (int j = 0; j < g.d; ++j) acc = fma(fac[j * g.d + r], zb[j], acc);
                    ud[r] = acc;
                    inside = inside && acc >= lo_s[r] && acc < b_s[r];
                }
            }
            __syncwarp();
            const double ljac = warp_sum(part);
            if (KIND == 2 && !__all_sync(0xffffffffu, inside)) continue;  // weight 0, counted in n
            const double S = warp_action<double>(ud, next, g, ga.cd) - ljac;
            if (S < m_acc - kRescaleMargin) {
                const double f = exp(S - m_acc), f2 = f * f;
                for (int kk = lane; kk < g.K; kk += 32) sd[kk] *= second_order(kk, g.R) ? f2 : f;
                m_acc = S;
                __syncwarp();  // another lane owns some of the sums it rescaled
            }
            const double w = exp(m_acc - S);
            if (lane == 0) {
                sd[0] += w;
                sd[1] += w * w;
            }
            lane_products(ud, g, [&](int r, double q) {
                const double wq = w * q;
                sd[2 + r] += wq;
                sd[2 + g.R + r] += w * wq;
                sd[2 + 2 * g.R + r] += wq * wq;
            });
            ++n_eval;
            __syncwarp();
        }
        if (lane == 0) {
            mw[warp] = m_acc;
            atomicAdd(cnt_all, n_eval);
        }
        __syncthreads();
        // chunk record: warps merged in order at the smallest warp shift
        double mb = mw[0];
        for (int w = 1; w < kGWarps; ++w) mb = fmin(mb, mw[w]);
        double *out = args.partials + c * (g.K + 2);
        for (int k = tid; k < g.K; k += kGBlock) {
            const bool sq = second_order(k, g.R);
            double acc = 0.0;
            for (int w = 0; w < kGWarps; ++w) {
                const double f = mw[w] == mb ? 1.0 : exp(mb - mw[w]);
                const double val = reinterpret_cast<const double *>(sm + L.sums)[w * (g.K + g.R + 1) + k];
                acc = __dadd_rn(acc, __dmul_rn(val, sq ? f * f : f));
            }
            out[2 + k] = acc;
        }
        if (tid == 0) {
            out[0] = static_cast<double>(v.cnt);
            out[1] = mb == kNoShift ? INFINITY : mb;  // no sample with weight in the chunk
            if (args.stats) atomicAdd(args.stats, static_cast<unsigned long long>(*cnt_all));
        }
    }
}

// Per-subvolume reference action: the smallest FP32 action among the first
// hint_samples(n_s) samples.  One CTA per subvolume, warp per sample.
__global__ void __launch_bounds__(kGBlock) generic_hint(const GenArgs ga) {
    extern __shared__ __align__(16) unsigned char sm[];
    const IntegrandArgs &args = ga.a;
    const GenShape &g = ga.g;
    const GenLayout &L = ga.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t s = blockIdx.x;
    int *s_min = reinterpret_cast<int *>(sm + L.mw);
    build_next(sm, L, g);
    load_box(sm, L, g, args.lo + s * g.d, args.hi + s * g.d);
    if (threadIdx.x == 0) *s_min = __float_as_int(INFINITY);
    __syncthreads();
    const uint16_t *next = reinterpret_cast<const uint16_t *>(sm + L.next);
    const float2 *bf = reinterpret_cast<const float2 *>(sm + L.box_f);
    float *uf = reinterpret_cast<float *>(sm + L.uf) + warp * g.dpad;
    const uint32_t sid = args.sub_id ? args.sub_id[s] : static_cast<uint32_t>(s);
    const uint64_t n = hint_samples(args.samples[s]);
    float mn = INFINITY;
    for (uint64_t k = warp; k < n; k += kGWarps) {
        warp_point<float>(k, sid, ga.rk, g, [&](int j, uint32_t w) { return Coord<float>::map(w, bf[j].x, bf[j].y); }, uf);
        mn = fminf(mn, warp_action<float>(uf, next, g, ga.cf));
        __syncwarp();
    }
    if (lane == 0) atomicMin(s_min, __float_as_int(mn));
    __syncthreads();
    if (threadIdx.x == 0) args.hint[s] = __int_as_float(*s_min);
}

// Action and products at given points, one warp per point.
__global__ void __launch_bounds__(kGBlock) generic_eval(const EvalArgs a, const GenArgs ga, int mode) {
    extern __shared__ __align__(16) unsigned char sm[];
    const GenShape &g = ga.g;
    const GenLayout &L = ga.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    build_next(sm, L, g);
    __syncthreads();
    const int64_t i = blockIdx.x * static_cast<int64_t>(kGWarps) + warp;
    if (i >= a.npts) return;  // warp-uniform
    const uint16_t *next = reinterpret_cast<const uint16_t *>(sm + L.next);
    float *uf = reinterpret_cast<float *>(sm + L.uf) + warp * g.dpad;
    double *ud = reinterpret_cast<double *>(sm + L.ud) + warp * g.dpad;
    for (int j = lane; j < g.d; j += 32) {
        ud[j] = a.y[i * g.d + j];
        uf[j] = static_cast<float>(a.y[i * g.d + j]);
    }
    __syncwarp();
    double S;
    if (mode == 0) {
        S = warp_action<double>(ud, next, g, ga.cd);
        lane_products(ud, g, [&](int r, double q) { a.P[i * g.R + r] = q / g.d; });
    } else {
        if (mode == 2) {
            const DF Sd = warp_action_df(uf, next, g, ga.cdf);
            S = static_cast<double>(Sd.h) + static_cast<double>(Sd.l);
        } else {
            S = static_cast<double>(warp_action<float>(uf, next, g, ga.cf));
        }
        lane_products(uf, g, [&](int r, DF q) { a.P[i * g.R + r] = static_cast<double>(q.h + q.l) / g.d; });
    }
    if (lane == 0) a.S[i] = S;
}

GenArgs make_gen_args(const IntegrandArgs &a, const LatticeParams &p, uint32_t seed, uint32_t job) {
    GenArgs ga;
    ga.a = a;
    ga.g = gen_shape(p.nx, p.nt);
    ga.L = gen_layout(ga.g);
    ga.cf = make_const<float>(p);
    ga.cd = make_const<double>(p);
    ga.cdf = make_const_df(p);
    ga.rk = make_round_keys(seed, job);
    return ga;
}

template <bool FP64, int SPL = 0, int NT = 0, int G = 32>
cudaError_t gen_integrand_launcher(const IntegrandArgs &args, const LatticeParams &p, uint32_t seed, uint32_t job,
                                   int grid, cudaStream_t st) {
    const GenArgs ga = make_gen_args(args, p, seed, job);
    cudaError_t e = cudaFuncSetAttribute(generic_hint, cudaFuncAttributeMaxDynamicSharedMemorySize, ga.L.total);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(generic_integrand<FP64, SPL, NT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 ga.L.total);
    if (e != cudaSuccess) return e;
    generic_hint<<<static_cast<unsigned>(args.nsub), kGBlock, ga.L.total, st>>>(ga);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    generic_integrand<FP64, SPL, NT, G><<<grid, kGBlock, ga.L.total, st>>>(ga);
    return cudaGetLastError();
}

template <bool FP64, int SPL = 0, int NT = 0, int G = 32>
cudaError_t gen_occupancy(int nx, int nt, int *blocks_per_sm) {
    const GenLayout L = gen_layout(gen_shape(nx, nt));
    cudaError_t e = cudaFuncSetAttribute(generic_integrand<FP64, SPL, NT, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, generic_integrand<FP64, SPL, NT, G>, kGBlock,
                                                         L.total);
}

cudaError_t gen_eval(const EvalArgs &a, const LatticeParams &p, int mode, cudaStream_t st) {
    if (a.npts == 0) return cudaSuccess;
    IntegrandArgs none{};
    const GenArgs ga = make_gen_args(none, p, 0, 0);
    cudaError_t e = cudaFuncSetAttribute(generic_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, ga.L.total);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.npts + kGWarps - 1) / kGWarps;
    generic_eval<<<static_cast<unsigned>(blocks), kGBlock, ga.L.total, st>>>(a, ga, mode);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t mapped_launcher(const IntegrandArgs &args, const LatticeParams &p, const MapArgs &m, uint32_t seed,
                            uint32_t job, int grid, cudaStream_t st) {
    GenArgs ga = make_gen_args(args, p, seed, job);
    ga.L = gen_layout(ga.g, KIND);
    cudaError_t e = cudaFuncSetAttribute(generic_mapped<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, ga.L.total);
    if (e != cudaSuccess) return e;
    generic_mapped<KIND><<<grid, kGBlock, ga.L.total, st>>>(ga, m);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t mapped_occupancy(int nx, int nt, int *blocks_per_sm) {
    const GenLayout L = gen_layout(gen_shape(nx, nt), KIND);
    cudaError_t e = cudaFuncSetAttribute(generic_mapped<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, generic_mapped<KIND>, kGBlock, L.total);
}

const ShapeKernels kGeneric = {0, 0, 1, {gen_integrand_launcher<true>, gen_integrand_launcher<false>},
                               {gen_occupancy<true>, gen_occupancy<false>}, gen_eval, nullptr, nullptr, nullptr, nullptr, 0};

// Shapes with Nx = G SPL and SPL NT in {4, 8, 16}: the register-resident
// screen.  The shapes whose lanes would own one Philox block each (32x4, 64x2,
// 128x1) screen two samples per warp in half-warp groups, eight coordinates a
// lane.
#define BFI_LANES(SPL, NT, G)                                                                                     \
    {G * SPL, NT, 1, {gen_integrand_launcher<true, SPL, NT, G>, gen_integrand_launcher<false, SPL, NT, G>},      \
     {gen_occupancy<true, SPL, NT, G>, gen_occupancy<false, SPL, NT, G>}, gen_eval, nullptr, nullptr, nullptr, \
     nullptr, 0}
const ShapeKernels kLanes[] = {BFI_LANES(2, 4, 16), BFI_LANES(1, 8, 32), BFI_LANES(1, 16, 32), BFI_LANES(4, 2, 16),
                               BFI_LANES(2, 4, 32), BFI_LANES(2, 8, 32), BFI_LANES(8, 1, 16), BFI_LANES(4, 2, 32),
                               BFI_LANES(4, 4, 32), BFI_LANES(8, 1, 32), BFI_LANES(8, 2, 32), BFI_LANES(16, 1, 32)};
#undef BFI_LANES

}  // namespace

cudaError_t launch_mapped(const IntegrandArgs &a, const LatticeParams &p, const MapArgs &m, uint32_t seed, uint32_t job,
                          int grid, cudaStream_t st) {
    if (m.kind == 1) return mapped_launcher<1>(a, p, m, seed, job, grid, st);
    if (m.kind == 2) return mapped_launcher<2>(a, p, m, seed, job, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t occupancy_mapped(int nx, int nt, int kind, int *blocks_per_sm) {
    if (kind == 1) return mapped_occupancy<1>(nx, nt, blocks_per_sm);
    if (kind == 2) return mapped_occupancy<2>(nx, nt, blocks_per_sm);
    return cudaErrorInvalidValue;
}

const ShapeKernels *generic_shape(int nx, int nt) {
    if (nx < 2 || nt < 1 || nx * nt > kMaxD) return nullptr;
    for (const ShapeKernels &k : kLanes)
        if (k.nx == nx && k.nt == nt) return &k;
    return &kGeneric;
}

}  // namespace bfi
