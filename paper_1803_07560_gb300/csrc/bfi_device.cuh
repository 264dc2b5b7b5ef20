// bfi_device.cuh -- device building blocks of the lattice Burgers integrand
// (Honkonen & Honkonen, arXiv:1803.07560): the Philox4x32-10 point generator,
// the uniform-to-box map, the action of Eq. (Gen2), the equal-time products,
// per-thread shifted accumulators and the merge of shifted records.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfi {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  The per-round keys are
// precomputed once per job (key + r * Weyl constant) and passed in the kernel
// parameters, so the XOR with the key reads the constant bank.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline RoundKeys make_round_keys(uint32_t seed, uint32_t job_id) {
    RoundKeys rk;
    uint32_t a = seed, b = job_id;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += kPhiloxW0;
        b += kPhiloxW1;
    }
    return rk;
}

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

// Rounds r0..9 of Philox4x32-10 on the state c.
__host__ __device__ __forceinline__ uint4 philox_rounds(uint4 c, const RoundKeys &rk, int r0) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int r = r0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi0 = mulhi32(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        const uint32_t hi1 = mulhi32(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) { return philox_rounds(c, rk, 0); }

// ---------------------------------------------------------------------------
// Philox4x32-10 with a per-chunk prefix.  The counters of one chunk differ
// only in the low index word x: (q, x, h, s) with the block q, the high index
// word h (chunks are a power-of-two number of samples, aligned, so they never
// cross a multiple of 2^32) and sub_id s fixed.  In round 1 both products
// (of q and of h) are then fixed, in round 2 the product of word 2, in round
// 3 the product of word 0; philox_prefix folds those, with the round keys
// they meet, into five words, and philox_from_prefix finishes from x with
// 16 of the 20 products.  The result equals philox4x32_10((q, x, h, s)).
// ---------------------------------------------------------------------------
struct __align__(16) PhiloxPrefix {
    uint32_t a;    // round 1: word 0 = a ^ x
    uint32_t g;    // round 2: word 2 = hi(M0 word0) ^ g
    uint32_t fk;   // round 3: word 0 = hi(M1 word2) ^ fk
    uint32_t h;    // round 3: word 2 = h ^ lo(M0 word0 of round 2)
    uint32_t l3;   // round 3: word 3
    uint32_t pad[3];
};

__host__ __device__ __forceinline__ PhiloxPrefix philox_prefix(uint32_t q, uint32_t h, uint32_t s,
                                                               const RoundKeys &rk) {
    // round 1 from (q, x, h, s): (hi(M1 h) ^ x ^ k0, lo(M1 h), hi(M0 q) ^ s ^ k1, lo(M0 q))
    const uint32_t w1 = kPhiloxM1 * h, w2 = mulhi32(kPhiloxM0, q) ^ s ^ rk.k1[0], w3 = kPhiloxM0 * q;
    // round 2: word 0 = hi(M1 w2) ^ w1 ^ k0 and word 1 = lo(M1 w2) are fixed
    const uint32_t e = mulhi32(kPhiloxM1, w2) ^ w1 ^ rk.k0[1], f = kPhiloxM1 * w2;
    PhiloxPrefix p;
    p.a = mulhi32(kPhiloxM1, h) ^ rk.k0[0];
    p.g = w3 ^ rk.k1[1];
    // round 3: the product of word 0 (= e) is fixed
    p.fk = f ^ rk.k0[2];
    p.h = mulhi32(kPhiloxM0, e) ^ rk.k1[2];
    p.l3 = kPhiloxM0 * e;
    return p;
}

__host__ __device__ __forceinline__ uint4 philox_from_prefix(uint32_t x, const PhiloxPrefix &p, const RoundKeys &rk) {
    const uint32_t c0 = p.a ^ x;                                   // round 1
    const uint32_t c2 = mulhi32(kPhiloxM0, c0) ^ p.g, c3 = kPhiloxM0 * c0;   // round 2
    const uint4 c = make_uint4(mulhi32(kPhiloxM1, c2) ^ p.fk, kPhiloxM1 * c2, p.h ^ c3, p.l3);  // round 3
    return philox_rounds(c, rk, 3);
}

// ---------------------------------------------------------------------------
// Uniform (0,1) from one 32-bit word, built from the exponent bits so that no
// integer-to-float conversion is issued:
//   float:  1 + (w>>9) 2^-23 in [1,2), minus (1 - 2^-24)  =  ((w>>9) + 0.5) 2^-23
//   double: 1 + w 2^-32 in [1,2),      minus (1 - 2^-33)  =  (w + 0.5) 2^-32
// Both subtractions are exact (the results have 24 and 33 significant bits).
// In float the exponent and the top word bits are joined by one funnel shift:
// shifting (0x7f : w) right by 9 gives 0x3f800000 | (w >> 9).  (In the FP64
// kernel's screen the constant it holds costs a spill, so that kernel keeps
// the shift-and-or form, with the same bits.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float unit_f32(uint32_t w) {
    return __uint_as_float(__funnelshift_r(w, 0x7fu, 9)) - 0.99999994f;
}

__device__ __forceinline__ double unit_f64(uint32_t w) {
    return __hiloint2double(static_cast<int>(0x3ff00000u | (w >> 12)), static_cast<int>(w << 20)) -
           0.99999999988358467817306518554688;  // 1 - 2^-33
}

// Standard normal pair from two unit coordinates (Box & Muller, 1958):
// z0 = r cos(2 pi u2), z1 = r sin(2 pi u2) with r = sqrt(-2 ln u1); u1 > 0
// always (a unit coordinate lies in (0, 1)).  One logarithm, one square root
// and one sincospi give two normals, where Phi^-1 costs about as much as all
// three for each one.
__device__ __forceinline__ void box_muller(double u1, double u2, double &z0, double &z1) {
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

template <typename Real>
struct Coord;

template <>
struct Coord<float> {
    __device__ __forceinline__ static float map(uint32_t w, float lo, float width) {
        return __fmaf_rn(unit_f32(w), width, lo);
    }
};

template <>
struct Coord<double> {
    __device__ __forceinline__ static double map(uint32_t w, double lo, double width) {
        return __fma_rn(unit_f64(w), width, lo);
    }
};

// ---------------------------------------------------------------------------
// Lattice constants of Eq. (Gen2) folded for the residual
//   R = v_next + v (c_adv (v_r - v_l) + (2 c_dif - 1)) - c_dif (v_r + v_l)
// which equals v_next - v + tau (v (v_r - v_l)/(2a) - nu (v_r - 2v + v_l)/a^2)
// with c_adv = nonlinear tau / (2a) and c_dif = nu tau / a^2.
// ---------------------------------------------------------------------------
template <typename Real>
struct LatticeConst {
    Real c_adv;
    Real k1;         // 2 c_dif - 1
    Real neg_c_dif;  // -c_dif
    Real inv_2Dtau;  // 1 / (2 D tau)
    Real half_mass2; // mass2 / 2
};

// Sum of squared residuals over the periodic lattice (d = NX * NT values in
// registers, coordinate j = m * NT + l).
template <int NX, int NT, typename Real>
__device__ __forceinline__ Real residual_sq_sum(const Real (&u)[NX * NT], const LatticeConst<Real> &c) {
    Real acc = Real(0);
#pragma unroll
    for (int m = 0; m < NX; ++m) {
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            const Real here = u[m * NT + l];
            const Real next = u[m * NT + (l + 1) % NT];
            const Real right = u[((m + 1) % NX) * NT + l];
            const Real left = u[((m + NX - 1) % NX) * NT + l];
            const Real t = fma(c.c_adv, right - left, c.k1);
            Real R = fma(here, t, next);
            R = fma(c.neg_c_dif, right + left, R);
            acc = fma(R, R, acc);
        }
    }
    return acc;
}

// Unscaled equal-time products Q_r = sum_{l,m} v_{l,m} v_{l,m+r} = d P_r,
// r = 0..NX/2.  For even NX the r = NX/2 pairs are counted twice.
template <int NX, int NT, typename Real>
__device__ __forceinline__ void products(const Real (&u)[NX * NT], Real (&Q)[NX / 2 + 1]) {
    constexpr int R = NX / 2 + 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        Real s = Real(0);
        const bool half = (2 * r == NX) && r > 0;
#pragma unroll
        for (int m = 0; m < (half ? NX / 2 : NX); ++m) {
#pragma unroll
            for (int l = 0; l < NT; ++l) s = fma(u[m * NT + l], u[((m + r) % NX) * NT + l], s);
        }
        Q[r] = half ? Real(2) * s : s;
    }
}

// ---------------------------------------------------------------------------
// Compensated ("double-float") FP32 arithmetic: a value is an unevaluated sum
// hi + lo of two floats.  Built from the error-free transformations TwoSum
// (Knuth) and TwoProduct (one FMA), as in Ogita, Rump & Oishi, "Accurate sum
// and dot product" (SIAM J. Sci. Comput. 26, 2005).  About 2^-44 relative
// accuracy, in FP32 instructions only.
// ---------------------------------------------------------------------------
struct DF {
    float h, l;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, __fmaf_rn(a, b, -p)};
}

// (a.h + a.l) * (b.h + b.l), dropping the a.l * b.l term
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    DF p = two_prod(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
    DF s = two_sum(a.h, b);
    s.l = __fadd_rn(s.l, a.l);
    return fast_two_sum(s.h, s.l);
}

// Compensated dot product of the FP32 evaluation, Q_r = sum_j u_j u_{j+r}
// (Dot2 of Ogita, Rump & Oishi: every product split exactly by two_prod, the
// running sum by two_sum, the errors summed in plain float), returned as
// hi + lo: |Q_r - (hi + lo)| <= 2^-24 |Q_r| + gamma_d^2 Q_0 with Q_0 >=
// |Q_r| by Cauchy-Schwarz.  For even NX the r = NX/2 pairs count twice.
template <int NX, int NT>
__device__ __forceinline__ DF product_df(const float (&u)[NX * NT], int r) {
    DF s{0.f, 0.f};
    const bool half = (2 * r == NX) && r > 0;
#pragma unroll
    for (int m = 0; m < (half ? NX / 2 : NX); ++m) {
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            const DF p = two_prod(u[m * NT + l], u[((m + r) % NX) * NT + l]);
            const DF t = two_sum(s.h, p.h);
            s.h = t.h;
            s.l = __fadd_rn(s.l, __fadd_rn(p.l, t.l));
        }
    }
    return half ? DF{2.f * s.h, 2.f * s.l} : s;
}

// Weight exp(m - S) of the FP32 evaluation with the shift m kept in double
// and the action S = S.h + S.l in compensated float.  The argument a = m - S
// is formed in double and split exactly into floats a_h + a_l (|a_l| <=
// ulp(a_h)/2), and exp(a) = exp(a_h) (1 + a_l + O(a_l^2)): so the weight
// carries expf's error (at most 2 ulp by CUDA's documented accuracy) and one
// rounding, whatever the size of the argument.
__device__ __forceinline__ float weight_f32(double m, DF S) {
    const double a = (m - static_cast<double>(S.h)) - static_cast<double>(S.l);
    const float ah = __double2float_rn(a);
    const float al = __double2float_rn(a - static_cast<double>(ah));
    const float e = expf(ah);
    return __fmaf_rn(e, al, e);
}

// Moving the FP32 evaluation's shift down past an action S: by k ln 2 with
// k = ceil((m - S) / ln 2), so that every sum scales by exactly 2^-k (first
// order) or 2^-2k (second order) and no rounding enters; the new shift lies in
// (S - ln 2, S].  pow2_neg(k) = 2^-k as a float (0 below the normal range: a
// sum scaled that far is below 2^-126 of the new largest weight).
constexpr double kLn2 = 0.693147180559945309417232121458;
__device__ __forceinline__ int shift_steps(double m, double S) {
    return static_cast<int>(ceil((m - S) * (1.0 / kLn2)));
}
__device__ __forceinline__ float pow2_neg(int k) { return k < 127 ? __int_as_float((127 - k) << 23) : 0.f; }

// The constants of the residual split into hi + lo floats.
struct LatticeConstDF {
    DF c_adv, k1, c_dif, inv_2Dtau, half_mass2;
};

inline DF split_df(double x) {
    const float h = static_cast<float>(x);
    return DF{h, static_cast<float>(x - static_cast<double>(h))};
}

// S of Eq. (Gen2) at float coordinates, in compensated FP32: every residual
// R = v_next + v (c_adv (v_r - v_l) + k1) - c_dif (v_r + v_l), its square and
// the sum over sites carry their rounding errors along.
template <int NX, int NT>
__device__ __forceinline__ DF action_df(const float (&u)[NX * NT], const LatticeConstDF &c) {
    DF acc{0.f, 0.f};
    DF mass{0.f, 0.f};
    const bool with_mass = c.half_mass2.h != 0.f;
#pragma unroll
    for (int m = 0; m < NX; ++m) {
#pragma unroll
        for (int l = 0; l < NT; ++l) {
            const float here = u[m * NT + l];
            const float next = u[m * NT + (l + 1) % NT];
            const float right = u[((m + 1) % NX) * NT + l];
            const float left = u[((m + NX - 1) % NX) * NT + l];
            const DF dx = two_sum(right, -left);                    // exact
            const DF t = df_add(df_mul(c.c_adv, dx), c.k1);         // c_adv dx + k1
            const DF q = df_add_f(df_mul_f(t, here), next);         // v t + v_next
            const DF lr = two_sum(right, left);                     // exact
            const DF R = df_add(q, df_mul(c.c_dif, DF{-lr.h, -lr.l}));
            DF sq = two_prod(R.h, R.h);
            sq.l = __fmaf_rn(2.f * R.h, R.l, sq.l);
            acc = df_add(acc, sq);
            if (with_mass) mass = df_add(mass, two_prod(here, here));
        }
    }
    DF S = df_mul(acc, c.inv_2Dtau);
    if (with_mass) S = df_add(S, df_mul(mass, c.half_mass2));
    return S;
}

// ---------------------------------------------------------------------------
// Shifted sums.  A record (m, s[K]) with K = 2 + 3R stands for the sums of
// w = exp(-(S - m)):   [0] w  [1] w^2  [2+r] w Q_r  [2+R+r] w^2 Q_r
// [2+2R+r] w^2 Q_r^2.  "order" 1 sums scale with exp(-dm), order 2 with
// exp(-2 dm) when the shift moves.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int sum_count(int R) { return 2 + 3 * R; }
__host__ __device__ constexpr bool second_order(int k, int R) { return k == 1 || k >= 2 + R; }

}  // namespace bfi
