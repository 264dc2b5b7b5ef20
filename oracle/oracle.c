/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the Monte Carlo evaluation of the
 * lattice Burgers functional integral (Honkonen & Honkonen, arXiv:1803.07560).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, import or
 * execute this file.  It is used by tests/, by the smoke check and by the
 * timed CPU baseline of the benchmark.  It shares no code with the CUDA path:
 * the Philox generator, the point mapping, the action, the correlation
 * products, the estimator and the merge are all written out here a second
 * time, step by step, in the order the paper states them.
 *
 * What it computes (all FP64, compiled with -ffp-contract=off so that only the
 * explicit fma() calls below fuse):
 *
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 *     easy as 1, 2, 3", SC'11): the counter-based generator that draws the
 *     integration points.  The paper only says "GSL Monte Carlo" (Sec. 3); the
 *     generator is our reading.
 *   - The lattice action of Eq. (Gen2): S = 1/(2 D tau) sum_{l,m} R_{l,m}^2 with
 *     R_{l,m} = v(t_{l+1},x_m) - v(t_l,x_m)
 *               + tau * ( v(t_l,x_m) [v(t_l,x_{m+1}) - v(t_l,x_{m-1})]/(2a)
 *                         - nu [v(t_l,x_{m+1}) - 2 v(t_l,x_m) + v(t_l,x_{m-1})]/a^2 ),
 *     periodic in space and time (Sec. 2, the sentence after Eq. (Gen2)).
 *     Two test knobs: 'nonlinear' multiplies the advection term (1 = Eq. (Gen2),
 *     0 = linear limit) and 'mass2' adds mass2/2 * sum v^2 (0 = Eq. (Gen2)).
 *   - The equal-time two-point products of Eq. (Gen2)'s left-hand side,
 *     averaged over sites: P_r = (1/d) sum_{l,m} v_{l,m} v_{l,(m+r) mod Nx},
 *     r = 0..floor(Nx/2).
 *   - Plain Monte Carlo over each subvolume (Sec. 3: result = V mean(f),
 *     error = V sigma_f / sqrt(n), the convention the Listing 2 output obeys),
 *     with weights exp(-(S - m_s)) shifted by the subvolume's minimum action
 *     m_s so that they neither underflow nor overflow.  Pass 1 finds m_s,
 *     pass 2 regenerates the same points and accumulates, in sample order with
 *     Neumaier-compensated sums.
 *   - The merge of independent subvolumes into Z, C(r) = N(r)/Z and their
 *     stated errors (Sec. 1 and 3: the value in any region is computed
 *     separately from the others and summed; Sec. 4: C(r) is normalised by the
 *     integral with the velocity factors set to 1).
 *
 * Layout conventions (shared by contract with the CUDA path, not by code):
 *   coordinate j = m*Nt + l holds v(t_l, x_m)  (site-major);
 *   sample i of a subvolume with id sid draws Philox words from
 *     counter (q, i mod 2^32, i div 2^32, sid), key (seed, job_id), q = j div 4,
 *     word j mod 4 of that block feeds coordinate j;
 *   FP64 points: u = (w + 0.5) 2^-32,            y = fma(u, hi - lo, lo);
 *   FP32 points: u = ((w >> 9) + 0.5) 2^-23 (float),
 *                y = fmaf(u, (float)(hi - lo), (float)lo), then widened.
 *   A subvolume's record ("slot") has 5 + 3R doubles:
 *     [0] n  [1] m_s  [2] log V_s  [3] sum w  [4] sum w^2
 *     [5 + r] sum w P_r  [5 + R + r] sum w^2 P_r  [5 + 2R + r] sum w^2 P_r^2
 *   with w = exp(-(S - m_s)).
 *   Totals have 4 + 2R doubles:
 *     [0] log Z  [1] relative std error of Z  [2] total samples
 *     [3] subvolumes with samples  [4 + r] C(r)  [4 + R + r] std error of C(r)
 */
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, written from the SC'11 definition.                          */
/* One round: two 32x32->64 products of counter words 0 and 2 with the       */
/* multipliers; the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0).  */
/* The key is bumped by the two Weyl constants between rounds.               */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The d raw 32-bit words of sample i of subvolume 'sid'. */
void oracle_sample_words(uint32_t seed, uint32_t job_id, uint32_t sid, uint64_t i,
                         int d, uint32_t *words)
{
    for (int q = 0; 4 * q < d; ++q) {
        uint32_t ctr[4], key[2], out[4];
        ctr[0] = (uint32_t)q;
        ctr[1] = (uint32_t)(i & 0xFFFFFFFFu);
        ctr[2] = (uint32_t)(i >> 32);
        ctr[3] = sid;
        key[0] = seed;
        key[1] = job_id;
        oracle_philox4x32_10(ctr, key, out);
        for (int t = 0; t < 4 && 4 * q + t < d; ++t) words[4 * q + t] = out[t];
    }
}

/* Map raw words to the coordinates of one sample in the box [lo, hi]. */
void oracle_words_to_point(int d, const uint32_t *words, const double *lo, const double *hi,
                           int fp32_points, double *y)
{
    for (int j = 0; j < d; ++j) {
        if (fp32_points) {
            float u = ((float)(words[j] >> 9) + 0.5f) * 0x1p-23f;
            float width = (float)(hi[j] - lo[j]);
            float base = (float)lo[j];
            y[j] = (double)fmaf(u, width, base);
        } else {
            double u = ((double)words[j] + 0.5) * 0x1p-32;
            y[j] = fma(u, hi[j] - lo[j], lo[j]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* The action of Eq. (Gen2) and the correlation products.                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t nx, nt;
    double nu, D, a, tau;
    double nonlinear, mass2;
} oracle_lattice;

static double v_at(const oracle_lattice *lat, const double *u, int l, int m)
{
    /* periodic in time (index l) and space (index m) */
    int L = lat->nt, M = lat->nx;
    l = ((l % L) + L) % L;
    m = ((m % M) + M) % M;
    return u[m * L + l];
}

double oracle_action(const oracle_lattice *lat, const double *u)
{
    double sum_r2 = 0.0, sum_u2 = 0.0;
    for (int l = 0; l < lat->nt; ++l) {
        for (int m = 0; m < lat->nx; ++m) {
            double here = v_at(lat, u, l, m);
            double next_t = v_at(lat, u, l + 1, m);
            double right = v_at(lat, u, l, m + 1);
            double left = v_at(lat, u, l, m - 1);
            double advection = here * (right - left) / (2.0 * lat->a);
            double diffusion = lat->nu * (right - 2.0 * here + left) / (lat->a * lat->a);
            double residual = next_t - here + (lat->nonlinear * advection - diffusion) * lat->tau;
            sum_r2 += residual * residual;
            sum_u2 += here * here;
        }
    }
    return sum_r2 / (2.0 * lat->D * lat->tau) + 0.5 * lat->mass2 * sum_u2;
}

int oracle_num_r(int nx) { return nx / 2 + 1; }

void oracle_correlations(const oracle_lattice *lat, const double *u, double *P)
{
    int R = oracle_num_r(lat->nx);
    double d = (double)(lat->nx * lat->nt);
    for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int l = 0; l < lat->nt; ++l)
            for (int m = 0; m < lat->nx; ++m)
                s += v_at(lat, u, l, m) * v_at(lat, u, l, m + r);
        P[r] = s / d;
    }
}

/* ------------------------------------------------------------------------- */
/* Compensated (Neumaier) summation.                                          */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------- */
/* Plain Monte Carlo over one subvolume (Sec. 3), shifted weights.            */
/* ------------------------------------------------------------------------- */
int oracle_slot_len(int nx) { return 5 + 3 * oracle_num_r(nx); }
int oracle_totals_len(int nx) { return 4 + 2 * oracle_num_r(nx); }

static void integrate_one(const oracle_lattice *lat, const double *lo, const double *hi,
                          uint64_t n, uint32_t sid, uint32_t seed, uint32_t job_id,
                          int fp32_points, double *slot)
{
    int d = lat->nx * lat->nt;
    int R = oracle_num_r(lat->nx);
    uint32_t *words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)d);
    double *y = (double *)malloc(sizeof(double) * (size_t)d);
    double *P = (double *)malloc(sizeof(double) * (size_t)R);
    nsum *acc = (nsum *)calloc((size_t)(2 + 3 * R), sizeof(nsum));

    double log_vol = 0.0;
    for (int j = 0; j < d; ++j) log_vol += log(hi[j] - lo[j]);

    /* pass 1: the smallest action in the subvolume */
    double m_s = INFINITY;
    for (uint64_t i = 0; i < n; ++i) {
        oracle_sample_words(seed, job_id, sid, i, d, words);
        oracle_words_to_point(d, words, lo, hi, fp32_points, y);
        double S = oracle_action(lat, y);
        if (S < m_s) m_s = S;
    }
    /* pass 2: the same points again, weights exp(-(S - m_s)) */
    for (uint64_t i = 0; i < n; ++i) {
        oracle_sample_words(seed, job_id, sid, i, d, words);
        oracle_words_to_point(d, words, lo, hi, fp32_points, y);
        double S = oracle_action(lat, y);
        oracle_correlations(lat, y, P);
        double w = exp(-(S - m_s));
        nsum_add(&acc[0], w);
        nsum_add(&acc[1], w * w);
        for (int r = 0; r < R; ++r) {
            nsum_add(&acc[2 + r], w * P[r]);
            nsum_add(&acc[2 + R + r], w * w * P[r]);
            nsum_add(&acc[2 + 2 * R + r], w * w * P[r] * P[r]);
        }
    }
    slot[0] = (double)n;
    slot[1] = m_s;
    slot[2] = log_vol;
    for (int k = 0; k < 2 + 3 * R; ++k) slot[3 + k] = nsum_value(&acc[k]);

    free(words); free(y); free(P); free(acc);
}

/* ------------------------------------------------------------------------- */
/* Merge of independent subvolumes into Z, C(r) and stated errors.            */
/*                                                                            */
/* Per subvolume s (n >= 1 samples), with ls = log V_s - log n - m_s:         */
/*   Z_s   = e^{ls} sum w                     N_s(r) = e^{ls} sum w P_r       */
/*   Var Z_s    = e^{2 ls} (n sum w^2     - (sum w)^2)        / (n - 1)        */
/*   Var N_s    = e^{2 ls} (n sum w^2 P^2 - (sum w P)^2)      / (n - 1)        */
/*   Cov(N_s,Z_s) = e^{2 ls} (n sum w^2 P - sum w sum w P)   / (n - 1)        */
/* (the plain-MC error V sigma/sqrt(n) of Sec. 3, with the unbiased sigma).   */
/* Totals: Z = sum Z_s, N(r) = sum N_s(r), C(r) = N(r)/Z and, by the delta    */
/* method for a ratio of sums of independent estimates,                       */
/*   Var C(r) = (1/Z^2) sum_s [Var N_s - 2 C Cov(N_s,Z_s) + C^2 Var Z_s].     */
/* Everything is scaled by e^{-L}, L = the largest ls, so nothing overflows.  */
/* A subvolume with n = 1 has no variance estimate: its errors are +inf.      */
/* ------------------------------------------------------------------------- */
void oracle_merge(int nx, int64_t nsub, const double *slots, double *totals)
{
    int R = oracle_num_r(nx);
    int SL = oracle_slot_len(nx);
    double L = -INFINITY, n_total = 0.0, used = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (q[0] <= 0.0) continue;
        n_total += q[0];
        used += 1.0;
        if (!(q[3] > 0.0)) continue;
        double ls = q[2] - log(q[0]) - q[1];
        if (ls > L) L = ls;
    }
    double *N = (double *)calloc((size_t)R, sizeof(double));
    double Z = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (q[0] <= 0.0 || !(q[3] > 0.0)) continue;
        double f = exp(q[2] - log(q[0]) - q[1] - L);
        Z += f * q[3];
        for (int r = 0; r < R; ++r) N[r] += f * q[5 + r];
    }
    totals[0] = L + log(Z);
    totals[2] = n_total;
    totals[3] = used;
    double varZ = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const double *q = slots + s * SL;
        if (q[0] <= 0.0 || !(q[3] > 0.0)) continue;
        double n = q[0];
        if (n < 2.0) { varZ = INFINITY; continue; }
        double f = exp(q[2] - log(q[0]) - q[1] - L);
        varZ += f * f * (n * q[4] - q[3] * q[3]) / (n - 1.0);
    }
    totals[1] = sqrt(varZ > 0.0 ? varZ : 0.0) / Z;
    for (int r = 0; r < R; ++r) {
        double C = N[r] / Z;
        double var = 0.0;
        for (int64_t s = 0; s < nsub; ++s) {
            const double *q = slots + s * SL;
            if (q[0] <= 0.0 || !(q[3] > 0.0)) continue;
            double n = q[0];
            if (n < 2.0) { var = INFINITY; continue; }
            double f = exp(q[2] - log(q[0]) - q[1] - L);
            double varN = (n * q[5 + 2 * R + r] - q[5 + r] * q[5 + r]) / (n - 1.0);
            double cov = (n * q[5 + R + r] - q[3] * q[5 + r]) / (n - 1.0);
            double vz = (n * q[4] - q[3] * q[3]) / (n - 1.0);
            var += f * f * (varN - 2.0 * C * cov + C * C * vz);
        }
        totals[4 + r] = C;
        totals[4 + R + r] = sqrt(var > 0.0 ? var : 0.0) / Z;
    }
    free(N);
}

/* Whole integration: every subvolume independently (OpenMP over subvolumes
 * only, each subvolume sequential, so the result does not depend on the
 * thread count), then the merge.  sub_id may be NULL (ids 0..nsub-1).
 * Returns 0, or 1 on invalid arguments. */
int oracle_integrate(const oracle_lattice *lat, int64_t nsub, const double *lo, const double *hi,
                     const uint64_t *samples, const uint32_t *sub_id, uint32_t seed,
                     uint32_t job_id, int fp32_points, int nthreads,
                     double *slots, double *totals)
{
    if (lat->nx < 2 || lat->nt < 1 || nsub < 0) return 1;
    int d = lat->nx * lat->nt;
    int SL = oracle_slot_len(lat->nx);
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t s = 0; s < nsub; ++s) {
        uint32_t sid = sub_id ? sub_id[s] : (uint32_t)s;
        integrate_one(lat, lo + s * d, hi + s * d, samples[s], sid, seed, job_id,
                      fp32_points, slots + s * SL);
    }
    if (totals) oracle_merge(lat->nx, nsub, slots, totals);
    return 0;
}

/* Per-sample action and correlation products at given points (for pins). */
void oracle_eval_points(const oracle_lattice *lat, int64_t npts, const double *y,
                        double *S, double *P)
{
    int d = lat->nx * lat->nt;
    int R = oracle_num_r(lat->nx);
    for (int64_t i = 0; i < npts; ++i) {
        S[i] = oracle_action(lat, y + i * d);
        if (P) oracle_correlations(lat, y + i * d, P + i * R);
    }
}

/* Coordinates of samples [first, first + count) of one subvolume. */
void oracle_points(int d, const double *lo, const double *hi, uint32_t sid, uint32_t seed,
                   uint32_t job_id, uint64_t first, int64_t count, int fp32_points, double *y)
{
    uint32_t *words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)d);
    for (int64_t k = 0; k < count; ++k) {
        oracle_sample_words(seed, job_id, sid, first + (uint64_t)k, d, words);
        oracle_words_to_point(d, words, lo, hi, fp32_points, y + k * d);
    }
    free(words);
}

/* ------------------------------------------------------------------------- */
/* The N-sphere integrand of Sec. 3 (Listings 1-2): f = sqrt(max(0, 1-|x|^2)) */
/* on a box, plain MC with the same point generator (FP64 points, sid 0).    */
/* Its integral over [-1,1]^k is half the volume of the unit (k+1)-ball.     */
/* ------------------------------------------------------------------------- */
void oracle_nsphere(int dims, const double *lo, const double *hi, uint64_t n,
                    uint32_t seed, uint32_t job_id, uint32_t sub_id, double *result, double *abs_err,
                    int *split_dim)
{
    uint32_t *words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)dims);
    double *x = (double *)malloc(sizeof(double) * (size_t)dims);
    nsum *below = (nsum *)calloc((size_t)dims, sizeof(nsum));
    double vol = 1.0;
    for (int j = 0; j < dims; ++j) vol *= hi[j] - lo[j];
    nsum sf = {0, 0}, sf2 = {0, 0};
    for (uint64_t i = 0; i < n; ++i) {
        oracle_sample_words(seed, job_id, sub_id, i, dims, words);
        oracle_words_to_point(dims, words, lo, hi, 0, x);
        double r2 = 0.0;
        for (int j = 0; j < dims; ++j) r2 += x[j] * x[j];
        double f = r2 < 1.0 ? sqrt(1.0 - r2) : 0.0;
        nsum_add(&sf, f);
        nsum_add(&sf2, f * f);
        /* how unevenly f falls on the two halves of each coordinate */
        for (int j = 0; j < dims; ++j)
            if (x[j] < 0.5 * (lo[j] + hi[j])) nsum_add(&below[j], f);
    }
    double nn = (double)n;
    double mean = nsum_value(&sf) / nn;
    double var = (nsum_value(&sf2) - nsum_value(&sf) * nsum_value(&sf) / nn) / (nn - 1.0);
    *result = vol * mean;
    *abs_err = vol * sqrt(var / nn);
    /* split suggestion (Sec. 3 prints one; the rule is our reading): the
     * coordinate with the largest |sum below the midpoint - sum above it| */
    if (split_dim) {
        int best = 0;
        double best_gap = -1.0;
        for (int j = 0; j < dims; ++j) {
            double b = nsum_value(&below[j]);
            double gap = fabs(b - (nsum_value(&sf) - b));
            if (gap > best_gap) { best_gap = gap; best = j; }
        }
        *split_dim = best;
    }
    free(words); free(x); free(below);
}
