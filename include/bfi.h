/*
 * bfi.h -- C ABI of the GB300 (sm_103a) library for the Monte Carlo
 * evaluation of the lattice Burgers functional integral of Honkonen &
 * Honkonen, "Modelling turbulence via numerical functional integration using
 * Burgers' equation" (arXiv:1803.07560).
 *
 * The library computes, for one lattice and a list of box-shaped
 * subvolumes of the integration volume, the plain Monte Carlo estimates of
 *
 *   Z    = int prod dv  exp(-S[v])                    (the normaliser, Sec. 4)
 *   N(r) = int prod dv  P_r[v] exp(-S[v])             (numerator of Eq. (Gen2))
 *   C(r) = N(r) / Z                                   (Eq. (Gen2), C = 1/Z)
 *
 * with S the lattice action of Eq. (Gen2):
 *
 *   S = 1/(2 D tau) sum_{l,m} R_{l,m}^2,
 *   R_{l,m} = v_{l+1,m} - v_{l,m}
 *           + tau ( v_{l,m} (v_{l,m+1} - v_{l,m-1}) / (2a)
 *                   - nu (v_{l,m+1} - 2 v_{l,m} + v_{l,m-1}) / a^2 ),
 *
 * periodic in time (l, Nt slices) and space (m, Nx sites) (Sec. 2), and
 * P_r = (1/d) sum_{l,m} v_{l,m} v_{l,m+r} the site-averaged equal-time
 * product at distance r = 0..floor(Nx/2), d = Nx Nt.  Subvolumes are
 * integrated independently and summed (Sec. 1 and 3); each gets plain MC
 * with uniform points (Sec. 3: result = V mean f, error = V sigma / sqrt n).
 *
 * Conventions used by every call below.
 *
 *  - Coordinates: coordinate j = m*Nt + l holds v(t_l, x_m).
 *  - Points: sample i (0-based) of subvolume s draws the Philox4x32-10 block
 *    (counter (j/4, i mod 2^32, i / 2^32, sub_id[s]), key (seed, job_id));
 *    word j%4 of it, w, gives coordinate j:
 *      BFI_FP64:  y = fma((w + 0.5) 2^-32, hi - lo, lo)               (double)
 *      BFI_FP32:  y = fmaf(((w >> 9) + 0.5) 2^-23, (float)(hi - lo), (float)lo)
 *  - Weights: w_i = exp(-(S_i - m_s)) with a per-subvolume shift m_s close to
 *    the smallest action, so nothing underflows or overflows whatever the
 *    lattice size.
 *  - Subvolume record ("slot"), bfi_slot_len(nx) = 5 + 3R doubles, R = nx/2+1:
 *      [0] n_s  [1] m_s  [2] log V_s  [3] sum w  [4] sum w^2
 *      [5 + r] sum w P_r   [5 + R + r] sum w^2 P_r   [5 + 2R + r] sum w^2 P_r^2
 *    so that Z_s = exp(log V_s - log n_s - m_s) * sum w.
 *  - Totals, bfi_totals_len(nx) = 4 + 2R doubles:
 *      [0] log Z  [1] relative standard error of Z  [2] samples  [3] subvolumes
 *      with samples  [4 + r] C(r)  [4 + R + r] standard error of C(r)
 *    The errors are the plain-MC standard errors, combined over independent
 *    subvolumes; the error of C(r) is the first-order (delta-method) error of
 *    a ratio of sums.  A subvolume with exactly one sample makes the errors
 *    +inf; subvolumes with no samples are skipped.
 *  - Precision: BFI_FP64 evaluates in double every sample that can carry
 *    weight (the FP32 screen under Negligible weights decides which):
 *    its FP64 point, action, products and weight, accumulated in double.
 *    BFI_FP32 evaluates the points, the action, the products and the weights
 *    in float, accumulates per thread in Kahan-compensated float, and keeps
 *    the log-weight shift and the merges in double: the action in
 *    compensated float (pairs of floats carrying the rounding error), the
 *    weight from an exactly split argument, the products as compensated dot
 *    products.  In both the shift m_s starts at the smallest FP32 action
 *    among the subvolume's first n_s/32 samples (256 to 4096; that action is
 *    rounded by up to ~4 d 2^-24 S) and moves down only when a sample beats
 *    it by more than 16: in BFI_FP64 to that sample's action, in BFI_FP32 by
 *    whole multiples of ln 2 to within ln 2 below it, so that the float sums
 *    rescale exactly (the records do not depend on its exact value beyond
 *    rounding).  The stated arithmetic error of each result, against the
 *    same estimator evaluated exactly on the same points, is what
 *    bfi_error_bound returns: in BFI_FP32 below 1e-6 relative on Z and on
 *    C(r) (relative to C(0)) for the 4x2 and 10x2 lattices, larger for big
 *    lattices at large actions.
 *  - Negligible weights: a sample whose action exceeds the subvolume's
 *    smallest action by more than W = c + ln(n_max) (n_max the largest
 *    budget of the plan; c = 34 in BFI_FP64, 20 in BFI_FP32) has weight below
 *    e^-W of the largest, and all such samples together move any sum by less
 *    than e^-c relative.  They are counted in n_s but left out of the sums.
 *    Both modes decide this from an FP32 action of a float point with a
 *    margin of 1 + 0.1% of S, far above its difference from the action the
 *    evaluation computes.
 *    The reference action starts at the smallest FP32 action among each
 *    subvolume's first n_s/32 samples (256 to 4096) and follows the smallest evaluated
 *    action, shared at fixed points of the sample loop, so the outcome is
 *    reproducible.
 *  - Errors: every call returns a bfi_status; bfi_last_error() gives a
 *    message for the calling thread.  No call aborts the process.
 *
 * Entry points, in the order below: sizes and errors; plans (the
 * device-resident path: create, execute on a stream, grid, timing, stats,
 * samplers); the allocation-free one-call path; batches of jobs in one CUDA
 * graph and the grid autotuner; the serving loop (submit, poll, wait,
 * cancel); contexts and the host-buffer one-call path; the N-sphere test
 * integrand and adaptive subdivision of Sec. 3; the host merge; single steps
 * (points, action and products) for step-by-step checks.
 *  - Pointers: "host" pointers are ordinary CPU memory, "device" pointers
 *    are CUDA device memory of the plan's or context's device.  The caller
 *    owns every array it passes and may free it once the call returns (for
 *    asynchronous calls: once the stream has passed the call).
 */
#ifndef BFI_H
#define BFI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFI_OK = 0,
    BFI_E_INVALID = 1,      /* an argument is out of range or inconsistent */
    BFI_E_NOMEM = 2,        /* a host or device allocation failed */
    BFI_E_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
    BFI_E_TIMEOUT = 4,      /* a bounded wait ran out */
    BFI_E_CANCELLED = 5,    /* the job was cancelled */
    BFI_E_BUSY = 6,         /* the resource is in use */
    BFI_E_UNSUPPORTED = 7   /* lattice shape not compiled into this library */
} bfi_status;

typedef enum {
    BFI_FP64 = 0,
    BFI_FP32 = 1,
    BFI_FP32_COMPENSATED = 2  /* bfi_eval only: the compensated FP32 action (see Precision) */
} bfi_precision;

/* Lattice and parameters of Eq. (Gen2) (Sec. 2; the paper uses
 * nu = D = a = tau = 1).  nx = M spatial sites (>= 2), nt = L time slices
 * (>= 1), d = nx * nt <= 512.  D is the variance of the random force.
 * Two test knobs that are not in the paper: 'nonlinear' multiplies the
 * advection term (1 = Eq. (Gen2), 0 = linear limit) and 'mass2' (>= 0) adds
 * mass2/2 * sum v^2 to S (0 = Eq. (Gen2)). */
typedef struct {
    int32_t nx;
    int32_t nt;
    double nu;
    double D;
    double a;
    double tau;
    double nonlinear;
    double mass2;
} bfi_lattice;

/* Sizes of the records above. */
int32_t bfi_num_r(int32_t nx);
int32_t bfi_slot_len(int32_t nx);
int32_t bfi_totals_len(int32_t nx);

/* Message describing the last failed call on this thread ("" if none). */
const char *bfi_last_error(void);

/* ------------------------------------------------------------------------ */
/* Plans: the device-resident hot path.                                      */
/* ------------------------------------------------------------------------ */

/* A plan fixes the lattice, the precision, the number of subvolumes and
 * their sample budgets (Sec. 3: "number of samples and the extent of the
 * integration volume"), and owns the device scratch the integration needs
 * (chunk table, per-chunk partial records).  Creating it allocates device
 * memory on 'device' and may take milliseconds; executing it allocates
 * nothing.  samples: host [nsub], per-subvolume budgets (0 allowed).
 * Errors: BFI_E_INVALID (bad lattice, nsub < 1, d > 512, a budget >= 2^48),
 * BFI_E_UNSUPPORTED, BFI_E_NOMEM, BFI_E_CUDA. */
typedef struct bfi_plan bfi_plan;

bfi_status bfi_plan_create(bfi_plan **out, const bfi_lattice *lattice, int64_t nsub,
                           const uint64_t *samples, bfi_precision precision, int device);
bfi_status bfi_plan_destroy(bfi_plan *plan);

typedef struct {
    int64_t nsub;
    int64_t chunks;            /* work units of one execution */
    int64_t chunk_samples;     /* samples per chunk (the last chunk of a subvolume is ragged) */
    int64_t total_samples;
    int32_t grid;              /* CTAs of the integrand kernel */
    int32_t block;             /* threads per CTA */
    int32_t kernel;            /* 0 = thread-per-sample (compiled shape), 1 = warp-per-sample */
    int32_t slot_len;
    int32_t totals_len;
    size_t scratch_bytes;      /* device scratch owned by the plan */
    int32_t ctas_per_sm_max;   /* occupancy limit of the integrand kernel */
    int32_t ctas_per_sm;       /* CTAs per SM the grid uses now */
    int64_t tail_subvolume;    /* subvolumes from this one on (nsub: none) are cut into ... */
    int64_t tail_chunk_samples;  /* ... chunks of this many samples (see bfi_chunking_of) */
} bfi_plan_info;

bfi_status bfi_plan_get_info(const bfi_plan *plan, bfi_plan_info *info);

/* How a job's budgets are cut into chunks, the work units of the integrand
 * kernels (host arithmetic only; no device is touched).  bfi_plan_create,
 * bfi_integrate_static_scratch and the server all cut a job this way, and
 * the cut depends on the budgets alone, so a job's rounding is the same on
 * any device and beside any other job.
 *   chunk_samples = 256 x rows, rows a power of two: at least 2048 chunks and
 *     at most 512 rows, then doubling up to 2048 rows while the job keeps at
 *     least 4096 chunks;
 *   the longest suffix of subvolumes holding at most 1/8 of the samples and
 *     at most 512 x chunk_samples (tail_subvolume .. nsub - 1) is cut into
 *     chunks of tail_chunk_samples = max(chunk_samples / 4, 256 x 256) when
 *     chunk_samples exceeds 256 x 256 (else tail_subvolume = nsub);
 *   subvolume s gives ceil(n_s / its chunk size) chunks, the last ragged;
 *     chunks are numbered subvolume by subvolume, and the kernels hand them
 *     out in that order, so the short ones run last.
 *   nsub, samples   as for bfi_plan_create
 *   out             chunk_samples, tail_subvolume, tail_chunk_samples, chunks
 * Errors: BFI_E_INVALID (nsub < 1, NULL pointer, a budget >= 2^48, total
 * budget >= 2^62). */
typedef struct {
    int64_t chunk_samples;
    int64_t tail_subvolume;
    int64_t tail_chunk_samples;
    int64_t chunks;
} bfi_chunking;

bfi_status bfi_chunking_of(int64_t nsub, const uint64_t *samples, bfi_chunking *out);

/* Run the whole hot path on 'stream' (a cudaStream_t; NULL = legacy default
 * stream): points, action, weights, products, per-subvolume reduction and
 * the FP64 merge.  Asynchronous: returns after enqueueing.
 *   lo, hi  device [nsub * d]  subvolume bounds (row s, coordinate j); lo < hi
 *   sub_id  device [nsub] or NULL (then sub_id[s] = s): Philox counter word 3
 *   seed, job_id               Philox key
 *   slots   device [nsub * bfi_slot_len(nx)]   out
 *   totals  device [bfi_totals_len(nx)]        out
 * Bounds are not validated on the device; lo >= hi gives undefined numbers
 * (never an out-of-range access).  One plan holds one execution's scratch
 * (chunk records, counters, the chunk hand-out counter): executions of the
 * same plan must not overlap on the GPU (order them on one stream); use one
 * plan per concurrent job.  Errors: BFI_E_INVALID (NULL pointers),
 * BFI_E_CUDA (launch failure). */
bfi_status bfi_plan_execute(bfi_plan *plan, const double *lo, const double *hi,
                            const uint32_t *sub_id, uint32_t seed, uint32_t job_id,
                            double *slots, double *totals, void *stream);

/* Persistent grid of the plan's integrand kernel: ctas_per_sm CTAs on each SM
 * (1 .. the occupancy limit; 0 restores the default, the occupancy limit).
 * The grid never changes the results (each chunk's record depends on the
 * chunk only), only the speed.  Errors: BFI_E_INVALID. */
bfi_status bfi_plan_set_grid(bfi_plan *plan, int32_t ctas_per_sm);

/* Samplers: how the unit point u (from Philox, see Conventions) becomes the
 * field v.  The box sampler (the default) takes v uniform in each box.  The
 * other two run in FP64 only (the FP32 screen's error bound does not hold
 * once a map stretches the coordinates, so every sample is evaluated in
 * FP64), on the warp-per-sample kernel:
 *
 *   BFI_SAMPLE_TRANSFORM  the infinite range mapped onto (-1, 1) (Sec. 4; the
 *       paper does not state its transform, this one is ours):
 *       v_j = y_j / (1 - y_j^2) with y uniform in the box, which must lie in
 *       [-1, 1]^d (outside it the numbers are undefined, never an
 *       out-of-range access); the Jacobian prod (1 + y^2)/(1 - y^2)^2 is in
 *       the weight, so a box of [-1, 1]^d integrates over all of R^d.
 *   BFI_SAMPLE_GAUSSIAN   importance sampling (the better-concentrated
 *       integrand Sec. 5 calls for): z standard normal from the unit point u
 *       in Box-Muller pairs, z_{2p} = r cos(2 pi u_{2p+1}), z_{2p+1} =
 *       r sin(2 pi u_{2p+1}), r = sqrt(-2 ln u_{2p}) (for odd d, u_d is the
 *       next Philox word), v = mean + F z, so
 *       v ~ N(mean, F F^T) with density q; the weight is exp(-S(v)) / q(v)
 *       for v in the box [lo, hi) and 0 outside, so each box's Z_s is still
 *       the integral over that box.  d <= 64.  The record's log V_s holds
 *       (d/2) ln(2 pi) + ln |det F| instead of the box volume.
 *
 * Z_s, C(r) and the errors keep their meaning (estimates over the boxes);
 * with GAUSSIAN, a box that no sample hits gives Z_s = 0 (m_s = +inf).
 * mean (NULL = 0) and factor are host arrays, copied by the call. */
typedef enum {
    BFI_SAMPLE_BOX = 0,
    BFI_SAMPLE_TRANSFORM = 1,
    BFI_SAMPLE_GAUSSIAN = 2
} bfi_sample_kind;

typedef struct {
    int32_t kind;          /* bfi_sample_kind */
    const double *mean;    /* GAUSSIAN: host [d] or NULL */
    const double *factor;  /* GAUSSIAN: host [d * d], row-major, non-singular */
} bfi_sampler;

/* Sets the plan's sampler for its next executions (re-sizes the grid for
 * the sampler's kernel).  Errors: BFI_E_INVALID (unknown kind, missing,
 * non-finite or singular factor), BFI_E_UNSUPPORTED (FP32 plan, d > 64 for
 * GAUSSIAN), BFI_E_NOMEM, BFI_E_CUDA. */
bfi_status bfi_plan_set_sampler(bfi_plan *plan, const bfi_sampler *sampler);

/* A proposal for the Gaussian sampler: the factor F (host [d * d],
 * row-major, upper triangular) with F F^T = (A + I / sigma0^2)^-1, where
 * v^T A v / 2 is the action of Eq. (Gen2) without the advection term (the
 * linear limit, mass2 included).  The linear limit has zero modes (the
 * constant field among them) unless mass2 > 0; zero_mode_sigma = sigma0 > 0
 * gives them a finite spread (INFINITY: no regulator).
 * Errors: BFI_E_INVALID (a zero mode left unregulated), BFI_E_UNSUPPORTED
 * (d > 64). */
bfi_status bfi_gaussian_proposal(const bfi_lattice *lattice, double zero_mode_sigma, double *factor);

/* Samples fully evaluated (point, action, products, weight) by the last
 * execution, and the plan's negligible-weight window (see "Negligible
 * weights").  Waits for the device.  Either pointer may be NULL.
 * Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_plan_get_stats(bfi_plan *plan, uint64_t *evaluated, float *skip_window);
/* The two-stage screen of the box sampler's thread-per-sample kernels
 * (compiled shapes with at least 3 Philox blocks per sample whose first ~60%
 * cover at least 35% of the sites: 8x2, 10x2, 16x2, 32x2, 8x4, 10x4, 16x4).
 * Stage 1 draws the first ~60% of a sample's Philox blocks and sums the
 * squared residuals of the sites whose neighbours they cover: a partial
 * action P <= S of Eq. (Gen2).  A sample with P above the negligible-weight
 * threshold (with the screen's margin) cannot carry weight and is dropped.
 * Stage 2 screens the rest with the full FP32 action (for Nt = 2 and
 * mass2 = 0: P plus the residuals stage 1 left out).  Chunks of fewer than
 * 256 samples per thread (jobs below about 2^27 samples) skip stage 1.
 * *two_stage is 1 when the last execution ran stage 1 on at least one chunk,
 * and *screened is then the number of samples the full screen or stage 2
 * examined; otherwise *screened is the plan's total sample count (every
 * sample fully screened or evaluated).  Waits for the device.  Either
 * pointer may be NULL.  Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_plan_get_screen_stats(bfi_plan *plan, uint64_t *screened, int32_t *two_stage);

/* The work the last execution did, sample by sample, for accounting (the
 * algorithmic operations of each part are fixed per sample, so these counts
 * give the work of the launch):
 *   samples      the plan's budget: every sample's Philox words are drawn
 *   stage1       samples of chunks that ran stage 1 of the two-stage screen
 *   survivors    of those, the samples stage 1 let through to stage 2
 *   full_screen  samples screened in one stage with the full FP32 action
 *                (samples = stage1 + full_screen for the box sampler)
 *   evaluated    samples fully evaluated (point, action, products, weight;
 *                for the TRANSFORM and GAUSSIAN samplers, which have no
 *                screen, every sample whose weight was computed)
 *   two_stage_shape  1 when the shape's kernels have the split compiled in
 *   rest_screen      1 when stage 2 adds the rest of the action to P (Nt = 2,
 *                    mass2 = 0), 0 when it screens survivors in full
 * Waits for the device.  Errors: BFI_E_INVALID, BFI_E_CUDA. */
typedef struct {
    uint64_t samples, stage1, survivors, full_screen, evaluated;
    int32_t two_stage_shape, rest_screen;
} bfi_work;

bfi_status bfi_plan_get_work(bfi_plan *plan, bfi_work *work);

/* Per-stage timing of bfi_plan_execute with CUDA events recorded on the
 * execution stream.  After bfi_plan_set_timing(plan, 1), each execution
 * records events around its integrand kernel and around its merge kernels;
 * bfi_plan_get_timing waits for the last execution's events and writes
 * ms[0] = integrand kernel, ms[1] = merges (milliseconds).  Off by default.
 * Errors: BFI_E_INVALID (NULL, or no timed execution yet), BFI_E_CUDA. */
bfi_status bfi_plan_set_timing(bfi_plan *plan, int enable);
bfi_status bfi_plan_get_timing(bfi_plan *plan, float *ms);

/* The whole integration without allocating anything, for callers that
 * cannot call cudaMalloc: for example a plugin inside a host application
 * whose memory manager owns the device heap, or a latency-critical loop where
 * an allocation and the synchronisation it may bring are not allowed after
 * start-up.  The paper has no counterpart; this is a deployment variant of
 * bfi_plan_create + bfi_plan_execute + bfi_plan_destroy with the same kernels,
 * chunking and results.
 *   samples          host [nsub]; the budgets reach the device by a
 *                    cudaMemcpyAsync from this array on 'stream': keep it
 *                    unchanged until 'stream' has passed the call (pageable
 *                    memory is copied before the call returns)
 *   lo, hi, sub_id, seed, job_id, slots, totals   as for bfi_plan_execute
 *   stream           cudaStream_t of the current device
 * The scratch is one 16 MiB device array that every device that loads the
 * library holds until the process exits; a job whose chunk records, chunk
 * table, hints and merge factors need more is rejected with BFI_E_INVALID and a message
 * giving both sizes.  The first call on a device looks up the array's device
 * address (once per device, kept for the process); make that first call
 * before any stream capture, and do not use the entry point across a
 * cudaDeviceReset of the device.
 * Every call uses the same array and leaves its contents behind; each call
 * clears what has to start at zero.  Calls whose work overlaps on the GPU
 * (other streams, other threads) race on the array: serialise them.
 * Asynchronous like bfi_plan_execute.  Errors: BFI_E_INVALID,
 * BFI_E_UNSUPPORTED, BFI_E_CUDA. */
bfi_status bfi_integrate_static_scratch(const bfi_lattice *lattice, int64_t nsub, const uint64_t *samples,
                                        const double *lo, const double *hi, const uint32_t *sub_id,
                                        uint32_t seed, uint32_t job_id, bfi_precision precision,
                                        double *slots, double *totals, void *stream);

/* ------------------------------------------------------------------------ */
/* Batches: many uneven jobs in one CUDA graph.                              */
/* ------------------------------------------------------------------------ */

/* One job of a batch (Sec. 3: a lattice, the extents of its subvolumes and
 * their sample budgets).  Device arrays stay owned by the caller and must
 * outlive the batch; 'samples' is read during bfi_batch_create only. */
typedef struct {
    bfi_lattice lattice;
    int64_t nsub;
    const uint64_t *samples;   /* host [nsub] */
    const double *lo, *hi;     /* device [nsub * d] */
    const uint32_t *sub_id;    /* device [nsub] or NULL */
    uint32_t seed, job_id;
    double *slots;             /* device [nsub * slot_len] out */
    double *totals;            /* device [totals_len] out */
} bfi_job;

typedef struct bfi_batch bfi_batch;

/* Plans every job (allocating its scratch) and captures all of their kernels
 * into one CUDA graph whose branches run on 'nstreams' forked streams, so that
 * small jobs overlap on the device.  With autotune != 0 the persistent grid of
 * each lattice shape is first chosen by timing (bfi_autotune_grid, cached per
 * process).  Results are those of bfi_plan_execute on each job alone.
 * Errors: as bfi_plan_create, BFI_E_CUDA (capture). */
bfi_status bfi_batch_create(bfi_batch **out, const bfi_job *jobs, int32_t njobs, bfi_precision precision,
                            int device, int32_t nstreams, int32_t autotune);
/* Replays the graph on 'stream' (asynchronous). */
bfi_status bfi_batch_launch(bfi_batch *batch, void *stream);
/* The work job 'job' (0-based, in the order given to bfi_batch_create) did in
 * the last replay, as bfi_plan_get_work counts it.  Waits for the device.
 * Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_batch_get_work(bfi_batch *batch, int32_t job, bfi_work *work);
bfi_status bfi_batch_destroy(bfi_batch *batch);

/* Autotuner of the persistent grid: times the integrand of a synthetic job of
 * this lattice shape ([-5,5]^d, 64 subvolumes) at every CTAs-per-SM value
 * from the occupancy limit down and returns the occupancy limit unless a
 * smaller grid is at least 2% faster (median of 5 runs); the choice is cached
 * per (shape, precision, device) for the process.  Errors: as
 * bfi_plan_create. */
bfi_status bfi_autotune_grid(const bfi_lattice *lattice, bfi_precision precision, int device,
                             int32_t *ctas_per_sm);

/* ------------------------------------------------------------------------ */
/* Serving: jobs admitted as they arrive, with adaptive splitting.           */
/* ------------------------------------------------------------------------ */

/* A server runs submitted jobs concurrently on one device: a scheduler thread
 * admits the next pass of a job whenever one of 'slots' streams is free and
 * the job's device memory fits in what remains of 'memory_budget'; passes of
 * different jobs overlap on the GPU.  After a pass, every subvolume whose
 * relative variance Var(Z_s)/Z_s^2 exceeds 'split_rel_var' is bisected along
 * its widest side and both halves are evaluated again with the parent's
 * budget (Sec. 3: subdivision of non-converged subvolumes; the paper's
 * re-evaluation doubles the samples of a region), for at most
 * 'max_split_rounds' rounds and at most 16 times the initial subvolume count;
 * the result merges the final (leaf) subvolumes.  Children draw Philox
 * streams with new sub_ids, numbered on from the job's largest, in subvolume
 * order, so a job's result does not depend on what else runs.  No call waits
 * without a bound. */
typedef struct {
    int32_t device;
    int32_t slots;              /* jobs on the GPU at once (one stream each), >= 1 */
    uint64_t memory_budget;     /* device bytes the server may hold for admitted jobs */
    bfi_precision precision;    /* BFI_FP64 or BFI_FP32 */
    double split_rel_var;       /* <= 0: never split */
    int32_t max_split_rounds;
} bfi_server_config;

typedef struct bfi_server bfi_server;
typedef struct bfi_request bfi_request;

typedef struct {
    int32_t state;              /* 0 queued, 1 running, 2 done, 3 cancelled, 4 failed */
    bfi_status status;          /* of a failed job */
    int64_t nsub_final;         /* leaf subvolumes of the result */
    int32_t passes;             /* evaluation passes run */
    uint64_t samples;           /* samples over all passes */
    double queued_ms;           /* submit -> first pass admitted */
    double latency_ms;          /* submit -> result ready */
} bfi_request_info;

typedef struct {
    uint64_t submitted, completed, failed, cancelled;
    uint64_t samples;           /* over completed passes */
    uint64_t bytes_in_use, bytes_peak;
    int32_t running, queued;
} bfi_server_stats;

/* Errors: BFI_E_INVALID, BFI_E_CUDA (no such device, stream or pool creation). */
bfi_status bfi_server_create(bfi_server **out, const bfi_server_config *config);
/* Stops admitting passes, cancels queued jobs and waits at most timeout_ms
 * (< 0: no limit) for the running passes to end and the scheduler to stop.
 * Passes wait on nothing but their own kernels, so they end; the limit is
 * for callers that must not block.  BFI_OK when stopped, BFI_E_TIMEOUT if
 * passes were still running (call it again, or destroy). */
bfi_status bfi_server_shutdown(bfi_server *server, int64_t timeout_ms);
/* bfi_server_shutdown without a limit, then frees the server (its streams
 * synchronised first).  Release every request handle of the server before
 * destroying it. */
bfi_status bfi_server_destroy(bfi_server *server);

/* Failure handling.  A pass that fails after admission fails its job alone,
 * with a status and a message, and its memory returns to the budget:
 *   - its device allocation from the pool fails: BFI_E_NOMEM;
 *   - a launch or copy fails: BFI_E_CUDA (what was enqueued is drained);
 *   - the stream reports an error when the pass completes, or while it is in
 *     flight (polled by the scheduler): BFI_E_CUDA, its records are not read.
 * If the scheduler thread itself stops on an error (a failed host
 * allocation), every queued and running job fails with BFI_E_NOMEM, waits
 * return, and bfi_submit answers BFI_E_BUSY.  bfi_server_inject_fault makes
 * one of these happen on the host, for tests of this path: the nth pass
 * (0-based, counting from the call) to reach 'point' fails there as if the
 * CUDA call had returned an error (no device work fails).  One fault at a
 * time; BFI_FAULT_NONE clears it.  Errors: BFI_E_INVALID. */
typedef enum {
    BFI_FAULT_NONE = 0,
    BFI_FAULT_POOL_ALLOC = 1,   /* the pass's device allocation */
    BFI_FAULT_LAUNCH = 2,       /* a launch of the pass (its merges) */
    BFI_FAULT_COMPLETION = 3,   /* the stream status read when the pass completes */
    BFI_FAULT_SCHEDULER = 4     /* the scheduler thread, after a pass completes */
} bfi_fault_point;

bfi_status bfi_server_inject_fault(bfi_server *server, int32_t point, int64_t nth);
bfi_status bfi_server_get_stats(bfi_server *server, bfi_server_stats *stats);

/* Queues a job: the integration request of Sec. 3 (the lattice of Eq. (Gen2)
 * with the parameters of Sec. 2, the extents of its subvolumes and their
 * sample budgets), to be subdivided further where it has not converged, as
 * the paper's wrapper does.  Host arrays (lo, hi [nsub * d], samples [nsub])
 * are copied before the call returns.  *out is the caller's handle (release it with
 * bfi_request_release).  Errors: BFI_E_INVALID, BFI_E_UNSUPPORTED, BFI_E_BUSY
 * (server stopping). */
bfi_status bfi_submit(bfi_server *server, const bfi_lattice *lattice, int64_t nsub, const double *lo,
                      const double *hi, const uint64_t *samples, uint32_t seed, uint32_t job_id,
                      bfi_request **out);
/* *done = 1 once the request is done, cancelled or failed. */
bfi_status bfi_poll(bfi_request *request, int32_t *done);
/* Waits at most timeout_ms (< 0: no limit) for the request to end.  Returns
 * BFI_OK when done, BFI_E_TIMEOUT, BFI_E_CANCELLED, or the failure status. */
bfi_status bfi_wait(bfi_request *request, int64_t timeout_ms);
/* Cancels a queued or running job (a running pass finishes; its results are dropped). */
bfi_status bfi_cancel(bfi_request *request);
bfi_status bfi_request_get_info(bfi_request *request, bfi_request_info *info);
/* Result of a done request: totals [totals_len]; optionally the leaf
 * subvolumes: slots [nsub_final * slot_len], lo and hi [nsub_final * d],
 * sub_id [nsub_final] (any of them NULL to skip).  Errors: BFI_E_BUSY (not
 * done), BFI_E_CANCELLED, the failure status. */
bfi_status bfi_request_get_result(bfi_request *request, double *totals, double *slots, double *lo, double *hi,
                                  uint32_t *sub_id);
/* The counted work (as bfi_plan_get_work counts it) of every pass of the
 * request that has completed so far, split parents included.
 * Errors: BFI_E_INVALID. */
bfi_status bfi_request_get_work(bfi_request *request, bfi_work *work);
/* Drops the caller's handle (a job still queued or running is cancelled). */
bfi_status bfi_request_release(bfi_request *request);

/* ------------------------------------------------------------------------ */
/* One-call integration with host buffers (the end-to-end path).            */
/* ------------------------------------------------------------------------ */

/* A context binds a device and a CUDA stream it creates, and caches the plan
 * and device buffers of the last job shape it ran: it stands for the paper's
 * integrand program (Sec. 3), which is started once and then answers one
 * integration request after another.  A context is used by one thread at a
 * time; a concurrent call returns BFI_E_BUSY.
 * Errors: BFI_E_INVALID, BFI_E_NOMEM, BFI_E_CUDA. */
typedef struct bfi_ctx bfi_ctx;

bfi_status bfi_ctx_create(bfi_ctx **out, int device);
bfi_status bfi_ctx_destroy(bfi_ctx *ctx);

/* The sampler of the context's next integrations (see bfi_plan_set_sampler);
 * d is the dimension the Gaussian factor is for (ignored otherwise).
 * Errors: BFI_E_INVALID, BFI_E_BUSY; the plan-level checks surface from
 * bfi_integrate. */
bfi_status bfi_ctx_set_sampler(bfi_ctx *ctx, const bfi_sampler *sampler, int32_t d);

/* Integrate one job with host inputs and outputs, the request of Sec. 3 (a
 * number of samples and the extent of each integration volume in, the
 * result and its error out), for the lattice of Eq. (Gen2) with the
 * parameters of Sec. 2, over the subvolumes whose results add up to the
 * integral over their union (Sec. 1 and 3): copies the bounds in, runs the
 * plan (re-planned only when the lattice, precision or budgets change),
 * copies the results out and waits for them.
 *   lo, hi   host [nsub * d]     samples host [nsub]     sub_id host [nsub] or NULL
 *   slots    host [nsub * slot_len] or NULL (then not copied back)
 *   totals   host [totals_len]
 * Page-locked host buffers make the copies asynchronous with respect to other
 * host work; pageable ones work too.
 * Errors: as bfi_plan_create and bfi_plan_execute, BFI_E_BUSY. */
bfi_status bfi_integrate(bfi_ctx *ctx, const bfi_lattice *lattice, int64_t nsub, const double *lo,
                         const double *hi, const uint64_t *samples, const uint32_t *sub_id,
                         uint32_t seed, uint32_t job_id, bfi_precision precision,
                         double *slots, double *totals);

/* ------------------------------------------------------------------------ */
/* The N-sphere test integrand of Sec. 3 (Listings 1 and 2).                 */
/* ------------------------------------------------------------------------ */

/* Plain Monte Carlo of f(x) = sqrt(max(0, 1 - |x|^2)) over the box
 * prod [lo_j, hi_j] (host arrays, 1 <= dims <= 32), n >= 2 samples with the
 * lattice integrand's points (Philox counter (j/4, i mod 2^32, i / 2^32,
 * sub_id), key (seed, job_id), FP64 points); over [-1,1]^k its integral is
 * half the volume of the unit (k+1)-ball.  Outputs the line of the paper's
 * integrand protocol: result = V mean f, abs_err = V sigma / sqrt(n) (unbiased
 * sigma) and, if split_dim is not NULL, the coordinate j across which f is
 * least even, the largest |sum_{x_j < mid} f - sum_{x_j >= mid} f| (the paper
 * prints a suggestion without stating a rule; this is ours).  Synchronous on
 * 'device'.  Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_nsphere(int32_t dims, const double *lo, const double *hi, uint64_t n, uint32_t seed,
                       uint32_t job_id, uint32_t sub_id, double *result, double *abs_err, int32_t *split_dim,
                       int device);

/* ------------------------------------------------------------------------ */
/* Adaptive subdivision with the convergence test of Sec. 3.                  */
/* ------------------------------------------------------------------------ */

/* Sec. 3: the volume is subdivided until each subvolume has converged.  A
 * subvolume is evaluated twice, with n samples and with factor * n, and has
 * converged when at least one of these holds for the two results r1, r2:
 *   (1) |r1 - r2| <= rel_tol * min(|r1|, |r2|)   (within a factor 1 + rel_tol;
 *       Sec. 4 quotes this threshold as the ratio 1.025 .. 1.085)
 *   (2) |r1 - r2| <= abs_tol
 *   (3) max(|r1|, |r2|) <= small
 * (a criterion whose threshold is <= 0 is off).  A converged subvolume keeps
 * its second evaluation; any other is halved along its split dimension and
 * both halves are evaluated in the next round with n and factor * n samples.
 * All subvolumes of a round go to the GPU in one launch.
 *
 * The tree is numbered like a heap: the whole volume is node 1, the halves of
 * node h are 2h (lower) and 2h + 1 (upper); node h's evaluations draw points
 * with sub_id 2h (n samples) and 2h + 1 (factor * n samples), so every result
 * is reproducible from (seed, job_id) alone.  A subvolume at depth max_depth
 * (the whole volume has depth 0; max_depth <= 30) is kept unconverged, and a
 * round that would evaluate more than max_leaves subvolumes halves them in
 * tree order while there is room and keeps the rest unconverged. */
typedef struct {
    double factor;       /* second evaluation: ceil(factor * n) samples, factor >= 1 (the paper doubles) */
    double rel_tol;      /* criterion (1) */
    double abs_tol;      /* criterion (2) */
    double small;        /* criterion (3) */
    int32_t max_depth;   /* 0..30 */
    int64_t max_leaves;  /* >= 1 */
} bfi_convergence;

typedef struct {
    int64_t rounds;            /* rounds of evaluation */
    int64_t evaluated;         /* subvolumes evaluated (each twice) */
    int64_t converged;         /* kept because a criterion held */
    int64_t kept_depth;        /* kept unconverged at max_depth */
    int64_t kept_budget;       /* kept unconverged for lack of room in max_leaves */
    int64_t leaves;            /* subvolumes in the result = converged + kept_depth + kept_budget */
    uint64_t samples;          /* samples drawn in all evaluations */
} bfi_adaptive_stats;

/* The N-sphere integrand over prod [lo_j, hi_j] (host arrays, dims <= 32):
 * result = sum of the kept second evaluations, abs_err = the root of the sum
 * of their squared errors.  The split dimension is the N-sphere
 * integrand's suggestion.  Synchronous on 'device'; stats may be NULL.
 * Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_adaptive_nsphere(int32_t dims, const double *lo, const double *hi, uint64_t n, uint32_t seed,
                                uint32_t job_id, const bfi_convergence *conv, double *result, double *abs_err,
                                bfi_adaptive_stats *stats, int device);

/* The lattice integral of Eq. (Gen2) over the box prod [lo_j, hi_j] (host
 * arrays [d]) with the context's device: the test compares r = Z_s (done in
 * logarithms, so Z_s may lie outside the double range), a subvolume is
 * halved along its widest side (the first on ties), and totals (host
 * [bfi_totals_len(nx)]) is the FP64 merge of the kept second evaluations.
 * The kept subvolumes, in the order they are kept (by round, then by
 * position in the round), go to leaf_lo / leaf_hi (host
 * [leaf_capacity * d]) and leaf_slots (host [leaf_capacity *
 * bfi_slot_len(nx)]) when those are not NULL, the first leaf_capacity of
 * them; stats->leaves tells how many there are.  Errors: BFI_E_INVALID,
 * BFI_E_UNSUPPORTED, BFI_E_NOMEM, BFI_E_CUDA. */
bfi_status bfi_adaptive_integrate(bfi_ctx *ctx, const bfi_lattice *lattice, const double *lo, const double *hi,
                                  uint64_t n, uint32_t seed, uint32_t job_id, bfi_precision precision,
                                  const bfi_convergence *conv, double *totals, bfi_adaptive_stats *stats,
                                  int64_t leaf_capacity, double *leaf_lo, double *leaf_hi, double *leaf_slots);

/* ------------------------------------------------------------------------ */
/* FP64 merge of subvolume records on the host.                             */
/* ------------------------------------------------------------------------ */

/* Merge nsub slots (host, [nsub * slot_len]) into totals (host) with the
 * same definitions as the device merge; used to combine records produced by
 * several executions, devices or processes (Sec. 1: the integral over a
 * region is the sum of the integrals over its parts).  Errors: BFI_E_INVALID. */
bfi_status bfi_merge_host(int32_t nx, int64_t nsub, const double *slots, double *totals);

/* ------------------------------------------------------------------------ */
/* Stated arithmetic error of a result.                                     */
/* ------------------------------------------------------------------------ */

/* A bound on the arithmetic error of one result of the box sampler: how far
 * its Z and C(r) can lie from the same Monte Carlo estimator (Sec. 3: V mean f
 * over each subvolume, summed) evaluated in exact arithmetic on the same
 * points -- in BFI_FP32 the same float points -- including the
 * negligible-weight truncation.  It adds up first-order rounding bounds of
 * each step of the path in the given precision: the action of Eq. (Gen2), the
 * weight (with the documented accuracy of CUDA's exp and expf), the products
 * P_r, the per-thread sums and the FP64 merges.  The statistical error (totals
 * [1] and [4 + R + r]) is separate and usually far larger.
 *   lattice, precision   those the result was computed with
 *   nsub, slots          host [nsub * bfi_slot_len(nx)]: the result's
 *                        subvolume records (their shifts and budgets enter)
 *   vmax                 the largest |coordinate| of any subvolume box (5 for
 *                        boxes inside [-5, 5]^d)
 *   bound                host [1 + R] out: bound[0] on |dZ| / Z, bound[1 + r]
 *                        on |dC(r)| / C(0)
 * In BFI_FP32 the bound is below 1e-6 for the lattices and boxes of the
 * workloads.  Errors: BFI_E_INVALID (bad arguments, records without
 * weight). */
bfi_status bfi_error_bound(const bfi_lattice *lattice, bfi_precision precision, int64_t nsub, const double *slots,
                           double vmax, double *bound);

/* ------------------------------------------------------------------------ */
/* Single steps of the path, for step-by-step checks.                        */
/* ------------------------------------------------------------------------ */

/* Coordinates of samples [first, first + count) of one subvolume (step 1 of
 * the path), widened to double.  lo, hi: device [d]; y: device [count * d].
 * Synchronous on 'stream'.  Errors: BFI_E_INVALID, BFI_E_CUDA. */
bfi_status bfi_points(int32_t d, const double *lo, const double *hi, uint32_t sub_id,
                      uint32_t seed, uint32_t job_id, uint64_t first, int64_t count,
                      bfi_precision precision, double *y, void *stream);

/* Action S and products P_r at given points (steps 2 and 4), evaluated by
 * the same device code as the integrand in the given precision (BFI_FP32
 * rounds y to float first).  y: device [npts * d]; S: device [npts];
 * P: device [npts * R].  Synchronous on 'stream'.
 * Errors: BFI_E_INVALID, BFI_E_UNSUPPORTED, BFI_E_CUDA. */
bfi_status bfi_eval(const bfi_lattice *lattice, int64_t npts, const double *y,
                    bfi_precision precision, double *S, double *P, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BFI_H */
