// bfi_kernels.h -- internal interface between the C ABI (api.cu) and the
// kernels (integrand.cu).  Not installed; the public header is include/bfi.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfi {

constexpr int kBlock = 256;   // threads per CTA of the integrand kernels
constexpr int kMaxD = 512;    // largest lattice (d = nx * nt) the library accepts
#ifndef BFI_TWO_STAGE_MIN_ROWS
#define BFI_TWO_STAGE_MIN_ROWS 256
#endif
// rows per thread from which a chunk runs the two-stage screen
constexpr uint64_t kTwoStageMinRows = BFI_TWO_STAGE_MIN_ROWS;

// Lattice shapes with compiled thread-per-sample kernels (NX, NT), in five
// translation units of about equal compile time that compile in parallel
// (shapes_*.cu, each instantiating shapes_table.cuh); every other shape with
// d = NX NT <= kMaxD runs on the generic warp-per-sample kernels.
#define BFI_SHAPES_SMALL(X) X(2, 1) X(3, 1) X(4, 1) X(2, 2) X(3, 2) X(4, 2) X(6, 2) X(8, 2) X(10, 2)
#define BFI_SHAPES_CONFIG_A(X) X(10, 4)
#define BFI_SHAPES_CONFIG_B(X) X(16, 2) X(4, 4)
#define BFI_SHAPES_CONFIG_C(X) X(32, 2) X(6, 4)
#define BFI_SHAPES_CONFIG_D(X) X(8, 4) X(16, 4)

struct LatticeParams {
    int32_t nx, nt;
    double nu, D, a, tau, nonlinear, mass2;
};

struct IntegrandArgs {
    const double *lo;          // [nsub * d]
    const double *hi;          // [nsub * d]
    const uint32_t *sub_id;    // [nsub] or null
    const uint64_t *samples;   // [nsub]
    const int64_t *chunk_off;  // [nsub + 1]
    double *partials;          // [nchunks * (K + 2)]
    float *hint;               // [nsub] reference actions written by hint_f32
    unsigned long long *stats; // [1] fully evaluated samples (zeroed per execution), or null
    int64_t nsub;
    int64_t nchunks;
    int64_t chunk_samples;
    float skip_window;         // samples above (reference + skip_window) have negligible weight
    unsigned long long *screened;  // [1] samples the full FP32 screen examined after the partial one, or null
    unsigned long long *stage1;    // [1] samples of chunks that ran stage 1 of the two-stage screen, or null
    unsigned long long *next_chunk;  // [1] zeroed per execution: after its first chunk (blockIdx.x) a CTA takes
                                     // the next chunk not yet taken; null: CTA b takes b, b + grid, ...
    int64_t tail_sub;              // subvolumes s >= tail_sub are cut into chunks of tail_chunk_samples
    int64_t tail_chunk_samples;    // (0: every subvolume into chunks of chunk_samples)
};

struct MergeArgs {
    const double *lo, *hi;
    const int64_t *chunk_off;
    const double *partials;
    double *slots;
    int64_t nsub;
    int32_t R, d;
    int32_t log_norm_set;      // 1: every record's log-volume is log_norm (Gaussian sampler)
    double log_norm;
};

struct TotalsArgs {
    const double *slots;
    double *totals;
    double *f_buf;             // [2 nsub] scratch: per-subvolume scale factors f_s, then f_s^2 / (n_s - 1)
    int64_t nsub;
    int32_t R;
};

struct PointsArgs {
    const double *lo, *hi;
    double *y;
    uint64_t first;
    int64_t count;
    int32_t d;
    uint32_t sub_id;
};

struct EvalArgs {
    const double *y;
    double *S, *P;
    int64_t npts;
};

using IntegrandLauncher = cudaError_t (*)(const IntegrandArgs &, const LatticeParams &, uint32_t, uint32_t, int,
                                          cudaStream_t);
struct MapArgs;
// Gaussian sampler: map arguments and whether the factor is upper triangular
using GaussLauncher = cudaError_t (*)(const IntegrandArgs &, const LatticeParams &, const MapArgs &, bool, uint32_t,
                                      uint32_t, int, cudaStream_t);
using OccupancyQuery = cudaError_t (*)(int nx, int nt, int *blocks_per_sm);
using EvalLauncher = cudaError_t (*)(const EvalArgs &, const LatticeParams &, int mode, cudaStream_t);

// index 0 = FP64, 1 = FP32
struct ShapeKernels {
    int nx, nt;
    int kernel;   // 0 = thread-per-sample (compiled shape), 1 = generic warp-per-sample
    IntegrandLauncher integrand[2];
    OccupancyQuery occupancy[2];
    EvalLauncher eval;   // mode 0 = FP64, 1 = FP32, 2 = FP32 compensated action
    IntegrandLauncher transform;      // the range map in FP64, thread per sample (null: generic_mapped)
    OccupancyQuery transform_occupancy;
    GaussLauncher gaussian;           // the Gaussian sampler in FP64, thread per sample (null: generic_mapped)
    OccupancyQuery gaussian_occupancy;
    int two_stage;                    // 1: the box-sampler kernels screen with the partial action first
};

// Compiled shape tables (shapes_*.cu) and the generic kernels (generic.cu);
// find_shape looks in the tables, then falls back to the generic kernels
// (null if d > kMaxD).
const ShapeKernels *shapes_small(int *n);
const ShapeKernels *shapes_config_a(int *n);
const ShapeKernels *shapes_config_b(int *n);
const ShapeKernels *shapes_config_c(int *n);
const ShapeKernels *shapes_config_d(int *n);
const ShapeKernels *generic_shape(int nx, int nt);
const ShapeKernels *find_shape(int nx, int nt);
cudaError_t launch_merges(const MergeArgs &m, const TotalsArgs &t, cudaStream_t st);

// Mapped samplers (generic.cu): kind 1 = the range map of Sec. 4, kind 2 =
// Gaussian importance sampling with device mean [d] (or null) and factor [d*d].
constexpr int kMaxGaussD = 64;
struct MapArgs {
    int kind;
    const double *mean;
    const double *factor;
};
cudaError_t launch_mapped(const IntegrandArgs &a, const LatticeParams &p, const MapArgs &m, uint32_t seed, uint32_t job,
                          int grid, cudaStream_t st);
cudaError_t occupancy_mapped(int nx, int nt, int kind, int *blocks_per_sm);
cudaError_t launch_points(const PointsArgs &a, bool fp32, uint32_t seed, uint32_t job, cudaStream_t st);

}  // namespace bfi
