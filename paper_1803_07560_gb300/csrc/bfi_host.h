// bfi_host.h -- host-side helpers shared by the C-ABI translation units
// (defined in api.cu).  Internal; the public header is include/bfi.h.
#pragma once

#include "bfi.h"

#include <cstdint>

namespace bfi {

// Records 'message' as the calling thread's last error and returns 'status'.
bfi_status set_error(bfi_status status, const char *message);
// Argument checks of a lattice (BFI_OK or BFI_E_INVALID with a message).
bfi_status validate_lattice(const bfi_lattice *lattice);
// How a job's budgets are cut into chunks (depends on the job only).
// Subvolume s is cut into chunks of samples_of(s), the last one ragged;
// chunk indices run subvolume by subvolume.
struct ChunkLayout {
    int64_t chunk_samples = 0;       // subvolumes s < tail_sub
    int64_t tail_chunk_samples = 0;  // subvolumes s >= tail_sub
    int64_t tail_sub = 0;            // nsub: no tail
    int64_t samples_of(int64_t s) const { return s >= tail_sub ? tail_chunk_samples : chunk_samples; }
    int64_t chunks_of(int64_t s, uint64_t n_s) const {
        const uint64_t c = static_cast<uint64_t>(samples_of(s));
        return static_cast<int64_t>((n_s + c - 1) / c);
    }
};
ChunkLayout plan_chunk_layout(const uint64_t *samples, int64_t nsub);
// Negligible-weight window for the largest per-subvolume budget n_max.
float plan_negligible_window(bfi_precision precision, uint64_t n_max);

// N-sphere integrand (nsphere.cu): nbox boxes (host arrays [nbox][dims],
// n and sub_id [nbox]) in one launch on 'device'; sums [nbox][2 + dims] are
// [sum f, sum f^2, sum_{x_j < mid_j} f for each j], written to host memory.
bfi_status nsphere_batch(int dims, int64_t nbox, const double *lo, const double *hi, const uint64_t *n,
                         const uint32_t *sub_id, uint32_t seed, uint32_t job_id, int device, double *sums);
// Result, error and split suggestion of one box from its sums.
void nsphere_finish(int dims, const double *lo, const double *hi, uint64_t n, const double *sums, double *result,
                    double *abs_err, int32_t *split_dim);

}  // namespace bfi
