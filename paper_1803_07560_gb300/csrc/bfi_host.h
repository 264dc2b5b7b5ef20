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
// Samples per chunk for a job of 'total' samples (depends on the job only).
int64_t plan_chunk_samples(uint64_t total);
// Negligible-weight window for the largest per-subvolume budget n_max.
float plan_negligible_window(bfi_precision precision, uint64_t n_max);

}  // namespace bfi
