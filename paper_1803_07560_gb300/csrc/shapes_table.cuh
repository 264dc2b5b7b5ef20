// shapes_table.cuh -- the table of one shapes_*.cu translation unit: for each
// lattice shape in BFI_TABLE_SHAPES (a list from bfi_kernels.h), the
// thread-per-sample integrand, range-map and Gaussian kernels with their
// launchers and occupancy queries, exported as the function BFI_TABLE_NAME.
// Each translation unit defines those two macros and includes this file once.
#pragma once

#include "integrand_kernels.cuh"
#include "mapped_kernels.cuh"

namespace bfi {

#define BFI_SHAPE_ENTRY(NX, NT)                                                   \
    {NX, NT, 0,                                                                   \
     {launch_integrand<NX, NT, double>, launch_integrand<NX, NT, float>},         \
     {occupancy_integrand<NX, NT, double>, occupancy_integrand<NX, NT, float>},   \
     launch_eval<NX, NT>, launch_transform<NX, NT>, occupancy_transform<NX, NT>,  \
     gaussian_entry<NX, NT>(), gaussian_occupancy_entry<NX, NT>(),                \
     PartialScreen<NX, NT>::enabled ? 1 : 0},

static const ShapeKernels kTable[] = {BFI_TABLE_SHAPES(BFI_SHAPE_ENTRY)};

const ShapeKernels *BFI_TABLE_NAME(int *n) {
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}

}  // namespace bfi
