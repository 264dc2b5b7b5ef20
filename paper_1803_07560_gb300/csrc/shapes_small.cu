// shapes_small.cu -- instantiates the thread-per-sample integrand and sampler kernels for the
// lattice shapes listed in BFI_SHAPES_SMALL (bfi_kernels.h).
#include "integrand_kernels.cuh"
#include "mapped_kernels.cuh"

namespace bfi {

#define BFI_SHAPE_ENTRY(NX, NT)                                                   \
    {NX, NT, 0,                                                                   \
     {launch_integrand<NX, NT, double>, launch_integrand<NX, NT, float>},         \
     {occupancy_integrand<NX, NT, double>, occupancy_integrand<NX, NT, float>},   \
     launch_eval<NX, NT>, launch_transform<NX, NT>, occupancy_transform<NX, NT>,     \
     gaussian_entry<NX, NT>(), gaussian_occupancy_entry<NX, NT>(),                  \
     PartialScreen<NX, NT>::enabled ? 1 : 0},

static const ShapeKernels kTable[] = {BFI_SHAPES_SMALL(BFI_SHAPE_ENTRY)};

const ShapeKernels *shapes_small(int *n) {
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}

}  // namespace bfi
