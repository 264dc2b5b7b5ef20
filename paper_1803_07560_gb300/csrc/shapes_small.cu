// shapes_small.cu -- the compiled thread-per-sample kernels for the shapes of
// BFI_SHAPES_SMALL (bfi_kernels.h).
#define BFI_TABLE_SHAPES BFI_SHAPES_SMALL
#define BFI_TABLE_NAME shapes_small
#include "shapes_table.cuh"
