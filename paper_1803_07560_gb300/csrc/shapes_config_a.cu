// shapes_config_a.cu -- the compiled thread-per-sample kernels for the shapes of
// BFI_SHAPES_CONFIG_A (bfi_kernels.h).
#define BFI_TABLE_SHAPES BFI_SHAPES_CONFIG_A
#define BFI_TABLE_NAME shapes_config_a
#include "shapes_table.cuh"
