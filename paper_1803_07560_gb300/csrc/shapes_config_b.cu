// shapes_config_b.cu -- the compiled thread-per-sample kernels for the shapes of
// BFI_SHAPES_CONFIG_B (bfi_kernels.h).
#define BFI_TABLE_SHAPES BFI_SHAPES_CONFIG_B
#define BFI_TABLE_NAME shapes_config_b
#include "shapes_table.cuh"
