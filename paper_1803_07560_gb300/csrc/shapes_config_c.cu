// shapes_config_c.cu -- the compiled thread-per-sample kernels for the shapes of
// BFI_SHAPES_CONFIG_C (bfi_kernels.h).
#define BFI_TABLE_SHAPES BFI_SHAPES_CONFIG_C
#define BFI_TABLE_NAME shapes_config_c
#include "shapes_table.cuh"
