// shapes_config_d.cu -- the compiled thread-per-sample kernels for the shapes of
// BFI_SHAPES_CONFIG_D (bfi_kernels.h).
#define BFI_TABLE_SHAPES BFI_SHAPES_CONFIG_D
#define BFI_TABLE_NAME shapes_config_d
#include "shapes_table.cuh"
