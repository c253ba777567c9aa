// Kernel instantiations for bf16 coefficient storage.
#include "wt_kernels.cuh"

WT_INSTANTIATE_TABLES(__nv_bfloat16, 1)
