// Kernel instantiations for f32 coefficient storage.
#include "wt_kernels.cuh"

WT_INSTANTIATE_TABLES(float, 0)
