// Kernel instantiations for f16 coefficient storage.
#include "wt_kernels.cuh"

WT_INSTANTIATE_TABLES(__half, 2)
