// Kernel instantiations for shared-exponent 16-bit coefficient storage.
#include "wt_kernels.cuh"

WT_INSTANTIATE_TABLES(wt::se16_t, 3)
