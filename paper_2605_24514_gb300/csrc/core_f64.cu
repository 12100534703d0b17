// Core SVD kernels for FP64 storage (one-sided Jacobi core).
#define ISVD_CORE_T double
#include "core_inst.cuh"
