// Core SVD kernels for FP32 storage (secular-equation core with the Jacobi fallback).
#define ISVD_CORE_T float
#include "core_inst.cuh"
