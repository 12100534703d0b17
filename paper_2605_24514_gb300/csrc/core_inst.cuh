// Instantiations of the core SVD kernel for one storage type (included by core_f32.cu and
// core_f64.cu with ISVD_CORE_T defined).
#include "launch.cuh"
#include "update_kernels.cuh"

namespace isvd {

template <typename T>
cudaError_t core_launch(int kb, int threads, size_t smem, cudaStream_t s, int kind, DevState* st, double* sig,
                        const double* p, const T* U, const T* V, int ld, int64_t ei, int64_t ej, double delta, T* A,
                        int64_t lda, T* UK, T* VKo, int ldo, double* px, double tol_rel, const T* RU,
                        const T* RV, int ldr, float* gq) {
#define ISVD_CORE_ARGS kind, st, sig, p, U, V, ld, ei, ej, delta, A, lda, UK, VKo, ldo, px, tol_rel, RU, RV, ldr, gq
  switch (kb) {
    case 16: k_core<T, T, 16><<<1, threads, smem, s>>>(ISVD_CORE_ARGS); break;
    case 32: k_core<T, T, 32><<<1, threads, smem, s>>>(ISVD_CORE_ARGS); break;
    case 64: k_core<T, T, 64><<<1, threads, smem, s>>>(ISVD_CORE_ARGS); break;
    default: k_core<T, T, 128><<<1, threads, smem, s>>>(ISVD_CORE_ARGS); break;
  }
#undef ISVD_CORE_ARGS
  return cudaGetLastError();
}

template <typename T>
cudaError_t core_set_attrs(const size_t smem[4]) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_core<T, T, 16>, a, (int)smem[0]);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_core<T, T, 32>, a, (int)smem[1]);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_core<T, T, 64>, a, (int)smem[2]);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_core<T, T, 128>, a, (int)smem[3]);
  return e;
}

template cudaError_t core_launch<ISVD_CORE_T>(int, int, size_t, cudaStream_t, int, DevState*, double*, const double*,
                                              const ISVD_CORE_T*, const ISVD_CORE_T*, int, int64_t, int64_t, double,
                                              ISVD_CORE_T*, int64_t, ISVD_CORE_T*, ISVD_CORE_T*, int, double*, double,
                                              const ISVD_CORE_T*, const ISVD_CORE_T*, int, float*);
template cudaError_t core_set_attrs<ISVD_CORE_T>(const size_t[4]);

}  // namespace isvd
