// The pool's hand-back kernel: the updates the warp-per-update path returns, one CTA each.
#include "launch.cuh"
#include "pool_kernels.cuh"

namespace isvd {

cudaError_t pool_retry_launch(int blocks, cudaStream_t s, const PoolOp* ops, const int* retry, const int* retry_n) {
  k_pool_retry<32><<<blocks, pool_threads(32), pool_smem_bytes<32>(), s>>>(ops, retry, retry_n);
  return cudaGetLastError();
}

cudaError_t pool_retry_set_attr() {
  return cudaFuncSetAttribute(k_pool_retry<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pool_smem_bytes<32>());
}

}  // namespace isvd
