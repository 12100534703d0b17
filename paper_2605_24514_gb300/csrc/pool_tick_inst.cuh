// The pool's CTA kernel for one rank bucket (included by pool_tick<KB>.cu with ISVD_TICK_KB set):
// one whole update per CTA (entry updates, column appends, rank bucket 64).
#include "launch.cuh"
#include "pool_kernels.cuh"

namespace isvd {

template <int KB>
cudaError_t pool_tick_launch(int count, cudaStream_t s, const PoolOp* ops) {
  k_pool_tick<KB><<<count, pool_threads(KB), pool_smem_bytes<KB>(), s>>>(ops);
  return cudaGetLastError();
}

template <int KB>
cudaError_t pool_tick_set_attr() {
  return cudaFuncSetAttribute(k_pool_tick<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pool_smem_bytes<KB>());
}

template cudaError_t pool_tick_launch<ISVD_TICK_KB>(int, cudaStream_t, const PoolOp*);
template cudaError_t pool_tick_set_attr<ISVD_TICK_KB>();

}  // namespace isvd
