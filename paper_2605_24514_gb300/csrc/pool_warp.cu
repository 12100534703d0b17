// Pool warp-per-update kernels (projection + core of one append per warp) and the row-parallel
// rotation kernels they feed, for rank buckets 8, 16 and 32.
#include "launch.cuh"
#include "pool_reorth.cuh"
#include "pool_rotate_tc.cuh"
#include "pool_warp.cuh"

namespace isvd {

namespace {
template <int KB>
void warp_launch(int count, cudaStream_t s, const PoolOp* ops, int base, int* retry, int* retry_n, void* scratch,
                 const int* chunks, int* block_op) {
  const int blocks = (count + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_pool_warp<KB><<<blocks, 32 * kWarpsPerBlock, warp_block_smem<KB>(), s>>>(
      ops, count, base, retry, retry_n, reinterpret_cast<RotScratch<KB>*>(scratch), chunks, block_op);
}
template <int KB>
void rotate_launch(int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch, const int* chunks,
                   const int* block_op) {
  k_pool_rotate<KB><<<nblocks, kPoolRotThreads, rot_smem_bytes<KB>(), s>>>(
      ops, reinterpret_cast<const RotScratch<KB>*>(scratch), chunks, block_op);
}
template <int KB>
void rotate_tc_launch(int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch, const int* chunks,
                      const int* block_op) {
  k_pool_rotate_tc<KB><<<nblocks, kTcRotThreads, TcRotLayout<KB>::kBytes, s>>>(
      ops, reinterpret_cast<const RotScratch<KB>*>(scratch), chunks, block_op);
}
}  // namespace

cudaError_t pool_warp_launch(int kb, int count, cudaStream_t s, const PoolOp* ops, int base, int* retry, int* retry_n,
                             void* scratch, const int* chunks, int* block_op) {
  switch (kb) {
    case 8: warp_launch<8>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op); break;
    case 16: warp_launch<16>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op); break;
    default: warp_launch<32>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op); break;
  }
  return cudaGetLastError();
}

cudaError_t pool_rotate_launch(int kb, int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch,
                               const int* chunks, const int* block_op, bool use_tc) {
  switch (kb) {
    case 8: rotate_launch<8>(nblocks, s, ops, scratch, chunks, block_op); break;
    case 16:
      if (use_tc) rotate_tc_launch<16>(nblocks, s, ops, scratch, chunks, block_op);
      else rotate_launch<16>(nblocks, s, ops, scratch, chunks, block_op);
      break;
    default:
      if (use_tc) rotate_tc_launch<32>(nblocks, s, ops, scratch, chunks, block_op);
      else rotate_launch<32>(nblocks, s, ops, scratch, chunks, block_op);
      break;
  }
  return cudaGetLastError();
}

cudaError_t pool_reorth_launch(int count, cudaStream_t s, const PoolReorthOp* list, double tol) {
  if (count <= 0) return cudaSuccess;
  k_pool_reorth<<<count, kReorthThreads, sizeof(ReorthSmem), s>>>(list, tol);
  return cudaGetLastError();
}

cudaError_t pool_warp_set_attrs() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pool_rotate<32>, a, (int)rot_smem_bytes<32>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate<16>, a, (int)rot_smem_bytes<16>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate<8>, a, (int)rot_smem_bytes<8>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<8>, a, (int)warp_block_smem<8>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<16>, a, (int)warp_block_smem<16>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<32>, a, (int)warp_block_smem<32>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate_tc<16>, a, (int)TcRotLayout<16>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate_tc<32>, a, (int)TcRotLayout<32>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_reorth, a, (int)sizeof(ReorthSmem));
  return e;
}

}  // namespace isvd
