// Pool warp-per-update kernels (projection + core of one append per warp) and the row-parallel
// rotation kernels they feed, for rank buckets 8, 16 and 32.
#include <algorithm>

#include "launch.cuh"
#include "pool_reorth.cuh"
#include "pool_rotate_tc.cuh"
#include "pool_warp.cuh"

namespace isvd {

namespace {
template <int KB>
void warp_launch(int count, cudaStream_t s, const PoolOp* ops, int base, int* retry, int* retry_n, void* scratch,
                 const int* chunks, int* block_op, int rot_rows, int nblocks, int* kcheck) {
  const int blocks = (count + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_pool_warp<KB><<<blocks, 32 * kWarpsPerBlock, warp_block_smem<KB>(), s>>>(
      ops, count, base, retry, retry_n, reinterpret_cast<RotScratch<KB>*>(scratch), chunks, block_op, rot_rows,
      nblocks, kcheck);
}
int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
  }
  return sms;
}
// Persistent CTAs over contiguous ranges of the rotation blocks: as many as fit on the SMs.
template <int KB>
void rotate_launch(int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch, const int* chunks,
                   const int* block_op, const void* tmaps, int nops, int nmaps, int* kcheck) {
  static int per_sm = 0;
  if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pool_rotate<KB>, kRotThreadsAll,
                                                                    RotTmaLayout<KB>::kBytes) != cudaSuccess ||
                      per_sm < 1)) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int grid = std::min(nblocks, per_sm * device_sms());
  if (grid <= 0) return;
  k_pool_rotate<KB><<<grid, kRotThreadsAll, RotTmaLayout<KB>::kBytes, s>>>(
      ops, reinterpret_cast<const RotScratch<KB>*>(scratch), chunks, block_op, nblocks,
      reinterpret_cast<const RowTensorMap*>(tmaps), nops, nmaps, kcheck);
}
template <int KB>
void rotate_tc_launch(int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch, const int* chunks,
                      const int* block_op, const void* tmaps) {
  // Persistent CTAs: a few per SM, each over a contiguous range of the rotation blocks.
  const int grid = std::min(nblocks, kTcCtasPerSm * device_sms());
  if (grid <= 0) return;
  k_pool_rotate_tc<KB><<<grid, kTcRotThreads, TcRotLayout<KB>::kBytes, s>>>(
      ops, reinterpret_cast<const RotScratch<KB>*>(scratch), chunks, block_op, nblocks,
      reinterpret_cast<const RowTensorMap*>(tmaps));
}
}  // namespace

cudaError_t pool_warp_launch(int kb, int count, cudaStream_t s, const PoolOp* ops, int base, int* retry, int* retry_n,
                             void* scratch, const int* chunks, int* block_op, int rot_rows, int nblocks, int* kcheck) {
  switch (kb) {
    case 8: warp_launch<8>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op, rot_rows, nblocks, kcheck); break;
    case 16: warp_launch<16>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op, rot_rows, nblocks, kcheck); break;
    default: warp_launch<32>(count, s, ops, base, retry, retry_n, scratch, chunks, block_op, rot_rows, nblocks, kcheck); break;
  }
  return cudaGetLastError();
}

int pool_rot_rows(int kb, bool use_tc) { return use_tc && (kb == 16 || kb == 32) ? kTcRotRows : kPoolRotRows; }

cudaError_t pool_rotate_launch(int kb, int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch,
                               const int* chunks, const int* block_op, bool use_tc, const void* tmaps, int nops,
                               int nmaps, int* kcheck) {
  switch (kb) {
    case 8: rotate_launch<8>(nblocks, s, ops, scratch, chunks, block_op, tmaps, nops, nmaps, kcheck); break;
    case 16:
      if (use_tc) rotate_tc_launch<16>(nblocks, s, ops, scratch, chunks, block_op, tmaps);
      else rotate_launch<16>(nblocks, s, ops, scratch, chunks, block_op, tmaps, nops, nmaps, kcheck);
      break;
    default:
      if (use_tc) rotate_tc_launch<32>(nblocks, s, ops, scratch, chunks, block_op, tmaps);
      else rotate_launch<32>(nblocks, s, ops, scratch, chunks, block_op, tmaps, nops, nmaps, kcheck);
      break;
  }
  return cudaGetLastError();
}

cudaError_t pool_reorth_launch(int count, cudaStream_t s, const PoolReorthOp* list, double tol) {
  if (count <= 0) return cudaSuccess;
  k_pool_reorth<<<count, kReorthThreads, sizeof(ReorthSmem), s>>>(list, tol);
  return cudaGetLastError();
}

namespace {
__global__ void k_pool_complete(const PoolOp* __restrict__ ops, int count, PoolCompletion* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const PoolOp& op = ops[q];
  const DevState* st = op.st;
  PoolCompletion c;
  c.seq = op.seq;
  c.stream = op.sid;
  c.kind = op.kind;
  const int status = st->status;
  c.status = status & kStNonFinite ? 9 : status & kStNotConv ? 6 : status & kStTimeout ? 7 : status & kStLayout ? 8 : 0;  // isvd_status
  c.r = st->r;
  c.rho = op.kind == kEntry ? 0.0 : st->rho;
  c.sigma_max = st->r > 0 ? op.sig[0] : 0.0;
  c.done_ns = tc::globaltimer_ns();
  out[q] = c;
}

__global__ void k_pool_gather_sigma(const double* const* __restrict__ sig, const DevState* const* __restrict__ st,
                                    int64_t n, int ld, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ld) return;
  const int64_t s = idx / ld;
  const int c = (int)(idx - s * ld);
  out[idx] = c < st[s]->r ? sig[s][c] : 0.0;
}
__global__ void k_pool_gather_status(const DevState* const* __restrict__ st, int64_t n, int* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = st[s]->status;
}
// Adaptive rank (Eq. evr-rank-rule as a growth rule), one thread per listed stream.
// The shrink side (tau_shrink > 0): when the leading k - 1 components explain at least tau_shrink
// of N_t, k <- k - 1 (at least 1) and the maintained rank is cut to it.
__global__ void k_pool_rank(const PoolRankOp* __restrict__ list, int count, double tau, double tau_shrink) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const PoolRankOp op = list[q];
  DevState* st = op.st;
  const int r = st->r, k = st->k;
  double ss = 0.0, ss_km1 = 0.0;
  for (int c = 0; c < r; ++c) {
    const double v = op.sig[c] * op.sig[c];
    ss += v;
    if (c < k - 1) ss_km1 += v;
  }
  const double N = st->N;
  if (!(N > 0.0)) return;
  if (ss / N < tau) {
    if (k < op.kcap) st->k = k + 1;
  } else if (tau_shrink > 0.0 && k > 1 && ss_km1 / N >= tau_shrink) {
    st->k = k - 1;
    st->r = min(r, k - 1);
  }
}
}  // namespace

cudaError_t pool_rank_launch(int count, cudaStream_t s, const PoolRankOp* list, double tau, double tau_shrink) {
  if (count <= 0) return cudaSuccess;
  k_pool_rank<<<(count + 127) / 128, 128, 0, s>>>(list, count, tau, tau_shrink);
  return cudaGetLastError();
}

cudaError_t pool_complete_launch(int count, cudaStream_t s, const PoolOp* ops, PoolCompletion* out) {
  if (count <= 0) return cudaSuccess;
  k_pool_complete<<<(count + 127) / 128, 128, 0, s>>>(ops, count, out);
  return cudaGetLastError();
}

cudaError_t pool_gather_sigma_launch(int64_t n, cudaStream_t s, const double* const* sig, const DevState* const* st,
                                     int ld, double* out) {
  if (n <= 0) return cudaSuccess;
  const int64_t tot = n * ld;
  k_pool_gather_sigma<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(sig, st, n, ld, out);
  return cudaGetLastError();
}

cudaError_t pool_gather_status_launch(int64_t n, cudaStream_t s, const DevState* const* st, int* out) {
  if (n <= 0) return cudaSuccess;
  k_pool_gather_status<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(st, n, out);
  return cudaGetLastError();
}

cudaError_t pool_warp_set_attrs() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pool_rotate<32>, a, (int)RotTmaLayout<32>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate<16>, a, (int)RotTmaLayout<16>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate<8>, a, (int)RotTmaLayout<8>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<8>, a, (int)warp_block_smem<8>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<16>, a, (int)warp_block_smem<16>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_warp<32>, a, (int)warp_block_smem<32>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate_tc<16>, a, (int)TcRotLayout<16>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_rotate_tc<32>, a, (int)TcRotLayout<32>::kBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pool_reorth, a, (int)sizeof(ReorthSmem));
  return e;
}

}  // namespace isvd

#ifdef ISVD_CORE_TIMING
// Phase timing of this translation unit's kernels (its own copies of the stamp counters).
extern "C" int isvd_debug_warp_clock_sums(unsigned long long* out, int reset) {
  int e = (int)cudaMemcpyFromSymbol(out, isvd::isvd_core_clock_sum, sizeof(unsigned long long) * 32);
  if (!e) e = (int)cudaMemcpyFromSymbol(out + 32, isvd::isvd_core_clock_cnt, sizeof(unsigned long long) * 32);
  if (!e && reset) {
    unsigned long long z[32] = {};
    e = (int)cudaMemcpyToSymbol(isvd::isvd_core_clock_sum, z, sizeof(z));
    if (!e) e = (int)cudaMemcpyToSymbol(isvd::isvd_core_clock_cnt, z, sizeof(z));
  }
  return e;
}
#endif
