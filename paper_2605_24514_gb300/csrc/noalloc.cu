// isvd_orth_error_noalloc: the loss-of-orthogonality measurement max|Q^T Q - I| for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory pool that forbids new
// allocations, inside a region that must not synchronise the device (cudaMalloc/cudaFree can), or
// in a process whose allocator belongs to another framework. This entry point needs no
// allocation: its scratch (the r x r FP64 Gram matrix and one result slot) lives in a file-scope
// __device__ array of fixed size, which every GPU that loads the library keeps until exit.
#include <algorithm>
#include <mutex>

#include "../../include/isvd.h"
#include "isvd_common.cuh"
#include "refresh_kernels.cuh"

namespace {

using isvd::k_gemm_tn;
using isvd::k_max_offident;
using isvd::kTnChunk;
using isvd::kTnTile;

constexpr int kNoAllocMaxR = ISVD_NOALLOC_MAX_R;
constexpr int kNoAllocMaxDevices = 64;

// Scratch shared by every call: the Gram matrix (kNoAllocMaxR^2 doubles = 128 KiB) plus 32
// doubles of padding/result space.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxR * kNoAllocMaxR + 32];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
isvd_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return ISVD_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ISVD_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return ISVD_OK;
}

template <typename T>
isvd_status orth_error_impl(const T* Q, int64_t rows, int r, int64_t ld, double* err_out, cudaStream_t st) {
  void* base = nullptr;
  isvd_status s = noalloc_scratch(&base);
  if (s) return s;
  double* G = static_cast<double*>(base);
  if (cudaMemsetAsync(G, 0, sizeof(double) * (size_t)r * r, st) != cudaSuccess) return ISVD_ECUDA;
  if (rows > 0) {
    // The library's Gram kernel with exact FP64 products (row splits summed by FP64 atomics), as
    // in the orthogonality monitor of isvd_reorthogonalize.
    const int64_t splits_target = 304;
    int64_t rps = (rows + splits_target - 1) / splits_target;
    rps = std::max<int64_t>(kTnChunk, (rps + kTnChunk - 1) / kTnChunk * kTnChunk);
    const unsigned tiles = (unsigned)((r + kTnTile - 1) / kTnTile);
    dim3 grid(tiles, tiles, (unsigned)((rows + rps - 1) / rps));
    k_gemm_tn<T, true><<<grid, 256, 0, st>>>(Q, ld, r, Q, ld, r, rows, rps, G, r);
    if (cudaGetLastError() != cudaSuccess) return ISVD_ECUDA;
  }
  k_max_offident<<<1, 256, 0, st>>>(G, r, err_out);
  if (cudaGetLastError() != cudaSuccess) return ISVD_ECUDA;
  return ISVD_OK;
}

}  // namespace

extern "C" isvd_status isvd_orth_error_noalloc(const void* Q, int64_t rows, int32_t r, int64_t ld, int32_t prec,
                                               double* err_out, void* cuda_stream) {
  if (!Q || !err_out || rows < 0 || r < 1 || ld < r) return ISVD_EINVAL;
  if (prec != ISVD_FP64 && prec != ISVD_FP32) return ISVD_EINVAL;
  if (r > kNoAllocMaxR) return ISVD_ESHAPE;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  return prec == ISVD_FP64 ? orth_error_impl<double>((const double*)Q, rows, r, ld, err_out, st)
                           : orth_error_impl<float>((const float*)Q, rows, r, ld, err_out, st);
}
