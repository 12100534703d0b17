// isvd_orth_error_noalloc: the loss-of-orthogonality measurement max|Q^T Q - I| for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory pool that forbids new
// allocations, inside a region that must not synchronise the device (cudaMalloc/cudaFree can), or
// in a process whose allocator belongs to another framework. This entry point needs no
// allocation: its scratch (the r x r FP64 Gram matrix and one result slot) lives in a file-scope
// __device__ array of fixed size, which every GPU that loads the library keeps until exit.
#include <mutex>

#include "../../include/isvd.h"
#include "isvd_common.cuh"

namespace {

constexpr int kNoAllocMaxR = ISVD_NOALLOC_MAX_R;
constexpr int kNoAllocTile = 32;
constexpr int kNoAllocChunk = 64;
constexpr int kNoAllocMaxDevices = 64;

// Scratch shared by every call: the Gram matrix (kNoAllocMaxR^2 doubles = 128 KiB) plus 32
// doubles of padding/result space.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxR * kNoAllocMaxR + 32];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// G[a, b] += sum over a slice of rows of Q[row, a] Q[row, b] (G zeroed by the caller), products
// summed in the storage type over runs of 16 rows and then in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_gram_noalloc(const T* __restrict__ Q, int64_t ld, int r, int64_t rows,
                                                      int64_t rows_per_split, double* __restrict__ G) {
  __shared__ T xs[kNoAllocChunk][kNoAllocTile + 1];
  __shared__ T ys[kNoAllocChunk][kNoAllocTile + 1];
  const int a0 = blockIdx.x * kNoAllocTile, b0 = blockIdx.y * kNoAllocTile;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  int64_t r_end = r_begin + rows_per_split;
  if (r_end > rows) r_end = rows;
  const int t = threadIdx.x;
  const int ta = t & 31, tb = t >> 5;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t base = r_begin; base < r_end; base += kNoAllocChunk) {
    for (int idx = t; idx < kNoAllocChunk * kNoAllocTile; idx += 256) {
      const int rr = idx / kNoAllocTile, c = idx - rr * kNoAllocTile;
      const int64_t row = base + rr;
      const bool okr = row < r_end;
      xs[rr][c] = (okr && a0 + c < r) ? Q[row * ld + a0 + c] : T(0);
      ys[rr][c] = (okr && b0 + c < r) ? Q[row * ld + b0 + c] : T(0);
    }
    __syncthreads();
    T part[4] = {0, 0, 0, 0};
    for (int rr = 0; rr < kNoAllocChunk; ++rr) {
      const T xv = xs[rr][ta];
#pragma unroll
      for (int q = 0; q < 4; ++q) part[q] += xv * ys[rr][tb + 8 * q];
      if ((rr & 15) == 15) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] += (double)part[q];
          part[q] = T(0);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ta, b = b0 + tb + 8 * q;
    if (a < r && b < r && acc[q] != 0.0) atomicAdd(&G[(int64_t)a * r + b], acc[q]);
  }
}

// *out = max |G - I| over the r x r matrix G.
__global__ void k_offident_noalloc(const double* __restrict__ G, int r, double* __restrict__ out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx - a * r;
    mx = fmax(mx, fabs(G[idx] - (a == b ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, red[w]);
    *out = m2;
  }
}

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
    const int64_t splits_target = 304;
    int64_t rps = (rows + splits_target - 1) / splits_target;
    rps = ((rps + kNoAllocChunk - 1) / kNoAllocChunk) * kNoAllocChunk;
    if (rps < kNoAllocChunk) rps = kNoAllocChunk;
    const int tiles = (r + kNoAllocTile - 1) / kNoAllocTile;
    dim3 grid((unsigned)tiles, (unsigned)tiles, (unsigned)((rows + rps - 1) / rps));
    k_gram_noalloc<T><<<grid, 256, 0, st>>>(Q, ld, r, rows, rps, G);
    if (cudaGetLastError() != cudaSuccess) return ISVD_ECUDA;
  }
  k_offident_noalloc<<<1, 256, 0, st>>>(G, r, err_out);
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
