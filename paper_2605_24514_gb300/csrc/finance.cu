// Causal centering of return rows (Section 5.1): the finance layer's front end. A row r_t of raw
// returns becomes R_t = r_t - mu_t before it is appended, with mu_t the expanding mean (Option A,
// mu_t = mu_{t-1} + (r_t - mu_{t-1}) / t) or the exponentially weighted mean (Option B,
// mu_t = (1 - a) mu_{t-1} + a r_t) of the returns seen so far, so that no row is centered with
// information from its future. The state (mu in FP64 and the row count) lives on the device.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/isvd.h"
#include "isvd_common.cuh"

struct isvd_center_ctx {
  int mode = ISVD_CENTER_CAUSAL;
  double alpha = 0.0;
  int64_t n = 0, cap = 0, count = 0;
  int prec = ISVD_FP64;
  cudaStream_t stream = nullptr;
  double* mu = nullptr;     // n means (FP64)
  void* stage = nullptr;    // device staging of host rows (in and out)
  int64_t stage_cap = 0;    // bytes
};

namespace {

// One thread per asset: walks the rows in order, updating its mean and writing the centered value.
// The arithmetic is spelled out with round-to-nearest intrinsics so that no contraction changes it.
template <typename T>
__global__ void k_center_rows(const T* __restrict__ raw, int64_t rows, int64_t ld_raw, T* __restrict__ out,
                              int64_t ld_out, int64_t n, double* __restrict__ mu, int64_t count0, int mode,
                              double alpha) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double m = mu[j];
  for (int64_t t = 0; t < rows; ++t) {
    const double r = (double)raw[t * ld_raw + j];
    if (mode == ISVD_CENTER_CAUSAL) {
      m = __dadd_rn(m, __ddiv_rn(__dsub_rn(r, m), (double)(count0 + t + 1)));
    } else {
      m = __dadd_rn(__dmul_rn(1.0 - alpha, m), __dmul_rn(alpha, r));
    }
    out[t * ld_out + j] = (T)__dsub_rn(r, m);
  }
  mu[j] = m;
}

isvd_status ensure_stage(isvd_center_ctx* c, int64_t bytes) {
  if (bytes <= c->stage_cap) return ISVD_OK;
  if (c->stage) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->stage);
    c->stage = nullptr;
  }
  c->stage_cap = std::max(bytes, 2 * c->stage_cap);
  if (cudaMalloc(&c->stage, (size_t)c->stage_cap) != cudaSuccess) {
    cudaGetLastError();
    c->stage_cap = 0;
    return ISVD_ENOMEM;
  }
  return ISVD_OK;
}

isvd_status grow_mu(isvd_center_ctx* c, int64_t n_new) {
  if (n_new <= c->cap) return ISVD_OK;
  const int64_t cap = std::max(n_new, 2 * c->cap);
  double* m2 = nullptr;
  if (cudaMalloc((void**)&m2, 8 * (size_t)cap) != cudaSuccess) {
    cudaGetLastError();
    return ISVD_ENOMEM;
  }
  if (c->mu && cudaMemcpyAsync(m2, c->mu, 8 * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return ISVD_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ISVD_ECUDA;
  if (c->mu) cudaFree(c->mu);
  c->mu = m2;
  c->cap = cap;
  return ISVD_OK;
}

}  // namespace

extern "C" {

isvd_status isvd_center_create(int32_t mode, double alpha, int64_t n, int32_t prec, void* cuda_stream,
                               isvd_center_t* out) {
  if (!out) return ISVD_EINVAL;
  *out = nullptr;
  if (n < 1 || (prec != ISVD_FP64 && prec != ISVD_FP32)) return ISVD_EINVAL;
  if (mode != ISVD_CENTER_CAUSAL && mode != ISVD_CENTER_EW) return ISVD_EINVAL;
  if (mode == ISVD_CENTER_EW && !(alpha > 0.0 && alpha < 1.0)) return ISVD_EINVAL;
  isvd_center_ctx* c = new isvd_center_ctx();
  c->mode = mode;
  c->alpha = alpha;
  c->prec = prec;
  c->stream = (cudaStream_t)cuda_stream;
  isvd_status s = grow_mu(c, n);
  if (s == ISVD_OK && cudaMemsetAsync(c->mu, 0, 8 * (size_t)n, c->stream) != cudaSuccess) s = ISVD_ECUDA;
  if (s != ISVD_OK) {
    isvd_center_destroy(c);
    return s;
  }
  c->n = n;
  *out = c;
  return ISVD_OK;
}

void isvd_center_destroy(isvd_center_t c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->mu) cudaFree(c->mu);
  if (c->stage) cudaFree(c->stage);
  delete c;
}

isvd_status isvd_center_rows(isvd_center_t c, const void* raw, int64_t rows, int64_t ld_raw, void* out,
                             int64_t ld_out, int on_device) {
  if (!c || !raw || !out || rows < 0 || ld_raw < c->n || ld_out < c->n) return ISVD_EINVAL;
  if (rows == 0) return ISVD_OK;
  const size_t es = c->prec == ISVD_FP64 ? 8 : 4;
  const void* din = raw;
  void* dout = out;
  if (!on_device) {
    const int64_t bytes = rows * c->n * (int64_t)es;
    isvd_status s = ensure_stage(c, 2 * bytes);
    if (s) return s;
    din = c->stage;
    dout = static_cast<char*>(c->stage) + bytes;
    if (cudaMemcpy2DAsync(c->stage, c->n * es, raw, ld_raw * es, c->n * es, rows, cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
      return ISVD_ECUDA;
  }
  const int64_t li = on_device ? ld_raw : c->n, lo = on_device ? ld_out : c->n;
  const unsigned blocks = (unsigned)((c->n + 127) / 128);
  if (c->prec == ISVD_FP64)
    k_center_rows<double><<<blocks, 128, 0, c->stream>>>((const double*)din, rows, li, (double*)dout, lo, c->n, c->mu,
                                                         c->count, c->mode, c->alpha);
  else
    k_center_rows<float><<<blocks, 128, 0, c->stream>>>((const float*)din, rows, li, (float*)dout, lo, c->n, c->mu,
                                                        c->count, c->mode, c->alpha);
  if (cudaGetLastError() != cudaSuccess) return ISVD_ECUDA;
  c->count += rows;
  if (!on_device) {
    if (cudaMemcpy2DAsync(out, ld_out * es, dout, c->n * es, c->n * es, rows, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return ISVD_ECUDA;
  }
  return ISVD_OK;
}

isvd_status isvd_center_add_assets(isvd_center_t c, const double* mu_new, int64_t count) {
  if (!c || count < 0 || (count > 0 && !mu_new)) return ISVD_EINVAL;
  isvd_status s = grow_mu(c, c->n + count);
  if (s) return s;
  if (count > 0 &&
      (cudaMemcpyAsync(c->mu + c->n, mu_new, 8 * (size_t)count, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
       cudaStreamSynchronize(c->stream) != cudaSuccess))
    return ISVD_ECUDA;
  c->n += count;
  return ISVD_OK;
}

isvd_status isvd_center_state(isvd_center_t c, double* mu, int64_t* count) {
  if (!c) return ISVD_EINVAL;
  if (mu && (cudaMemcpyAsync(mu, c->mu, 8 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
             cudaStreamSynchronize(c->stream) != cudaSuccess))
    return ISVD_ECUDA;
  if (count) *count = c->count;
  return ISVD_OK;
}

}  // extern "C"
