// Loss-of-orthogonality monitor and re-orthogonalisation for the batched pool: one CTA per listed
// stream measures max|Q^T Q - I| for Q = U and Q = V (FP32 products summed over chunks of rows,
// then in FP64: the measurement error stays near 1e-8, well below the FP32 orthogonality level)
// and, when it exceeds the tolerance, re-orthonormalises that side by two Cholesky-QR passes
// (Q <- Q R^-1 with R^T R = Q^T Q, equivalent to CGS2 for nearly orthonormal Q); sigma is
// unchanged. The single-stream engine runs the same monitor through its own kernels.
#pragma once

#include "isvd_common.cuh"

namespace isvd {

struct PoolReorthOp {
  float* U;        // m x ld
  float* V;        // n x ld
  DevState* st;
  int64_t m, n;    // shape after the updates queued before this launch
  int32_t ld;      // row stride (a multiple of 4), >= r
  int32_t pad;
};

constexpr int kReorthThreads = 256;
constexpr int kReorthMaxR = 64;
constexpr int kReorthChunk = 32;  // rows staged per round
constexpr int kReorthPairs = (kReorthMaxR * (kReorthMaxR + 1) / 2 + kReorthThreads - 1) / kReorthThreads;

struct ReorthSmem {
  double G[kReorthMaxR * kReorthMaxR];   // Gram, then its Cholesky factor L (lower triangle)
  double Li[kReorthMaxR * kReorthMaxR];  // L^-1
  float Rinv[kReorthMaxR * kReorthMaxR]; // (L^T)^-1, upper triangular
  float rows[kReorthChunk * kReorthMaxR];
  double red[kReorthThreads / 32];
  int bad;
};

// G = Q^T Q (r x r, symmetric, FP64) over `rows` rows of Q (row stride ld).
__device__ inline void reorth_gram(const float* Q, int64_t rows, int ld, int r, ReorthSmem& S) {
  const int tid = threadIdx.x;
  const int npairs = r * (r + 1) / 2;
  int pa[kReorthPairs], pb[kReorthPairs];
#pragma unroll
  for (int q = 0; q < kReorthPairs; ++q) {
    int p = tid + q * kReorthThreads, a = 0;
    if (p < npairs) {
      while (p >= r - a) {  // pair index -> (a, b) with a <= b
        p -= r - a;
        ++a;
      }
      pa[q] = a;
      pb[q] = a + p;
    } else {
      pa[q] = pb[q] = -1;
    }
  }
  double acc[kReorthPairs];
#pragma unroll
  for (int q = 0; q < kReorthPairs; ++q) acc[q] = 0.0;
  const int c4 = ld / 4;
  for (int64_t r0 = 0; r0 < rows; r0 += kReorthChunk) {
    const int nr = (int)(rows - r0 < kReorthChunk ? rows - r0 : kReorthChunk);
    __syncthreads();
    const float4* src = reinterpret_cast<const float4*>(Q + r0 * ld);
    for (int f = tid; f < nr * c4; f += kReorthThreads) {
      const int rr = f / c4, cc = f - rr * c4;
      if (4 * cc < r) *reinterpret_cast<float4*>(&S.rows[rr * kReorthMaxR + 4 * cc]) = src[f];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kReorthPairs; ++q) {
      if (pa[q] < 0) continue;
      float s = 0.f;
      for (int rr = 0; rr < nr; ++rr) s = fmaf(S.rows[rr * kReorthMaxR + pa[q]], S.rows[rr * kReorthMaxR + pb[q]], s);
      acc[q] += (double)s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kReorthPairs; ++q) {
    if (pa[q] < 0) continue;
    S.G[pa[q] * r + pb[q]] = acc[q];
    S.G[pb[q] * r + pa[q]] = acc[q];
  }
  __syncthreads();
}

// max |G - I| (NaN-propagating), block-uniform result.
__device__ inline double reorth_offident(int r, ReorthSmem& S) {
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < r * r; idx += kReorthThreads) {
    const int a = idx / r, b = idx - a * r;
    const double v = fabs(S.G[idx] - (a == b ? 1.0 : 0.0));
    mx = (v > mx || isnan(v)) ? v : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (v > mx || isnan(v)) ? v : mx;
  }
  if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double m2 = 0.0;
  for (int w = 0; w < kReorthThreads / 32; ++w) {
    const double v = S.red[w];
    m2 = (v > m2 || isnan(v)) ? v : m2;
  }
  __syncthreads();
  return m2;
}

// One Cholesky-QR pass on Q (G must hold Q^T Q): L L^T = G, Q <- Q (L^T)^-1. Returns false (Q
// untouched) when G is not numerically positive definite.
__device__ inline bool reorth_cholqr(float* Q, int64_t rows, int ld, int r, ReorthSmem& S) {
  const int tid = threadIdx.x;
  if (tid == 0) S.bad = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      double d = S.G[j * r + j];
      for (int l = 0; l < j; ++l) d -= S.G[j * r + l] * S.G[j * r + l];
      if (!(d > 0.0)) {
        S.bad = 1;
        d = 1.0;
      }
      S.G[j * r + j] = sqrt(d);
    }
    __syncthreads();
    const double djj = S.G[j * r + j];
    for (int i = j + 1 + tid; i < r; i += kReorthThreads) {
      double s = S.G[i * r + j];
      for (int l = 0; l < j; ++l) s -= S.G[i * r + l] * S.G[j * r + l];
      S.G[i * r + j] = s / djj;
    }
    __syncthreads();
  }
  if (S.bad) return false;
  for (int col = tid; col < r; col += kReorthThreads) {
    for (int i = 0; i < r; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int l = col; l < i; ++l) s -= S.G[i * r + l] * S.Li[l * r + col];
      S.Li[i * r + col] = i < col ? 0.0 : s / S.G[i * r + i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += kReorthThreads) {
    const int a = idx / r, b = idx - a * r;
    S.Rinv[a * kReorthMaxR + b] = (float)S.Li[b * r + a];
  }
  __syncthreads();
  // Row by row: q <- q Rinv (Rinv upper triangular: output column j uses q[0..j]).
  for (int64_t row = tid; row < rows; row += kReorthThreads) {
    float* q = Q + row * ld;
    float in[kReorthMaxR];
    for (int c = 0; c < r; ++c) in[c] = q[c];
    for (int j = 0; j < r; ++j) {
      float s = 0.f;
      for (int c = 0; c <= j; ++c) s = fmaf(in[c], S.Rinv[c * kReorthMaxR + j], s);
      q[j] = s;
    }
  }
  __syncthreads();
  return true;
}

static __global__ void __launch_bounds__(kReorthThreads) k_pool_reorth(const PoolReorthOp* __restrict__ list, double tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  ReorthSmem& S = *reinterpret_cast<ReorthSmem*>(smem);
  const PoolReorthOp op = list[blockIdx.x];
  DevState* st = op.st;
  const int r = st->r;
  if (r < 1 || r > kReorthMaxR || r > op.ld) return;
  double err[2];
  bool fixed = false;
  for (int side = 0; side < 2; ++side) {
    float* Q = side == 0 ? op.U : op.V;
    const int64_t rows = side == 0 ? op.m : op.n;
    reorth_gram(Q, rows, op.ld, r, S);
    err[side] = reorth_offident(r, S);
    if (isnan(err[side])) {
      if (threadIdx.x == 0) atomicOr(&st->status, kStNonFinite);
      return;
    }
    if (err[side] > tol) {
      bool ok = reorth_cholqr(Q, rows, op.ld, r, S);
      if (ok) {
        reorth_gram(Q, rows, op.ld, r, S);
        ok = reorth_cholqr(Q, rows, op.ld, r, S);
      }
      fixed = fixed || ok;
    }
  }
  if (threadIdx.x == 0) {
    st->orth_u = err[0];
    st->orth_v = err[1];
    st->orth_runs += 1;
    if (fixed) st->reorths += 1;
  }
}

}  // namespace isvd
