// Refresh (Section 2.4), metrics (Section 2.5) and re-orthogonalisation kernels.
#pragma once

#include "core_svd.cuh"
#include "isvd_common.cuh"

namespace isvd {

// C[a, b] += sum_row X[row, a] * Y[row, b] for a < cx, b < cy (C row-major FP64, ldc), over a
// slice of rows per block (grid.z). Products are summed in T over runs of 16 rows, then in FP64;
// with kExact every product is formed and summed in FP64 (exact products of FP32 data).
// 32 x 32 output tile per block, 256 threads, 4 outputs per thread.
constexpr int kTnTile = 32;
constexpr int kTnChunk = 64;
template <typename T, bool kExact = false>
__global__ void __launch_bounds__(256) k_gemm_tn(const T* __restrict__ X, int64_t ldx, int cx, const T* __restrict__ Y,
                                                 int64_t ldy, int cy, int64_t rows, int64_t rows_per_split,
                                                 double* __restrict__ C, int64_t ldc) {
  __shared__ T xs[kTnChunk][kTnTile + 1];
  __shared__ T ys[kTnChunk][kTnTile + 1];
  const int a0 = blockIdx.x * kTnTile, b0 = blockIdx.y * kTnTile;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_split;
  int64_t r_end = r_begin + rows_per_split;
  if (r_end > rows) r_end = rows;
  const int t = threadIdx.x;
  const int ta = t & 31, tb = t >> 5;  // outputs (a0+ta, b0 + tb + 8*q), q < 4
  double acc[4] = {0, 0, 0, 0};
  for (int64_t base = r_begin; base < r_end; base += kTnChunk) {
    for (int idx = t; idx < kTnChunk * kTnTile; idx += 256) {
      const int rr = idx / kTnTile, c = idx - rr * kTnTile;
      const int64_t row = base + rr;
      const bool okr = row < r_end;
      xs[rr][c] = (okr && a0 + c < cx) ? X[row * ldx + a0 + c] : T(0);
      ys[rr][c] = (okr && b0 + c < cy) ? Y[row * ldy + b0 + c] : T(0);
    }
    __syncthreads();
    if constexpr (kExact) {
#pragma unroll 4
      for (int rr = 0; rr < kTnChunk; ++rr) {
        const double xv = (double)xs[rr][ta];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(xv, (double)ys[rr][tb + 8 * q], acc[q]);
      }
    } else {
      T part[4] = {0, 0, 0, 0};
#pragma unroll 4
      for (int rr = 0; rr < kTnChunk; ++rr) {
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
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ta, b = b0 + tb + 8 * q;
    if (a < cx && b < cy && acc[q] != 0.0) atomicAdd(&C[(int64_t)a * ldc + b], acc[q]);
  }
}

// G[i, j] = sum_c A[i, c] A[j, c] for a short-wide A (m <= 128 rows): one warp per entry.
template <typename T>
__global__ void k_gram_rows(const T* __restrict__ A, int64_t lda, int m, int64_t n, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= (int64_t)m * m) return;
  const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
  if (j < i) return;
  double s = 0.0;
  for (int64_t c = lane; c < n; c += 32) s += (double)A[i * lda + c] * (double)A[j * lda + c];
  s = warp_sum(s);
  if (lane == 0) {
    G[(int64_t)i * m + j] = s;
    G[(int64_t)j * m + i] = s;
  }
}

// Symmetric eigendecomposition of the n x n FP64 matrix G (n <= kKmaxLimit + 1) in one CTA by
// one-sided Jacobi on G itself: G V = W with orthogonal columns, and for a positive
// semidefinite G the column norms ||W_j|| = lambda_j. With JT = float the eigenvalues are
// recomputed in FP64 as v_j^T G v_j / v_j^T v_j. Outputs: evals (n, descending), evecs (n x n
// row-major, column j = eigenvector of evals[j]), sweeps in *info.
// With vk_global set, the accumulated rotations live there (n x n, global memory) instead of in
// shared memory, so that FP64 fits for every n <= 129.
template <typename JT>
__global__ void k_sym_eig(const double* __restrict__ G, int n, double* __restrict__ evals,
                          double* __restrict__ evecs, int* info, JT* vk_global) {
  extern __shared__ __align__(16) unsigned char smem[];
  JT* W = reinterpret_cast<JT*>(smem);
  JT* VK = vk_global ? vk_global : W + (size_t)n * n;
  JT* tail = vk_global ? W + (size_t)n * n : VK + (size_t)n * n;
  double* ev = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tail) + 15) & ~uintptr_t(15));
  int* perm = reinterpret_cast<int*>(ev + n);
  int* flag = perm + n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    W[idx] = (JT)G[idx];
    const int c = idx / n, row = idx - c * n;
    VK[idx] = (row == c) ? JT(1) : JT(0);
  }
  const JT tol = (sizeof(JT) < sizeof(double) ? JT(0.5) : JT(2)) * Eps<JT>::v * sqrt((JT)n);
  const int sw = jacobi_cta<JT>(W, n, n, VK, n, n, tol, 60, flag);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < n; j += nw) {
    double lam;
    if (sizeof(JT) < sizeof(double)) {
      // Rayleigh quotient in FP64: v^T G v / v^T v.
      double num = 0.0, den = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double vi = (double)VK[(size_t)j * n + i];
        den += vi * vi;
        double gv = 0.0;
        for (int l = 0; l < n; ++l) gv += G[(size_t)i * n + l] * (double)VK[(size_t)j * n + l];
        num += vi * gv;
      }
      num = warp_sum(num);
      den = warp_sum(den);
      lam = den > 0 ? num / den : 0.0;
    } else {
      double s2 = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double w = (double)W[(size_t)j * n + i];
        s2 += w * w;
      }
      lam = sqrt(warp_sum(s2));
    }
    if (lane == 0) ev[j] = lam;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) perm[j] = j;  // NaN-safe: no slot left unset
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = ev[j];
    int rank = 0;
    for (int l = 0; l < n; ++l) rank += (ev[l] > sj) || (ev[l] == sj && l < j);
    perm[rank] = j;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int row = idx / n, jj = idx - row * n;
    const int j = perm[jj];
    evecs[idx] = (double)VK[(size_t)j * n + row];
  }
  for (int jj = threadIdx.x; jj < n; jj += blockDim.x) evals[jj] = ev[perm[jj]];
  if (threadIdx.x == 0) *info = sw;
}

// Converts the top-r eigenpairs into refresh factors: sig[j] = sqrt(max(lambda_j, 0)),
// R[c, j] = evecs[c, j] (as T, row stride ldr) and inv[j] = 1 / sig[j] (0 when sig[j] == 0).
// Also E_opt^2 = sum_{j >= r} max(lambda_j, 0) (the tail of the spectrum, Section 2.5).
template <typename T>
__global__ void k_eig_to_factors(const double* __restrict__ evals, const double* __restrict__ evecs, int n, int r,
                                 double* __restrict__ sig, double* __restrict__ inv, T* __restrict__ R, int ldr,
                                 double* __restrict__ tail) {
  for (int idx = threadIdx.x; idx < n * r; idx += blockDim.x) {
    const int c = idx / r, j = idx - c * r;
    R[(int64_t)c * ldr + j] = (T)evecs[(int64_t)c * n + j];
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    const double s = sqrt(fmax(evals[j], 0.0));
    sig[j] = s;
    inv[j] = s > 0.0 ? 1.0 / s : 0.0;
  }
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int j = r + threadIdx.x; j < n; j += 32) t += fmax(evals[j], 0.0);
    t = warp_sum(t);
    if (threadIdx.x == 0) *tail = t;
  }
}

// Out[c, j] = (T)(C[c, j] * scale[j]) (FP64 C, row-major).
template <typename T>
__global__ void k_scale_cast(const double* __restrict__ C, int64_t rows, int cols, int64_t ldc,
                             const double* __restrict__ scale, T* __restrict__ out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t c = idx / cols;
  const int j = (int)(idx - c * cols);
  out[c * ldo + j] = (T)(C[c * ldc + j] * (scale ? scale[j] : 1.0));
}

// E_inc^2 = ||A - U diag(sig) V^T||_F^2 accumulated in FP64 (Section 2.5, Eq. frob-errors):
// 64 x 64 tiles of A; U and V tiles (64 x r) in shared memory; 4 x 4 outputs per thread.
constexpr int kResTile = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_resid_norm(const T* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                    const T* __restrict__ U, const T* __restrict__ V, int ld,
                                                    const double* __restrict__ sig, const DevState* st,
                                                    double* __restrict__ out, int r_fixed = -1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = r_fixed >= 0 ? r_fixed : st->r;
  T* Us = reinterpret_cast<T*>(smem);       // [r][kResTile + 1], scaled by sigma
  T* Vs = Us + (size_t)r * (kResTile + 1);  // [r][kResTile + 1]
  __shared__ double red[8];
  const int64_t i0 = (int64_t)blockIdx.y * kResTile, j0 = (int64_t)blockIdx.x * kResTile;
  const int t = threadIdx.x;
  for (int idx = t; idx < kResTile * r; idx += 256) {
    const int rr = idx / r, c = idx - rr * r;
    const int64_t i = i0 + rr, j = j0 + rr;
    Us[c * (kResTile + 1) + rr] = i < m ? (T)((double)U[i * ld + c] * sig[c]) : T(0);
    Vs[c * (kResTile + 1) + rr] = j < n ? V[j * ld + c] : T(0);
  }
  __syncthreads();
  const int ty = t >> 4, tx = t & 15;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int c = 0; c < r; ++c) {
    T ua[4], vb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ua[a] = Us[c * (kResTile + 1) + ty * 4 + a];
#pragma unroll
    for (int b = 0; b < 4; ++b) vb[b] = Vs[c * (kResTile + 1) + tx * 4 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += ua[a] * vb[b];
  }
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + ty * 4 + a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + tx * 4 + b;
      if (i < m && j < n) {
        const double d = (double)A[i * lda + j] - (double)acc[a][b];
        s += d * d;
      }
    }
  }
  s = warp_sum(s);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    atomicAdd(out, tot);
  }
}

// Small helpers on r x r FP64 matrices (one CTA).
// E = B - C^T C (tr = 0) or E = B - C C^T (tr = 1); C is rc x cc row-major; E is q x q.
static __global__ void k_angle_matrix(const double* __restrict__ B, const double* __restrict__ C, int rc, int cc, int tr,
                               double* __restrict__ E) {
  const int q = tr ? rc : cc;
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int a = idx / q, b = idx - a * q;
    double s = 0.0;
    if (tr) {
      for (int l = 0; l < cc; ++l) s += C[a * cc + l] * C[b * cc + l];
    } else {
      for (int l = 0; l < rc; ++l) s += C[l * cc + a] * C[l * cc + b];
    }
    E[idx] = B[idx] - s;
  }
}

// NaN-propagating maximum: a NaN operand wins (fmax would drop it), so a factor holding NaN or
// Inf reports a NaN orthogonality error instead of a small one.
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || isnan(b)) ? b : a; }

// max |B - I| over an r x r FP64 matrix into *out (NaN if any entry is NaN).
static __global__ void k_max_offident(const double* __restrict__ B, int r, double* __restrict__ out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx - a * r;
    mx = nan_max(mx, fabs(B[idx] - (a == b ? 1.0 : 0.0)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = nan_max(m2, red[w]);
    *out = m2;
  }
}

// Cholesky B = L L^T (FP64, one CTA, r <= 128) and Rinv = (L^T)^{-1} written as T (r x r,
// row stride ldr), so that Q = X Rinv has orthonormal columns when B = X^T X (one Cholesky-QR
// pass). Sets *info = 1 when B is not numerically positive definite.
template <typename T>
__global__ void k_chol_rinv(const double* __restrict__ B, int r, double* __restrict__ Li, T* __restrict__ Rinv,
                            int ldr, int* info) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* L = reinterpret_cast<double*>(smem);  // r x r in shared memory; Li = L^{-1} in global scratch
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    L[idx] = B[idx];
    Li[idx] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      double d = L[j * r + j];
      for (int l = 0; l < j; ++l) d -= L[j * r + l] * L[j * r + l];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      L[j * r + j] = sqrt(d);
    }
    __syncthreads();
    const double djj = L[j * r + j];
    for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) {
      double s = L[i * r + j];
      for (int l = 0; l < j; ++l) s -= L[i * r + l] * L[j * r + l];
      L[i * r + j] = s / djj;
    }
    __syncthreads();
  }
  // Li = L^{-1}: column by column forward substitution, one thread per column.
  for (int col = threadIdx.x; col < r; col += blockDim.x) {
    for (int i = col; i < r; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int l = col; l < i; ++l) s -= L[i * r + l] * Li[l * r + col];
      Li[i * r + col] = s / L[i * r + i];
    }
  }
  __syncthreads();
  // Rinv = (L^T)^{-1} = (L^{-1})^T.
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx - a * r;
    Rinv[(int64_t)a * ldr + b] = (T)Li[b * r + a];
  }
  if (threadIdx.x == 0) *info = bad;
}

// Portfolio risk and covariance error from r x r Gram matrices (Section 5.3): g = V^T w,
// G1 = V^T V, and for the optimal factors gopt, G2 = Vopt^T Vopt, C = V^T Vopt. With
// S = V diag(s^2) V^T, w^T S w = sum_i s_i^2 g_i^2 and ||S1 - S2||_F^2 = sum s1_i^2 s1_j^2 G1_ij^2 +
// sum s2_i^2 s2_j^2 G2_ij^2 - 2 sum s1_i^2 s2_j^2 C_ij^2 (no orthonormality assumed). out = {vol,
// vol_opt, risk_error, cov_error, cov_norm}.
static __global__ void k_risk_finish(const double* __restrict__ s1, const double* __restrict__ s2,
                                     const double* __restrict__ g, const double* __restrict__ gopt,
                                     const double* __restrict__ G1, const double* __restrict__ G2,
                                     const double* __restrict__ Cx, int r, double inv_t1, int full,
                                     double* __restrict__ out) {
  __shared__ double red[5][8];
  double a = 0.0, b = 0.0, x = 0.0, v1 = 0.0, v2 = 0.0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int i = idx / r, j = idx - i * r;
    const double q1 = s1[i] * s1[i] * s1[j] * s1[j];
    a += q1 * G1[idx] * G1[idx];
    if (full) {
      b += s2[i] * s2[i] * s2[j] * s2[j] * G2[idx] * G2[idx];
      x += s1[i] * s1[i] * s2[j] * s2[j] * Cx[idx] * Cx[idx];
    }
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    v1 += s1[i] * s1[i] * g[i] * g[i];
    if (full) v2 += s2[i] * s2[i] * gopt[i] * gopt[i];
  }
  double vals[5] = {a, b, x, v1, v2};
  for (int q = 0; q < 5; ++q) {
    double v = vals[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 5; ++q)
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[q] += red[q][w];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[0] = sqrt(fmax(t[3], 0.0) * inv_t1);
    out[4] = sqrt(fmax(t[0], 0.0)) * inv_t1;
    if (full) {
      out[1] = sqrt(fmax(t[4], 0.0) * inv_t1);
      out[2] = fabs(out[0] - out[1]) / out[1];
      out[3] = sqrt(fmax(t[0] + t[1] - 2.0 * t[2], 0.0) / t[1]);
    } else {
      out[1] = out[2] = out[3] = nan;
    }
  }
}

// v[i] = value, i < n.
template <typename T>
__global__ void k_fill(T* __restrict__ v, int64_t n, T value) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = value;
}

}  // namespace isvd

namespace isvd {

// C (M x L, row stride ldc) = A (M x K, row stride lda) * B (K x L, row stride ldb), optionally
// C[:, :L0] copied from a given block instead (warm start). 64 x 64 output tile, K in chunks of
// 16, 256 threads with 4 x 4 outputs each, storage-type arithmetic with FP32/FP64 accumulation
// matching T. Used by the randomized refresh (Y = A Omega, Y = A Z).
constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16;
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn(const T* __restrict__ A, int64_t lda, int64_t M, int64_t K,
                                                 const T* __restrict__ B, int64_t ldb, int L, T* __restrict__ Cm,
                                                 int64_t ldc) {
  __shared__ T As[kGemmBK][kGemmBM + 4];
  __shared__ T Bs[kGemmBK][kGemmBN + 4];
  const int64_t i0 = (int64_t)blockIdx.x * kGemmBM;
  const int j0 = blockIdx.y * kGemmBN;
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t k0 = 0; k0 < K; k0 += kGemmBK) {
    for (int idx = t; idx < kGemmBM * kGemmBK; idx += 256) {
      const int rr = idx / kGemmBK, kk = idx - rr * kGemmBK;
      const int64_t row = i0 + rr, kc = k0 + kk;
      As[kk][rr] = (row < M && kc < K) ? A[row * lda + kc] : T(0);
    }
    for (int idx = t; idx < kGemmBK * kGemmBN; idx += 256) {
      const int kk = idx / kGemmBN, cc = idx - kk * kGemmBN;
      const int64_t kc = k0 + kk;
      Bs[kk][cc] = (kc < K && j0 + cc < L) ? B[kc * ldb + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmBK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[kk][ty * 4 + q];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t row = i0 + ty * 4 + x;
    if (row >= M) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int col = j0 + tx * 4 + y;
      if (col < L) Cm[row * ldc + col] = acc[x][y];
    }
  }
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014):
// the output function applied to seed + counter * golden gamma, as a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// sq[j] += sum over a slice of rows of B[row, j]^2 in FP64 (j < r; sq zeroed by the caller).
// Block (32 columns x 8 row lanes), grid (ceil(r / 32), row slices).
template <typename T>
__global__ void __launch_bounds__(256) k_col_sumsq(const T* __restrict__ B, int64_t rows, int64_t ldb, int r,
                                                   int64_t rows_per_split, double* __restrict__ sq) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r1 = r0 + rows_per_split < rows ? r0 + rows_per_split : rows;
  double acc = 0.0;
  if (j < r)
    for (int64_t row = r0 + warp; row < r1; row += 8) {
      const double v = (double)B[row * ldb + j];
      acc = fma(v, v, acc);
    }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && j < r) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    atomicAdd(&sq[j], t);
  }
}

// Singular values from column norms, descending: sig[jj] = sqrt(sq[perm[jj]]), inv[jj] = 1 / sig[jj]
// (0 for a zero column); ties keep the column order. One block.
static __global__ void k_sort_norms(const double* __restrict__ sq, int r, double* __restrict__ sig, int* __restrict__ perm,
                             double* __restrict__ inv) {
  for (int j = threadIdx.x; j < r; j += blockDim.x) {  // NaN-safe defaults: no slot left unset
    perm[j] = j;
    sig[j] = 0.0;
    inv[j] = 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    const double v = sq[j];
    int rank = 0;
    for (int l = 0; l < r; ++l) rank += (sq[l] > v) || (sq[l] == v && l < j);
    const double sv = sqrt(fmax(v, 0.0));
    perm[rank] = j;
    sig[rank] = sv;
    inv[rank] = sv > 0.0 ? 1.0 / sv : 0.0;
  }
}

// out[row, jj] = in[row, perm[jj]] * scale[jj] (scale optional) for jj < r <= kKmaxLimit + 1; one
// warp per row, staged through shared memory, so in and out may be the same array.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_permute_cols(const Tin* in, int64_t ldi, Tout* out, int64_t ldo, int64_t rows,
                                                      int r, const int* __restrict__ perm,
                                                      const double* __restrict__ scale) {
  __shared__ double buf[8][kKmaxLimit + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * 8 + warp;
  if (row >= rows) return;
  for (int c = lane; c < r; c += 32) buf[warp][c] = (double)in[row * ldi + c];
  __syncwarp();
  for (int jj = lane; jj < r; jj += 32) out[row * ldo + jj] = (Tout)(buf[warp][perm[jj]] * (scale ? scale[jj] : 1.0));
}

// Columns j < r of Q (rows x r, row stride ldq) whose singular value is at most rel * sig[0]
// (or zero) are overwritten with SplitMix64 uniforms in [-1, 1): there A v_j / sigma_j is
// dominated by rounding, so an orthonormal completion (the re-orthonormalisation that follows)
// replaces it.
template <typename T>
__global__ void k_seed_small_cols(T* __restrict__ Q, int64_t rows, int64_t ldq, const double* __restrict__ sig, int r,
                                  double rel, uint64_t seed) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * r) return;
  const int64_t row = idx / r;
  const int j = (int)(idx - row * r);
  const double s0 = sig[0];
  if (!(sig[j] <= rel * s0) && sig[j] > 0.0) return;
  const uint64_t h = splitmix64(seed ^ (uint64_t)idx);
  Q[row * ldq + j] = (T)((double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// Test matrix Omega (rows x l, row stride ld): columns [0, c0) copied from W (warm start with the
// current factor), columns [c0, l) standard normal by Box-Muller on two SplitMix64 uniforms.
template <typename T>
__global__ void k_fill_omega(T* __restrict__ Om, int64_t rows, int l, int64_t ld, const T* __restrict__ W, int64_t ldw,
                             int c0, uint64_t seed) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * l) return;
  const int64_t row = idx / l;
  const int c = (int)(idx - row * l);
  T v;
  if (c < c0) {
    v = W[row * ldw + c];
  } else {
    const uint64_t h1 = splitmix64(seed ^ (uint64_t)(2 * idx));
    const uint64_t h2 = splitmix64(seed ^ (uint64_t)(2 * idx + 1));
    const double u1 = ((double)(h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    v = (T)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
  Om[row * ld + c] = v;
}

// Out (rows x r, storage T, row stride ldo) = Zd (rows x l, FP64, row stride l) *
// Bd[:, :r] (l x l, FP64) * diag(scale). One thread per output element.
template <typename T>
__global__ void k_small_gemm_cast(const double* __restrict__ Zd, int64_t rows, int l, const double* __restrict__ Bd,
                                  int r, const double* __restrict__ scale, T* __restrict__ out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * r) return;
  const int64_t row = idx / r;
  const int j = (int)(idx - row * r);
  double s = 0.0;
  for (int a = 0; a < l; ++a) s += Zd[row * l + a] * Bd[(int64_t)a * l + j];
  out[row * ldo + j] = (T)(s * (scale ? scale[j] : 1.0));
}

// Adds shift to the diagonal of an r x r FP64 matrix (shifted Cholesky-QR first pass).
static __global__ void k_add_diag(double* __restrict__ B, int r, double rel_shift) {
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += B[i * r + i];
    tr = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) B[i * r + i] += rel_shift * tr + 1e-300;
}

}  // namespace isvd
