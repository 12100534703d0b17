// Batched updates of many independent streams (FP32 bulk, FP64-class core): one CTA performs one
// whole update of one stream (Section 2.2 row/column append or Section 2.3 entry update) -
// projection with CGS2, core SVD in shared memory, rotations of that stream's U and V, dense-A and
// N_t bookkeeping - so one launch advances every stream of a tick by one update.
#pragma once

#include "core_fast.cuh"
#include "core_svd.cuh"
#include "isvd_common.cuh"

namespace isvd {

// Rows per TMA box of the pools' row tensor maps over U and V (row width = the rank bucket).
constexpr int kRowBoxRows = 32;

// One update of one stream, as the fused kernel reads it.
struct PoolOp {
  float* U;            // m x r (row stride ld)
  float* V;            // n x r
  float* A;            // m x n (row stride lda)
  DevState* st;        // the stream's device state
  double* sig;         // the stream's singular values
  const float* x;      // payload: n values (row append) or m values (column append)
  int64_t m, n, lda;   // shape before the update
  int64_t i, j;        // entry position
  double delta;        // entry increment
  double tol_rel;      // rank test threshold
  int32_t ld;          // row stride of U and V
  int32_t kind;        // kRow, kCol, kEntry
  int32_t sid;         // pool stream id (completion records)
  int32_t pad;
  int64_t seq;         // pool-wide sequence number of the op (completion records)
  float* z1;           // per projection-side row: x - P p1 after the first projection pass (written by
                       // the warp kernel of an append, read by its rotation for z_hat)
};

// A stream whose adaptive-rank check is due (Eq. evr-rank-rule read as a growth rule).
struct PoolRankOp {
  DevState* st;
  const double* sig;
  int32_t kcap;  // the stream's rank capacity (its bucket, at most the pool's k_max)
  int32_t pad;
};

// One completion record (layout of isvd_completion in include/isvd.h).
struct PoolCompletion {
  int64_t seq;
  int32_t stream, kind, status, r;
  double rho, sigma_max;
  uint64_t done_ns;
};



__host__ __device__ constexpr int pool_threads(int kb) {
  return kb <= 8 ? 128 : kb <= 16 ? 256 : kb <= 32 ? 288 : 544;
}
// Rank bucket of the fused kernel for a stream of working-rank capacity k.
// Bucket 128 has no batched kernel: its updates run through the single-stream kernels, in order.
__host__ __device__ constexpr int pool_bucket(int k) {
  return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128;
}

template <int KB>
__host__ __device__ inline size_t pool_smem_bytes() {
  size_t core = core_fast_smem_bytes<float>(KB);
  const size_t jac = core_smem_bytes<float>(KB);
  if (jac > core) core = jac;
  const size_t outs = (size_t)2 * (KB + 1) * KB * sizeof(float);          // U_K, V_K
  const size_t red = (size_t)(pool_threads(KB) / 32) * (KB + 4) * sizeof(double);
  const size_t vecs = (size_t)6 * (KB + 2) * sizeof(double);               // p1, p2, a, b, ...
  return core + outs + red + vecs + 256;
}

// Sum over the CTA's warps of per-warp column partials red[w][c] -> out[c] (FP64), c < cols.
__device__ __forceinline__ void pool_reduce_cols(const double* red, int stride, int cols, double* out) {
  const int nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * stride + c];
    out[c] = s;
  }
}

// p_c = sum_rows X[row, c] * y[row] over rows (warps own rows, lanes own columns), accumulated
// in FP32 over runs of 8 rows and then in FP64; also returns sum y^2 (FP64) in *ysq if given.
template <int KB>
__device__ void pool_project(const float* X, int ld, int64_t rows, const float* y, int r, double* red, double* out,
                             double* ysq_out) {
  constexpr int Q = (KB + 31) / 32;
  constexpr int U4 = 4;  // rows in flight per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc[Q];
  float accs[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    acc[q] = 0.0;
    accs[q] = 0.f;
  }
  float ysq = 0.f;
  double ysqd = 0.0;
  int run = 0;
  for (int64_t row0 = warp; row0 < rows; row0 += (int64_t)U4 * nw) {
    float yv[U4], xv[U4][Q];
#pragma unroll
    for (int u = 0; u < U4; ++u) {  // issue every load of the group first
      const int64_t row = row0 + (int64_t)u * nw;
      const bool ok = row < rows;
      yv[u] = ok ? y[row] : 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int c = lane + 32 * q;
        xv[u][q] = (ok && c < r) ? X[row * (int64_t)ld + c] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U4; ++u) {
#pragma unroll
      for (int q = 0; q < Q; ++q) accs[q] = fmaf(xv[u][q], yv[u], accs[q]);
      ysq = fmaf(yv[u], yv[u], ysq);
    }
    if (++run == 2) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        acc[q] += (double)accs[q];
        accs[q] = 0.f;
      }
      ysqd += (double)ysq;
      ysq = 0.f;
      run = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    acc[q] += (double)accs[q];
    const int c = lane + 32 * q;
    if (c < KB) red[warp * (KB + 4) + c] = acc[q];
  }
  ysqd += (double)ysq;
  if (lane == 0) red[warp * (KB + 4) + KB] = ysqd;  // lanes hold identical y^2 sums
  __syncthreads();
  pool_reduce_cols(red, KB + 4, r, out);
  if (ysq_out && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * (KB + 4) + KB];
    *ysq_out = s;
  }
  __syncthreads();
}

// Rotation of one side in place, one thread per row (R broadcast from shared memory):
//   Y[row, :k_out] = X[row, :c_in] R[:c_in, :k_out] (+ zhat_row R[c_in, :] when zsrc != nullptr,
//   zhat_row = (zsrc[row] - X[row, :c_in] . p2) / rho), and the new row Y[rows, :] = R[c_in, :].
template <int KB>
__device__ void pool_rotate(float* X, int ld, int64_t rows, const float* R, int ldr, int c_in, int k_out,
                            const float* zsrc, const float* p2f, float inv_rho, bool newrow) {
  constexpr int HALF = KB <= 16 ? KB : 16;  // outputs per pass (bounds the live registers)
  for (int64_t row = threadIdx.x; row < rows; row += blockDim.x) {
    float* xr = X + row * (int64_t)ld;
    float xv[KB];
#pragma unroll
    for (int c4 = 0; c4 < KB; c4 += 4) {
      if (c4 < c_in) {
        const float4 v = *reinterpret_cast<const float4*>(xr + c4);
        xv[c4] = v.x;
        xv[c4 + 1] = v.y;
        xv[c4 + 2] = v.z;
        xv[c4 + 3] = v.w;
      } else {
        xv[c4] = xv[c4 + 1] = xv[c4 + 2] = xv[c4 + 3] = 0.f;
      }
    }
    float zh = 0.f;
    if (zsrc) {
      float d = 0.f;
#pragma unroll
      for (int c = 0; c < KB; ++c)
        if (c < c_in) d = fmaf(xv[c], p2f[c], d);
      zh = (zsrc[row] - d) * inv_rho;
    }
#pragma unroll
    for (int h0 = 0; h0 < KB; h0 += HALF) {
      float o[HALF];
#pragma unroll
      for (int jj = 0; jj < HALF; ++jj) o[jj] = 0.f;
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        if (c < c_in) {
          const float* rr = R + (size_t)c * ldr + h0;
#pragma unroll
          for (int jj = 0; jj < HALF; ++jj) o[jj] = fmaf(xv[c], rr[jj], o[jj]);
        }
      }
      if (zsrc) {
        const float* rr = R + (size_t)c_in * ldr + h0;
#pragma unroll
        for (int jj = 0; jj < HALF; ++jj) o[jj] = fmaf(zh, rr[jj], o[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < HALF; jj += 4) {
        if (h0 + jj < k_out) {
          if (h0 + jj + 3 < k_out) {
            *reinterpret_cast<float4*>(xr + h0 + jj) = make_float4(o[jj], o[jj + 1], o[jj + 2], o[jj + 3]);
          } else {
            for (int e = 0; e < 4 && h0 + jj + e < k_out; ++e) xr[h0 + jj + e] = o[jj + e];
          }
        }
      }
    }
  }
  if (newrow) {
    for (int jj = threadIdx.x; jj < k_out; jj += blockDim.x) X[rows * (int64_t)ld + jj] = R[(size_t)c_in * ldr + jj];
  }
}

// Resident CTAs per SM the register budget is shaped for.
__host__ __device__ constexpr int pool_min_blocks(int kb) { return kb <= 8 ? 6 : kb <= 16 ? 4 : kb <= 32 ? 3 : 1; }

// One whole update of one stream by the calling CTA (blockDim = pool_threads(KB), dynamic shared
// memory pool_smem_bytes<KB>()).
template <int KB>
__device__ void pool_tick_body(const PoolOp& op) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int t = threadIdx.x;
  const int nw = blockDim.x >> 5;
  size_t core_b = core_fast_smem_bytes<float>(KB);
  if (core_smem_bytes<float>(KB) > core_b) core_b = core_smem_bytes<float>(KB);
  unsigned char* core_smem = smem;
  float* UKs = reinterpret_cast<float*>(smem + core_b);
  float* VKs = UKs + (KB + 1) * KB;
  // z1 rows of an append's projection side: the op's residual buffer in global memory (any length)
  float* zbuf = op.z1;
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(VKs + (KB + 1) * KB) + 15) & ~uintptr_t(15));
  double* p1 = red + (size_t)nw * (KB + 4);
  double* p2 = p1 + (KB + 2);
  double* av = p2 + (KB + 2);
  double* bv = av + (KB + 2);
  float* p2f = reinterpret_cast<float*>(bv + (KB + 2));
  __shared__ double s_sc[4];
  __shared__ int s_sweeps;
  DevState* st = op.st;
  const int r = st->r;
  const int kind = op.kind;
  ISVD_STAMP(16);
  // Projection side: V for a row append, U for a column append.
  float* Xp = kind == kRow ? op.V : op.U;
  const int64_t prow = kind == kRow ? op.n : op.m;
  if (kind != kEntry) {
    // Store the new row / column of A.
    for (int64_t row = t; row < prow; row += blockDim.x) {
      const float v = op.x[row];
      if (kind == kRow) op.A[op.m * op.lda + row] = v;
      else op.A[row * op.lda + op.n] = v;
    }
    // Pass 1: p1 = X^T x, ||x||^2.
    pool_project<KB>(Xp, op.ld, prow, op.x, r, red, p1, &s_sc[0]);
    ISVD_STAMP(17);
    // Pass 2: z1 = x - X p1 per row (float-float, one thread per row) into op.z1, ||z1||^2.
    float* p1h = reinterpret_cast<float*>(red);  // p1 as float pairs (red is free now)
    float* p1l = p1h + (KB + 2);
    for (int c = t; c < r; c += blockDim.x) {
      const ff q = ff_of(p1[c]);
      p1h[c] = q.hi;
      p1l[c] = q.lo;
    }
    __syncthreads();
    ff zn{0.f, 0.f};
    for (int64_t row = t; row < prow; row += blockDim.x) {
      const float* xr = Xp + row * (int64_t)op.ld;
      float xv[KB];  // the row, loaded with vector loads before any arithmetic
#pragma unroll
      for (int c4 = 0; c4 < KB; c4 += 4) {
        if (c4 < r) {
          const float4 v = *reinterpret_cast<const float4*>(xr + c4);
          xv[c4] = v.x;
          xv[c4 + 1] = v.y;
          xv[c4 + 2] = v.z;
          xv[c4 + 3] = v.w;
        } else {
          xv[c4] = xv[c4 + 1] = xv[c4 + 2] = xv[c4 + 3] = 0.f;
        }
      }
      ff s{op.x[row], 0.f};
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        if (c < r) {
          ff pr = two_prod(xv[c], p1h[c]);
          pr.lo = fmaf(xv[c], p1l[c], pr.lo);
          s = ff_add(s, ff{-pr.hi, -pr.lo});
        }
      }
      zbuf[row] = s.hi + s.lo;
      zn = ff_add(zn, ff_sqr(s));
    }
    zn = ff_group_sum<32>(zn);
    __syncthreads();
    double* zred = reinterpret_cast<double*>(p2f);  // one slot per warp (p2f is unused until pass 3)
    if ((t & 31) == 0) zred[t >> 5] = (double)zn.hi + (double)zn.lo;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += zred[w];
      s_sc[1] = s;
    }
    __syncthreads();
    ISVD_STAMP(18);
    // Pass 3 (CGS2): p2 = X^T z1; p = p1 + p2; rho^2 = ||z1||^2 - ||p2||^2.
    pool_project<KB>(Xp, op.ld, prow, zbuf, r, red, p2, nullptr);
    if (t < 32) {
      double pn = 0.0;
      for (int c = t; c < r; c += 32) {
        pn += p2[c] * p2[c];
        p2f[c] = (float)p2[c];
        p1[c] += p2[c];
      }
      pn = warp_sum(pn);
      if (t == 0) {
        const double xn2 = s_sc[0];
        const double rho2 = s_sc[1] - pn;
        const double rho = sqrt(fmax(rho2, 0.0));
        const double xnorm = sqrt(xn2);
        if (!isfinite(xn2) || !isfinite(rho2)) atomicOr(&st->status, kStNonFinite);
        st->rho = rho;
        st->grew = rho > op.tol_rel * xnorm ? 1 : 0;
        st->novelty = xnorm > 0.0 ? rho / xnorm : 0.0;
        st->xnorm2 = xn2;
        st->N += xn2;
        s_sc[2] = rho;
      }
    }
    __syncthreads();
  } else {
    for (int c = t; c < r; c += blockDim.x) {
      av[c] = (double)op.U[op.i * (int64_t)op.ld + c];
      bv[c] = (double)op.V[op.j * (int64_t)op.ld + c];
    }
    if (t == 0) {
      float* aij = op.A + op.i * op.lda + op.j;
      const double old = (double)*aij;
      st->N += 2.0 * op.delta * old + op.delta * op.delta;
      *aij = (float)(old + op.delta);
    }
    __syncthreads();
  }
  ISVD_STAMP(19);
  // Core SVD into shared memory.
  CoreIn in;
  in.kind = kind;
  in.r = r;
  in.grew = kind == kEntry ? 0 : st->grew;
  in.kt = st->k;
  in.sig = op.sig;
  in.p = p1;
  in.rho = kind == kEntry ? 0.0 : st->rho;
  in.a = av;
  in.b = bv;
  in.delta = op.delta;
  int it = 0;
  int k_out = core_fast_cta<float, KB>(in, core_smem, UKs, VKs, KB, op.sig, &it);
  if (t == 0) s_sweeps = 100 + it;
  __syncthreads();
  if (k_out < 0) k_out = core_svd_cta<float, float>(in, core_smem, UKs, VKs, KB, op.sig, &s_sweeps);
  __syncthreads();
  const bool grew = kind != kEntry && in.grew;
  __shared__ float s_inv_rho;
  if (t == 0) s_inv_rho = grew ? (float)(1.0 / st->rho) : 0.f;
  __syncthreads();
  const float inv_rho = s_inv_rho;
  ISVD_STAMP(20);
  // Rotations (Step 3): row append U <- [U; 0] U_K + new row, V <- V V_K + z_hat V_K[r];
  // column append swaps the roles; entry: U <- U U_K, V <- V V_K.
  if (kind == kRow) {
    pool_rotate<KB>(op.U, op.ld, op.m, UKs, KB, r, k_out, nullptr, nullptr, 0.f, true);
    ISVD_STAMP(21);
    pool_rotate<KB>(op.V, op.ld, op.n, VKs, KB, r, k_out, grew ? zbuf : nullptr, p2f, inv_rho, false);
  } else if (kind == kCol) {
    pool_rotate<KB>(op.U, op.ld, op.m, VKs, KB, r, k_out, grew ? zbuf : nullptr, p2f, inv_rho, false);
    pool_rotate<KB>(op.V, op.ld, op.n, UKs, KB, r, k_out, nullptr, nullptr, 0.f, true);
  } else {
    pool_rotate<KB>(op.U, op.ld, op.m, UKs, KB, r, k_out, nullptr, nullptr, 0.f, false);
    pool_rotate<KB>(op.V, op.ld, op.n, VKs, KB, r, k_out, nullptr, nullptr, 0.f, false);
  }
  __syncthreads();
  ISVD_STAMP(22);
  if (t == 0) {
    st->r_in = r;
    st->k_out = k_out;
    st->r = k_out;
    st->sweeps = s_sweeps;
    if (s_sweeps < 0) atomicOr(&st->status, kStNotConv);
    if (kind == kEntry) st->ang_u = st->ang_v = 0.0;
    else append_signals<float>(st, kind == kRow, UKs, VKs, KB, r, k_out, grew, in.kt);
  }
}

template <int KB>
__global__ void __launch_bounds__(pool_threads(KB), pool_min_blocks(KB)) k_pool_tick(const PoolOp* __restrict__ ops) {
  const PoolOp op = ops[blockIdx.x];
  pool_tick_body<KB>(op);
}

// The updates listed in retry[0 .. *retry_n) (indices into ops), one at a time per block. Rare, so
// it is not shaped for occupancy (one block per SM, registers unconstrained).
template <int KB>
__global__ void __launch_bounds__(pool_threads(KB), 1)
    k_pool_retry(const PoolOp* __restrict__ ops, const int* __restrict__ retry, const int* __restrict__ retry_n) {
  const int n = *retry_n;
#pragma unroll 1
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const PoolOp op = ops[retry[b]];
    pool_tick_body<KB>(op);
    __syncthreads();
  }
}

}  // namespace isvd
