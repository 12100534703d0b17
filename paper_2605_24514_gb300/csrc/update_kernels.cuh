// Per-update kernels of one stream: projection and residual (Section 2.2 Step 1, Eq.
// (row-residual)), the core SVD launch (Step 2 / Section 2.3) and the rotations of the tall
// factors (Step 3: U' = blkdiag(U, 1) U_K, V' = [V z_hat] V_K; entry: U' = U U_K, V' = V V_K).
#pragma once

#include "core_fast.cuh"
#include "core_svd.cuh"
#include "isvd_common.cuh"

namespace isvd {

constexpr int kProjThreads = 256;
constexpr int kProjWarps = kProjThreads / 32;
constexpr int kPartStride = kKmaxLimit + 4;  // doubles per block partial (k values + extras)

// Last-block-done reduction helper: returns true in the block that arrives last.
__device__ __forceinline__ bool last_block_arrives(unsigned int* counter, bool* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int v = atomicAdd(counter, 1u);
    *s_last = (v == gridDim.x - 1);
  }
  __syncthreads();
  return *s_last;
}

// Pass 1: p = X^T x and ||x||^2 (X = V for a row append, X = U for a column append), and the
// copy of x into the stored matrix A (dst[row * dst_stride] = x[row]). Warps own rows; lanes own
// columns c = lane + 32 q, so each row is one coalesced read and no shuffles are needed.
// Products are summed in the storage type over runs of 8 rows, then in FP64.
template <typename T>
__global__ void __launch_bounds__(kProjThreads) k_proj1(const T* __restrict__ X, int ld, int64_t rows,
                                                        const T* __restrict__ x, DevState* st,
                                                        double* __restrict__ part, double* __restrict__ p_out,
                                                        T* __restrict__ dst, int64_t dst_stride) {
  __shared__ double red[kProjWarps][kPartStride];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = st->r;
  const int nq = (r + 31) >> 5;
  double acc[4] = {0, 0, 0, 0};
  T acc_s[4] = {0, 0, 0, 0};
  double xn = 0.0;
  int run = 0;
  const int64_t gw = (int64_t)blockIdx.x * kProjWarps + warp;
  const int64_t tw = (int64_t)gridDim.x * kProjWarps;
  for (int64_t row = gw; row < rows; row += tw) {
    const T xv = x[row];
    if (lane == 0) {
      xn += (double)xv * (double)xv;
      if (dst) dst[row * dst_stride] = xv;
    }
    const T* xr = X + row * (int64_t)ld;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (q < nq && c < r) acc_s[q] += xr[c] * xv;
    }
    if (++run == 8) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += (double)acc_s[q];
        acc_s[q] = T(0);
      }
      run = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc[q] += (double)acc_s[q];
    const int c = lane + 32 * q;
    if (c < kKmaxLimit) red[warp][c] = acc[q];
  }
  xn = warp_sum(xn);
  if (lane == 0) red[warp][kKmaxLimit] = xn;
  __syncthreads();
  double* mypart = part + (size_t)blockIdx.x * kPartStride;
  for (int c = threadIdx.x; c <= kKmaxLimit; c += blockDim.x) {
    if (c < r || c == kKmaxLimit) {
      double s = 0.0;
      for (int w = 0; w < kProjWarps; ++w) s += red[w][c];
      mypart[c] = s;
    }
  }
  if (last_block_arrives(&st->counter, &s_last)) {
    for (int c = threadIdx.x; c <= kKmaxLimit; c += blockDim.x) {
      if (c < r || c == kKmaxLimit) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)part)[(size_t)b * kPartStride + c];
        if (c < r) p_out[c] = s;
        else st->xnorm2 = s;
      }
    }
    if (threadIdx.x == 0) st->counter = 0;
  }
}

// Pass 2: z = x - X p (FP64 accumulation per row), ||z||^2 and, with CGS2 (FP32 storage), the
// second projection p2 = X^T z. The last block finishes rho and the rank test:
//   rho^2 = ||z||^2 - ||p2||^2 (CGS2) or ||z||^2, p <- p + p2,
//   grew = rho > tol_rel * ||x||  (Section 2.2: z_hat = z / rho only when rho > tol),
//   N_t += ||x||^2 (Section 2.4), novelty = rho / ||x|| (Section 3.3).
template <typename T, bool CGS2>
__global__ void __launch_bounds__(kProjThreads) k_proj2(const T* __restrict__ X, int ld, int64_t rows,
                                                        const T* __restrict__ x, DevState* st,
                                                        double* __restrict__ part, double* __restrict__ p,
                                                        double tol_rel) {
  __shared__ double red[kProjWarps][kPartStride];
  __shared__ double ps[kKmaxLimit];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = st->r;
  const int nq = (r + 31) >> 5;
  for (int c = threadIdx.x; c < r; c += blockDim.x) ps[c] = p[c];
  __syncthreads();
  double acc[4] = {0, 0, 0, 0};
  T acc_s[4] = {0, 0, 0, 0};
  double zn = 0.0;
  int run = 0;
  const int64_t gw = (int64_t)blockIdx.x * kProjWarps + warp;
  const int64_t tw = (int64_t)gridDim.x * kProjWarps;
  for (int64_t row = gw; row < rows; row += tw) {
    const T* xr = X + row * (int64_t)ld;
    T xv_c[4];
    double d = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      xv_c[q] = (q < nq && c < r) ? xr[c] : T(0);
      if (q < nq && c < r) d += (double)xv_c[q] * ps[c];
    }
    d = warp_sum(d);
    const double z = (double)x[row] - d;
    if (lane == 0) zn += z * z;
    if (CGS2) {
      const T zt = (T)z;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc_s[q] += xv_c[q] * zt;
      if (++run == 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] += (double)acc_s[q];
          acc_s[q] = T(0);
        }
        run = 0;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc[q] += (double)acc_s[q];
    const int c = lane + 32 * q;
    if (c < kKmaxLimit) red[warp][c] = acc[q];
  }
  zn = warp_sum(zn);
  if (lane == 0) red[warp][kKmaxLimit] = zn;
  __syncthreads();
  double* mypart = part + (size_t)blockIdx.x * kPartStride;
  for (int c = threadIdx.x; c <= kKmaxLimit; c += blockDim.x) {
    if ((CGS2 && c < r) || c == kKmaxLimit) {
      double s = 0.0;
      for (int w = 0; w < kProjWarps; ++w) s += red[w][c];
      mypart[c] = s;
    }
  }
  if (last_block_arrives(&st->counter, &s_last)) {
    __shared__ double sp2[kKmaxLimit + 1];
    for (int c = threadIdx.x; c <= kKmaxLimit; c += blockDim.x) {
      if ((CGS2 && c < r) || c == kKmaxLimit) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)part)[(size_t)b * kPartStride + c];
        sp2[c] = s;
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      double p2n = 0.0;
      if (CGS2) {
        for (int c = threadIdx.x; c < r; c += 32) {
          p2n += sp2[c] * sp2[c];
          p[c] = ps[c] + sp2[c];
        }
      }
      p2n = warp_sum(p2n);
      if (threadIdx.x == 0) {
        const double rho2 = sp2[kKmaxLimit] - p2n;
        const double rho = sqrt(fmax(rho2, 0.0));
        const double xn2 = st->xnorm2;
        const double xnorm = sqrt(xn2);
        if (!isfinite(xn2) || !isfinite(rho2)) atomicOr(&st->status, kStNonFinite);
        st->rho = rho;
        st->grew = rho > tol_rel * xnorm ? 1 : 0;
        st->novelty = xnorm > 0.0 ? rho / xnorm : 0.0;
        st->N += xn2;
        st->counter = 0;
      }
    }
  }
}

// Core SVD of one update (single CTA). For an entry update it first gathers s_u = U[i, :] and
// s_v = V[j, :] and applies A_ij += delta with N_t += 2 delta A_ij + delta^2 (Section 2.5).
// Threads of the core kernel: up to 1024 for rank buckets <= 64 (so one secular-solver round covers
// every root), 512 for the 128 bucket (register budget).
__host__ __device__ constexpr int core_max_threads(int kb) { return kb <= 64 ? 1024 : 512; }

// Deferred rotations (RU != nullptr, kEntry only): U and V are held as U0 R_U and V0 R_V with
// U0, V0 of defer_rows columns, so the gathered rows are U0[i, :] R_U and V0[j, :] R_V, summed in T
// by four lanes per output.
// kEntryX (the rank-increasing form): e_i = U p + alpha P, e_j = V q + beta Q with p = U[i, :],
// q = V[j, :], alpha^2 = 1 - ||p||^2 and beta^2 = 1 - ||q||^2 (unit vectors against orthonormal
// bases; a residual norm <= tol_rel counts as zero); the core is the (r+1) x (r+1) diagonal-plus-
// rank-one matrix diag(sigma, 0) + delta [p; alpha] [q; beta]^T. px receives p, q (stride
// kKmaxLimit + 2) and alpha, beta (at 2 (kKmaxLimit + 2) and + 1) for the rotations.
template <typename T, typename JT, int KB>
__global__ void __launch_bounds__(core_max_threads(KB)) k_core(int kind, DevState* st, double* sig, const double* __restrict__ p, const T* U,
                       const T* V, int ld, int64_t ei, int64_t ej, double delta, T* A, int64_t lda, T* UK,
                       T* VKo, int ldo, double* px, double tol_rel, const T* RU, const T* RV, int ldr,
                       float* gq) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* ab = reinterpret_cast<double*>(smem);
  unsigned char* core_smem = smem + (size_t)2 * (kKmaxLimit + 1) * sizeof(double);
  const int r = st->r;
  const bool entry = kind == kEntry || kind == kEntryX;
  if (entry && RU) {
    const int dr = st->defer_rows;
    const int part = threadIdx.x & 3;
    for (int base = 0; base < 2 * r; base += (int)blockDim.x >> 2) {
      const int o = base + ((int)threadIdx.x >> 2);
      const bool side_v = o >= r;
      const int c = side_v ? o - r : o;
      T s = T(0);
      if (o < 2 * r) {
        const T* row = side_v ? V + ej * (int64_t)ld : U + ei * (int64_t)ld;
        const T* R = side_v ? RV : RU;
        for (int l = part; l < dr; l += 4) s += row[l] * R[(int64_t)l * ldr + c];
      }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (o < 2 * r && part == 0) ab[(side_v ? kKmaxLimit + 1 : 0) + c] = (double)s;
    }
  } else if (entry) {
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      ab[c] = (double)U[ei * (int64_t)ld + c];
      ab[kKmaxLimit + 1 + c] = (double)V[ej * (int64_t)ld + c];
    }
  }
  if (entry) {
    if (threadIdx.x == 0) {
      T* aij = A + ei * lda + ej;
      const double old = (double)*aij;
      st->N += 2.0 * delta * old + delta * delta;
      *aij = (T)(old + delta);
    }
  }
  __syncthreads();
  bool grew_u = false, grew_v = false;
  if (kind == kEntryX) {
    // Residual norms of e_i and e_j (FP64 sums of the gathered rows), the extended core vectors.
    __shared__ double s_ab[2];
    if (threadIdx.x < 32) {
      double su = 0.0, sv = 0.0;
      for (int c = threadIdx.x; c < r; c += 32) {
        su += ab[c] * ab[c];
        sv += ab[kKmaxLimit + 1 + c] * ab[kKmaxLimit + 1 + c];
      }
      su = warp_sum(su);
      sv = warp_sum(sv);
      if (threadIdx.x == 0) {
        const double al = sqrt(fmax(1.0 - su, 0.0)), be = sqrt(fmax(1.0 - sv, 0.0));
        s_ab[0] = al > tol_rel ? al : 0.0;
        s_ab[1] = be > tol_rel ? be : 0.0;
      }
    }
    __syncthreads();
    grew_u = s_ab[0] > 0.0;
    grew_v = s_ab[1] > 0.0;
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      px[c] = ab[c];
      px[kKmaxLimit + 2 + c] = ab[kKmaxLimit + 1 + c];
    }
    if (threadIdx.x == 0) {
      ab[r] = s_ab[0];
      ab[kKmaxLimit + 1 + r] = s_ab[1];
      px[2 * (kKmaxLimit + 2)] = s_ab[0];
      px[2 * (kKmaxLimit + 2) + 1] = s_ab[1];
      sig[r] = 0.0;  // the core's extra pole
    }
    __syncthreads();
  }
  CoreIn in;
  in.kind = entry ? kEntry : kind;
  in.r = kind == kEntryX ? r + 1 : r;
  in.grew = entry ? 0 : st->grew;
  in.kt = st->k;
  in.sig = sig;
  in.p = p;
  in.rho = st->rho;
  in.a = ab;
  in.b = ab + kKmaxLimit + 1;
  in.delta = delta;
  __shared__ int s_sweeps;
  int k_out = -1;
  if (sizeof(JT) < sizeof(double) && KB <= kFastCoreMaxKB && kind != kEntryX) {
    // Secular-equation core (O(k^2) roots + verification); -1 means "use the Jacobi path".
    int it = 0;
    k_out = core_fast_cta<T, KB>(in, core_smem, UK, VKo, ldo, sig, &it, gq);
    if (threadIdx.x == 0) s_sweeps = 100 + it;
    __syncthreads();
  }
  if (k_out < 0) k_out = core_svd_cta<T, JT>(in, core_smem, UK, VKo, ldo, sig, &s_sweeps);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->r_in = r;
    st->k_out = k_out;
    st->r = k_out;
    st->sweeps = s_sweeps;
    if (s_sweeps < 0) atomicOr(&st->status, kStNotConv);
    if (kind == kEntry) {
      st->ang_u = st->ang_v = 0.0;
    } else if (kind == kEntryX) {
      // both sides may have gained a direction: the angles from row r of U_K and of V_K
      T cu = T(0), cv = T(0);
      if (k_out <= r)
        for (int j = 0; j < k_out; ++j) {
          const T a = grew_u ? UK[(int64_t)r * ldo + j] : T(0), b = grew_v ? VKo[(int64_t)r * ldo + j] : T(0);
          cu += a * a;
          cv += b * b;
        }
      st->ang_u = (double)asin(sqrt(cu) < T(1) ? sqrt(cu) : T(1));
      st->ang_v = (double)asin(sqrt(cv) < T(1) ? sqrt(cv) : T(1));
    } else {
      append_signals<T>(st, kind == kRow, UK, VKo, ldo, r, k_out, in.grew != 0, in.kt);
    }
  }
}

// Tall-skinny product Y[row, :k_out] = X[row, :c_in] R[:c_in, :k_out] (+ z_row R[c_in, :] for the
// z_hat column), one 64-row tile per block, R staged in shared memory. X may equal Y (rows are
// independent and each tile is read completely before it is written). Used for the rotations of
// Step 3 and for the refresh's U = A V S^-1.
struct RotSide {
  const void* X;     // input rows
  void* Y;           // output rows (may equal X)
  int64_t rows;      // existing rows
  int64_t ldx, ldy;  // row strides
  const void* R;     // c_in (+1) x k_out, row stride ldr
  int64_t ldr;
  int c_in;          // inner dimension (excluding the z_hat row); -1: take st->r_in, -2: st->defer_rows
  int zhat;          // add z_row * R[c_in, :] with z_row = (xz[row] - X[row, :] p) / rho
  int newrow;        // also write Y[rows, :] = R[c_in, :]
  int k_out;         // -1: take st->k_out, -2: st->r
  const double* colscale;  // optional per-output-column scale (1 / sigma for U = A V S^-1)
  // Residual direction of a unit vector e_zunit (rank-increasing entry update): when zrho is set,
  // z_row = ([row == zunit] - X[row, :] . zp) / *zrho replaces the append's (xz[row] - X p) / rho,
  // and the column is used only when *zrho > 0.
  const double* zp;
  const double* zrho;
  int64_t zunit;
};

constexpr int kRotRows = 64;
constexpr int kRotThreads = 256;

template <typename T, int KB>
__host__ __device__ inline size_t rot_smem_bytes() {
  return (size_t)KB * (kRotRows + 1) * sizeof(T) + (size_t)(KB + 1) * KB * sizeof(T) + kRotRows * sizeof(T);
}

template <typename T, int KB>
__global__ void __launch_bounds__(kRotThreads) k_rotate(RotSide s0, RotSide s1, int tiles0, const T* __restrict__ xz,
                                                        const double* __restrict__ p, const DevState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CPT = KB / 16;
  T* Xs = reinterpret_cast<T*>(smem);                 // [KB][kRotRows + 1]
  T* Rs = Xs + KB * (kRotRows + 1);                   // [KB + 1][KB]
  T* zs = Rs + (KB + 1) * KB;                         // [kRotRows]
  const bool first = (int)blockIdx.x < tiles0;
  const RotSide& sd = first ? s0 : s1;
  const int64_t tile = first ? blockIdx.x : blockIdx.x - tiles0;
  const int c_in = sd.c_in >= 0 ? sd.c_in : sd.c_in == -2 ? st->defer_rows : st->r_in;
  const int k_out = sd.k_out >= 0 ? sd.k_out : sd.k_out == -2 ? st->r : st->k_out;
  if (c_in > KB || k_out > KB) return;  // the host picks KB >= both; never taken
  const bool zhat = sd.zhat && (sd.zrho ? *sd.zrho > 0.0 : st->grew != 0);
  const double* zp = sd.zrho ? sd.zp : p;
  const int nrr = c_in + (zhat || sd.newrow ? 1 : 0);
  const T* X = reinterpret_cast<const T*>(sd.X);
  T* Y = reinterpret_cast<T*>(sd.Y);
  const T* R = reinterpret_cast<const T*>(sd.R);
  const int64_t row0 = tile * kRotRows;
  const int t = threadIdx.x;
  for (int idx = t; idx < (KB + 1) * KB; idx += kRotThreads) {
    const int c = idx / KB, j = idx - c * KB;
    T v = T(0);
    if (c < nrr && j < k_out) {
      v = R[(int64_t)c * sd.ldr + j];
      if (sd.colscale && c < c_in) v = (T)((double)v * sd.colscale[j]);
    }
    Rs[idx] = v;
  }
  for (int idx = t; idx < kRotRows * KB; idx += kRotThreads) {
    const int rr = idx / KB, c = idx - rr * KB;
    const int64_t row = row0 + rr;
    T v = T(0);
    if (row < sd.rows && c < c_in) v = X[row * sd.ldx + c];
    Xs[c * (kRotRows + 1) + rr] = v;
  }
  __syncthreads();
  if (zhat) {
    const int rr = t >> 2, part = t & 3;
    double d = 0.0;
    for (int c = part; c < c_in; c += 4) d += (double)Xs[c * (kRotRows + 1) + rr] * zp[c];
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    if (part == 0) {
      const int64_t row = row0 + rr;
      const double src = sd.zrho ? (row == sd.zunit ? 1.0 : 0.0) : (row < sd.rows ? (double)xz[row] : 0.0);
      zs[rr] = row < sd.rows ? (T)((src - d) / (sd.zrho ? *sd.zrho : st->rho)) : T(0);
    }
    __syncthreads();
  }
  const int ty = t >> 4, tx = t & 15;
  T acc[4][CPT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = T(0);
  for (int c = 0; c < c_in; ++c) {
    T xa[4], rb[CPT];
#pragma unroll
    for (int i = 0; i < 4; ++i) xa[i] = Xs[c * (kRotRows + 1) + ty * 4 + i];
#pragma unroll
    for (int j = 0; j < CPT; ++j) rb[j] = Rs[c * KB + tx * CPT + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[i][j] += xa[i] * rb[j];
  }
  if (zhat) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[i][j] += zs[ty * 4 + i] * Rs[c_in * KB + tx * CPT + j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + ty * 4 + i;
    if (row < sd.rows) {
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int col = tx * CPT + j;
        if (col < k_out) Y[row * sd.ldy + col] = acc[i][j];
      }
    }
  }
  if (sd.newrow && tile == 0) {
    for (int j = t; j < k_out; j += kRotThreads) Y[sd.rows * sd.ldy + j] = Rs[c_in * KB + j];
  }
}

// ---- deferred rotations (Brand's U = U0 R_U, V = V0 R_V) -------------------------------------
//
// The rank-1 entry update of Section 2.3 rotates both tall factors by its core factors: U' = U U_K,
// V' = V V_K. Written as U = U0 R_U with a small R_U (rows = defer_rows, the columns of U0), the
// update only needs R_U <- R_U U_K (O(k^3) on k x k data instead of O((m + n) k^2) on the tall
// factors), and the gathers of the next core read U0[i, :] R_U. Everything that needs U itself
// (appends, refresh, metrics, re-orthogonalisation, reads) first folds U <- U0 R_U in one pass of
// the rotation kernel (c_in = -2, k_out = -2).

// R_U = R_V = I of the current rank r (rows x ldr, rows >= r, zero elsewhere); defer_rows <- r.
template <typename T>
__global__ void __launch_bounds__(256) k_defer_init(T* RU, T* RV, int ldr, int rows, DevState* st) {
  const int dr = st->r;
  const int64_t total = (int64_t)rows * ldr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx / ldr), c = (int)(idx - (int64_t)l * ldr);
    const T v = (l == c && l < dr) ? T(1) : T(0);
    RU[idx] = v;
    RV[idx] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->defer_rows = dr;
}

// R <- R[:, :r_in] K[:r_in, :k_out] for both sides (blockIdx.y: 0 = R_U with U_K, 1 = R_V with
// V_K), one row of R per block, in place (the row is staged before it is overwritten); columns
// k_out .. r_in - 1 of a truncated product are cleared. Sums in T, in the order of the tall
// rotation's.
template <typename T>
__global__ void __launch_bounds__(128) k_defer_compose(T* RU, T* RV, int ldr, const T* __restrict__ UK,
                                                       const T* __restrict__ VK, int ldo, const DevState* st) {
  __shared__ T row[kKmaxLimit + 1];
  const int l = blockIdx.x;
  const int dr = st->defer_rows, r_in = st->r_in, k_out = st->k_out;
  if (l >= dr || r_in > kKmaxLimit || k_out > r_in) return;  // uniform over the block
  T* R = blockIdx.y ? RV : RU;
  const T* K = blockIdx.y ? VK : UK;
  for (int c = threadIdx.x; c < r_in; c += blockDim.x) row[c] = R[(int64_t)l * ldr + c];
  __syncthreads();
  for (int j = threadIdx.x; j < r_in; j += blockDim.x) {
    T s = T(0);
    if (j < k_out)
      for (int c = 0; c < r_in; ++c) s += row[c] * K[(int64_t)c * ldo + j];
    R[(int64_t)l * ldr + j] = s;
  }
}

}  // namespace isvd
