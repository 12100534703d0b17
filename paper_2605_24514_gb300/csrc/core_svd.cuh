// Core SVD of the small update matrix K (Section 2.2 Step 2 and Section 2.3): one CTA,
// one-sided (Hestenes) Jacobi held in shared memory, plus assembly of K, FP64 singular values,
// descending sort and truncation to the working rank.
#pragma once

#include "isvd_common.cuh"

namespace isvd {

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Dot product of two shared-memory vectors over the rows of one half-warp (16 lanes), with the
// storage type's rounding (JT = double) or, for JT = float, in the compensated "Dot2" form of
// Ogita, Rump and Oishi (2005): exact products by FMA, TwoSum accumulation, so the result is as
// accurate as if computed in twice the working precision. Every lane of the half-warp returns it.
template <typename JT>
__device__ __forceinline__ JT half_dot(const JT* x, const JT* y, int n, int hl, bool valid);
template <>
__device__ __forceinline__ double half_dot<double>(const double* x, const double* y, int n, int hl, bool valid) {
  double g = 0.0;
  if (valid)
    for (int row = hl; row < n; row += 16) g += x[row] * y[row];
  return half_sum(g);
}
template <>
__device__ __forceinline__ float half_dot<float>(const float* x, const float* y, int n, int hl, bool valid) {
  float s = 0.f, c = 0.f;
  if (valid) {
    for (int row = hl; row < n; row += 16) {
      const float a = x[row], b = y[row];
      const float p = a * b;
      const float pe = fmaf(a, b, -p);
      float t;
      two_sum(s, p, s, t);
      c += t + pe;
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float t;
    two_sum(s, s2, s, t);
    c = c + c2 + t;
  }
  return s + c;
}

// Same over a full warp (32 lanes), returned in FP64 on every lane.
__device__ __forceinline__ double warp_dot2(const float* x, int sx, const float* y, int sy, int n, int lane) {
  float s = 0.f, c = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float a = x[(size_t)i * sx], b = y[(size_t)i * sy];
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float t;
    two_sum(s, p, s, t);
    c += t + pe;
  }
  double d = (double)s + (double)c;
  return warp_sum(d);
}

// One-sided Jacobi on the nr x nc matrix W (column-major in shared memory, column stride ldw).
// Rotations are applied to W's columns and accumulated into VK (nc x nc, column stride ldv,
// initialised to I by the caller), so on exit W = K VK has mutually orthogonal columns.
// Pairs follow the round-robin (circle) ordering: N-1 rounds of N/2 disjoint pairs (N = nc
// rounded up to even), each pair on one half-warp (16 lanes over rows), so every round is one
// barrier. A pair is rotated when |w_i^T w_j| > tol ||w_i|| ||w_j||. Returns the number of sweeps
// run, or -1 when the last allowed sweep still rotated.
template <typename JT>
__device__ int jacobi_cta(JT* W, int ldw, int nr, JT* VK, int ldv, int nc, JT tol, int max_sweeps,
                          int* s_flag) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4;
  const int hl = lane & 15;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int N = nc + (nc & 1);
  const int npairs = N / 2;
  const int nq2 = (npairs + 1) / 2;
  if (nc < 2) return 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    for (int rd = 0; rd < N - 1; ++rd) {
      for (int q2 = warp; q2 < nq2; q2 += nw) {
        const int q = 2 * q2 + half;
        int i = 0, j = 0;
        bool valid = q < npairs;
        if (valid) {
          if (q == 0) {
            i = rd;
            j = N - 1;
          } else {
            i = (rd + q) % (N - 1);
            j = (rd - q + N - 1) % (N - 1);
          }
          if (i > j) {
            const int t = i;
            i = j;
            j = t;
          }
          valid = j < nc;
        }
        JT a = 0, b = 0;
        JT* wi = W + (size_t)i * ldw;
        JT* wj = W + (size_t)j * ldw;
        if (valid) {
          for (int row = hl; row < nr; row += 16) {
            const JT x = wi[row], y = wj[row];
            a += x * x;
            b += y * y;
          }
        }
        a = half_sum(a);
        b = half_sum(b);
        const JT g = half_dot<JT>(wi, wj, nr, hl, valid);
        if (valid && a > JT(0) && b > JT(0) && fabs(g) > tol * sqrt(a) * sqrt(b)) {
          const JT zeta = (b - a) / (JT(2) * g);
          JT t;
          if (fabs(zeta) > JT(1e15)) {
            t = JT(0.5) / zeta;
          } else {
            t = copysign(JT(1), zeta) / (fabs(zeta) + sqrt(JT(1) + zeta * zeta));
          }
          const JT c = JT(1) / sqrt(JT(1) + t * t);
          const JT s = c * t;
          for (int row = hl; row < nr; row += 16) {
            const JT x = wi[row], y = wj[row];
            wi[row] = c * x - s * y;
            wj[row] = s * x + c * y;
          }
          JT* vi = VK + (size_t)i * ldv;
          JT* vj = VK + (size_t)j * ldv;
          for (int row = hl; row < nc; row += 16) {
            const JT x = vi[row], y = vj[row];
            vi[row] = c * x - s * y;
            vj[row] = s * x + c * y;
          }
          if (hl == 0) *s_flag = 1;
        }
      }
      __syncthreads();
    }
    if (*s_flag == 0) return sweep + 1;
  }
  return -1;
}

// Input of one core SVD (everything FP64, as the paper's core and rho are kept in FP64).
struct CoreIn {
  int kind;          // kRow / kCol (arrow core) or kEntry (diagonal plus rank one)
  int r;             // current rank
  int grew;          // arrow only: rho > tol, so K is (r+1) x (r+1) with rho at (r, r)
  int kt;            // working rank k_t (truncation target)
  const double* sig; // r singular values (descending)
  const double* p;   // arrow: projection coefficients p (r)
  double rho;        // arrow: residual norm
  const double* a;   // entry: s_u = U[i, :] (r)
  const double* b;   // entry: s_v = V[j, :] (r)
  double delta;      // entry: increment
};

// Shared-memory bytes needed by core_svd_cta for the given rank capacity.
template <typename JT>
__host__ __device__ inline size_t core_smem_bytes(int kmax) {
  const int n = kmax + 1;
  const int mats = sizeof(JT) < sizeof(double) ? 3 : 2;  // W, V_K (+ the polish matrix E)
  return (size_t)mats * n * n * sizeof(JT) + (size_t)n * (sizeof(double) * 2 + sizeof(int) * 2) + 64;
}

// Assembles K (Section 2.2 Step 2: K = [[Sigma, 0], [p, rho]]; Section 2.3: K = Sigma +
// delta s_u s_v^T), takes its SVD, sorts descending, truncates to min(kt, nc) and writes
//   UK (nr x k_out, row stride ldo, element type T): left singular vectors,
//   VKo (nc x k_out, row stride ldo): right singular vectors,
//   sig_out (k_out doubles).
// Reading (rank-preserving append, rho <= tol): K is the (r+1) x r matrix [[Sigma], [p]].
// JT is the Jacobi arithmetic; with JT = float the singular values are recomputed in FP64 as
// ||K v_j|| / ||v_j|| using K's structure (O(r) per value), so only the singular vectors carry
// FP32 rounding. Returns k_out; sets *sweeps (-1 = not converged). All threads must call it.
template <typename T, typename JT>
__device__ int core_svd_cta(const CoreIn& in, unsigned char* smem, T* UK, T* VKo, int ldo,
                            double* sig_out, int* sweeps) {
  const int r = in.r;
  int nr, nc;
  if (in.kind == kEntry) {
    nr = r;
    nc = r;
  } else {
    nr = r + 1;
    nc = in.grew ? r + 1 : r;
  }
  const int ldw = nr, ldv = nc;
  JT* W = reinterpret_cast<JT*>(smem);
  JT* VK = W + (size_t)nc * ldw;
  JT* Ep = VK + (size_t)nc * ldv;  // nc x nc polish matrix (FP32 Jacobi only)
  const bool low = sizeof(JT) < sizeof(double);
  double* sref = reinterpret_cast<double*>(Ep + (low ? (size_t)nc * nc : 0));
  sref = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(sref) + 15) & ~uintptr_t(15));
  double* nrm = sref + nc;
  int* perm = reinterpret_cast<int*>(nrm + nc);
  int* flag = perm + nc;

  // K, column-major.
  for (int idx = threadIdx.x; idx < nc * nr; idx += blockDim.x) {
    const int c = idx / nr, row = idx - c * nr;
    double v = 0.0;
    if (in.kind == kEntry) {
      v = (row == c ? in.sig[c] : 0.0) + in.delta * in.a[row] * in.b[c];
    } else if (c < r) {
      v = (row == c) ? in.sig[c] : (row == r ? in.p[c] : 0.0);
    } else {
      v = (row == r) ? in.rho : 0.0;
    }
    W[(size_t)c * ldw + row] = (JT)v;
  }
  for (int idx = threadIdx.x; idx < nc * nc; idx += blockDim.x) {
    const int c = idx / nc, row = idx - c * nc;
    VK[(size_t)c * ldv + row] = (row == c) ? JT(1) : JT(0);
  }
  // FP64 Jacobi: tolerance 2 eps sqrt(nr). FP32 Jacobi: the compensated dot product resolves
  // w_i^T w_j below the FP32 rounding of the products, so the tolerance is eps sqrt(nr) / 2.
  const JT tol = (low ? JT(0.5) : JT(2)) * Eps<JT>::v * sqrt((JT)(nr > 1 ? nr : 1));
  const int sw = jacobi_cta<JT>(W, ldw, nr, VK, ldv, nc, tol, 40, flag);
  if (threadIdx.x == 0) *sweeps = sw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (low) {
    // The FP32-accumulated rotations leave V_K orthogonal to only ~sqrt(rotations) eps. One
    // additive Newton-Schulz step V <- V + V E, E = (I - V^T V) / 2, with V^T V from the
    // compensated dot product, restores orthogonality to the FP32 rounding level.
    for (int e = warp; e < nc * nc; e += nw) {
      const int a = e / nc, b = e - a * nc;
      if (b < a) continue;
      const double g = warp_dot2(reinterpret_cast<const float*>(VK) + (size_t)a * ldv, 1,
                                 reinterpret_cast<const float*>(VK) + (size_t)b * ldv, 1, nc, lane);
      if (lane == 0) {
        const JT v = (JT)(((a == b ? 1.0 : 0.0) - g) * 0.5);
        Ep[(size_t)a * nc + b] = v;
        Ep[(size_t)b * nc + a] = v;
      }
    }
    __syncthreads();
    // Row by row (one warp per row of V_K): row <- row + row E. Rows are independent, so the
    // update is in place.
    for (int row = warp; row < nc; row += nw) {
      JT acc[5];
      JT rv[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int c = lane + 32 * q;
        rv[q] = c < nc ? VK[(size_t)c * ldv + row] : JT(0);
        acc[q] = JT(0);
      }
      for (int l = 0; l < nc; ++l) {
        const JT vl = __shfl_sync(0xffffffffu, rv[l >> 5], l & 31);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const int c = lane + 32 * q;
          if (c < nc) acc[q] += vl * Ep[(size_t)l * nc + c];
        }
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int c = lane + 32 * q;
        if (c < nc) VK[(size_t)c * ldv + row] = rv[q] + acc[q];
      }
    }
    __syncthreads();
  }

  // Column norms of W = K VK (Jacobi arithmetic) and FP64 singular values.
  for (int j = warp; j < nc; j += nw) {
    double s2 = 0.0;
    for (int row = lane; row < nr; row += 32) {
      const double w = (double)W[(size_t)j * ldw + row];
      s2 += w * w;
    }
    s2 = warp_sum(s2);
    double sig = sqrt(s2);
    if (sizeof(JT) < sizeof(double)) {
      // ||K v|| / ||v|| in FP64 through K's structure.
      const JT* v = VK + (size_t)j * ldv;
      double nv = 0.0, acc = 0.0, dot = 0.0;
      for (int i = lane; i < nc; i += 32) {
        const double vi = (double)v[i];
        nv += vi * vi;
      }
      nv = warp_sum(nv);
      if (in.kind == kEntry) {
        for (int i = lane; i < r; i += 32) dot += in.b[i] * (double)v[i];
        dot = warp_sum(dot);
        for (int i = lane; i < r; i += 32) {
          const double y = in.sig[i] * (double)v[i] + in.delta * in.a[i] * dot;
          acc += y * y;
        }
        acc = warp_sum(acc);
      } else {
        for (int i = lane; i < r; i += 32) {
          const double vi = (double)v[i];
          acc += (in.sig[i] * vi) * (in.sig[i] * vi);
          dot += in.p[i] * vi;
        }
        acc = warp_sum(acc);
        dot = warp_sum(dot);
        const double yr = dot + (in.grew ? in.rho * (double)v[r] : 0.0);
        acc += yr * yr;
      }
      sig = nv > 0.0 ? sqrt(acc / nv) : 0.0;
    }
    if (lane == 0) {
      nrm[j] = sqrt(s2);
      sref[j] = sig;
    }
  }
  // Descending order, ties by index (stable); identity first, so a NaN value can misorder but
  // never leave a slot unset.
  for (int j = threadIdx.x; j < nc; j += blockDim.x) perm[j] = j;
  __syncthreads();
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    const double sj = sref[j];
    int rank = 0;
    for (int l = 0; l < nc; ++l) {
      const double sl = sref[l];
      rank += (sl > sj) || (sl == sj && l < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
  const int k_out = in.kt < nc ? in.kt : nc;
  double nmax = 0.0;
  for (int j = 0; j < nc; ++j) nmax = fmax(nmax, nrm[j]);
  const double null_thr = nmax * 1e-30;
  for (int idx = threadIdx.x; idx < nr * k_out; idx += blockDim.x) {
    const int row = idx / k_out, jj = idx - row * k_out;
    const int j = perm[jj];
    const double nj = nrm[j];
    UK[(size_t)row * ldo + jj] = (nj > null_thr) ? (T)((double)W[(size_t)j * ldw + row] / nj) : T(0);
  }
  for (int idx = threadIdx.x; idx < nc * k_out; idx += blockDim.x) {
    const int row = idx / k_out, jj = idx - row * k_out;
    VKo[(size_t)row * ldo + jj] = (T)VK[(size_t)perm[jj] * ldv + row];
  }
  for (int jj = threadIdx.x; jj < k_out; jj += blockDim.x) sig_out[jj] = sref[perm[jj]];
  __syncthreads();
  __threadfence_block();
  // Orthonormal completion of left vectors whose singular value is exactly zero (their
  // direction is arbitrary; only orthonormality of U_K matters). Rare: one warp, serial in jj.
  if (warp == 0) {
    for (int jj = 0; jj < k_out; ++jj) {
      if (nrm[perm[jj]] > null_thr) continue;
      for (int cand = 0; cand < nr; ++cand) {
        // v = e_cand - sum_q u_q u_q[cand], two passes; lanes over rows.
        double vloc[8];
        const int per = (nr + 31) / 32;
        for (int t = 0; t < per && t < 8; ++t) {
          const int row = lane + 32 * t;
          vloc[t] = (row == cand) ? 1.0 : 0.0;
        }
        for (int pass = 0; pass < 2; ++pass) {
          for (int q = 0; q < k_out; ++q) {
            if (q == jj || (nrm[perm[q]] <= null_thr && q > jj)) continue;
            double d = 0.0;
            for (int t = 0; t < per && t < 8; ++t) {
              const int row = lane + 32 * t;
              if (row < nr) d += (double)UK[(size_t)row * ldo + q] * vloc[t];
            }
            d = warp_sum(d);
            for (int t = 0; t < per && t < 8; ++t) {
              const int row = lane + 32 * t;
              if (row < nr) vloc[t] -= d * (double)UK[(size_t)row * ldo + q];
            }
          }
        }
        double n2 = 0.0;
        for (int t = 0; t < per && t < 8; ++t) {
          const int row = lane + 32 * t;
          if (row < nr) n2 += vloc[t] * vloc[t];
        }
        n2 = warp_sum(n2);
        if (n2 > 0.25) {
          const double inv = 1.0 / sqrt(n2);
          for (int t = 0; t < per && t < 8; ++t) {
            const int row = lane + 32 * t;
            if (row < nr) UK[(size_t)row * ldo + jj] = (T)(vloc[t] * inv);
          }
          __syncwarp();
          break;
        }
      }
    }
  }
  __syncthreads();
  return k_out;
}

}  // namespace isvd
