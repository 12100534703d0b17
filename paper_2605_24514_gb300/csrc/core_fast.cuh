// Fast core SVD for the FP32-bulk path (Section 2.2 Step 2 and Section 2.3 cores).
//
// Both cores are low-rank modifications of a diagonal matrix, so their right singular
// vectors are eigenvectors of K^T K = diag + low rank:
//   append:  K^T K = diag(sigma^2, 0) + w w^T,  w = (p, rho)            (one rank-one update)
//   entry:   K^T K = Sigma^2 + c b^T + b c^T + mu b b^T,  c = delta Sigma a, mu = delta^2 |a|^2
//            = Sigma^2 + m1 u1 u1^T + m0 u0 u0^T with m1 > 0 > m0     (two rank-one updates)
// Each rank-one eigenproblem diag(d) + w w^T is solved through its secular equation
// 1 + sum_i w_i^2 / (d_i - lambda) = 0 (Golub 1973; Bunch, Nielsen and Sorensen 1978): one root
// per interval between consecutive poles, found by bisection in the shifted variable
// tau = lambda - (nearer pole) so that lambda - d_i keeps its relative accuracy, with eigenvector
// v_i = w_i / (d_i - lambda). This is O(k^2) work, parallel over roots, instead of the O(k^3)
// sequential rounds of a Jacobi sweep. The result is checked (Gram of W = K V and of V) and, if
// needed, polished by one first-order correction step; if the check still fails (ties among the
// poles, strong coupling) the caller falls back to the one-sided Jacobi.
#pragma once

#include "core_svd.cuh"
#include "isvd_common.cuh"

namespace isvd {

constexpr int kSecLanes = 8;  // lanes per root
// Two non-deflated poles closer than kTieRel * (largest pole) count as tied (the CTA Jacobi core
// takes the update). The poles are float pairs (relative precision ~1e-14) and every difference is
// formed from them, so gaps well below FP32 resolution still give accurate roots and weights.
constexpr float kTieRel = 1e-12f;
// Largest accepted |w_hat_i - w_i| of the corrected weights, in units of eps ||w||: the product
// for w_hat_i^2 has ~2 n roundings (a random walk of ~4 sqrt(n) eps for n <= 65), so 32 eps
// rejects only inaccurate roots while keeping the backward error at the FP32 level.
constexpr float kGeTolEps = 32.f;

// Float-float ("double-FP32") helpers: error-free transformations give FP64-class accuracy on
// the FP32 pipes, which on this part run ~57x faster than FP64.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {  // (a.hi + a.lo) * b
  ff p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  const float h = p.hi + p.lo;
  return {h, p.lo - (h - p.hi)};
}
__device__ __forceinline__ ff ff_sqr(ff a) {
  ff p = two_prod(a.hi, a.hi);
  p.lo = fmaf(2.f * a.hi, a.lo, p.lo);
  const float h = p.hi + p.lo;
  return {h, p.lo - (h - p.hi)};
}
__device__ __forceinline__ float ff_sub_to_f(ff a, ff b) {  // a - b rounded once (exact hi part when close)
  return (a.hi - b.hi) + (a.lo - b.lo);
}
template <int W>
__device__ __forceinline__ ff ff_group_sum(ff v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    ff w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w);
  }
  return v;
}

// Secular-equation eigensolver for diag(d) + w w^T (one CTA). Poles d are given in ASCENDING order
// as float pairs (dhi + dlo) with weights w in the same order; row[s] is the output row of sorted
// entry s. On exit column j of V (column-major, stride ldv) is the unit eigenvector of the j-th
// smallest eigenvalue, stored as (lam_hi[j] + lam_lo[j]). Returns false (on all threads) when two
// non-deflated poles coincide to within the FP32 resolution or the order is violated.
// With tau_out set, the vectors are not formed; instead each root is returned as its origin pole
// org_out[j] and the offset tau_out[j] from it (lambda_j = d[org_out[j]] + tau_out[j]), for the
// corrected-weight construction below.
template <int kTerms>
__device__ bool secular_cta(int n, const float* dhi, const float* dlo, const float* w, const int* row, float* V,
                            int ldv, float* lam_hi, float* lam_lo, int* nxt, float* sc, int* s_flag,
                            float* tau_out = nullptr, int* org_out = nullptr) {
  const int t = threadIdx.x;
  if (t == 0) *s_flag = 0;
  if (t < 32) {
    float s = 0.f, c = 0.f;
    for (int i = t; i < n; i += 32) {
      const ff q = two_prod(w[i], w[i]);
      float e;
      two_sum(s, q.hi, s, e);
      c += e + q.lo;
    }
    ff v = ff_group_sum<32>(ff{s, c});
    if (t == 0) {
      sc[0] = v.hi + v.lo;                                   // ||w||^2
      sc[1] = fmaxf(fabsf(dhi[0]), fabsf(dhi[n - 1]));       // pole scale
    }
  }
  __syncthreads();
  const float defl_thr = 1e-7f * sqrtf(sc[0]);
  const float dscale = sc[1];
  for (int j = t; j < n; j += blockDim.x) {
    int nx = -1;
    for (int l = j + 1; l < n; ++l)
      if (fabsf(w[l]) > defl_thr) {
        nx = l;
        break;
      }
    nxt[j] = nx;
    if (j + 1 < n && ff_sub_to_f(ff{dhi[j + 1], dlo[j + 1]}, ff{dhi[j], dlo[j]}) < 0.f) atomicOr(s_flag, 1);
    if (fabsf(w[j]) > defl_thr && nx >= 0 &&
        ff_sub_to_f(ff{dhi[nx], dlo[nx]}, ff{dhi[j], dlo[j]}) <= kTieRel * dscale)
      atomicOr(s_flag, 1);
  }
  if (t < 32) {  // sum of the non-deflated squared weights (width of the last interval)
    float s = 0.f;
    for (int i = t; i < n; i += 32)
      if (fabsf(w[i]) > defl_thr) s += w[i] * w[i];
    s = warp_sum(s);
    if (t == 0) sc[2] = s * (1.f + 1e-5f);
  }
  __syncthreads();
  ISVD_STAMP(8);
  if (*s_flag) return false;
  const float wsum = sc[2];
  const int lane = t & 31;
  const int g = lane & (kSecLanes - 1);
  const int group = t / kSecLanes;
  const int ngroups = blockDim.x / kSecLanes;
  const int rounds = (n + ngroups - 1) / ngroups;
  const int nq = (n + kSecLanes - 1) / kSecLanes;
  for (int rr = 0; rr < rounds; ++rr) {
    const int j = group + rr * ngroups;
    const bool live = j < n;
    const bool solve = live && fabsf(w[j]) > defl_thr;
    const int nx = solve ? nxt[j] : -1;
    const bool last = solve && nx < 0;
    const ff lo = live ? ff{dhi[j], dlo[j]} : ff{0.f, 0.f};
    const ff hi = (solve && !last) ? ff{dhi[nx], dlo[nx]} : lo;
    // This lane's terms: poles shifted to both interval ends and squared weights.
    float dl[kTerms], dh[kTerms], w2[kTerms];
#pragma unroll
    for (int q = 0; q < kTerms; ++q) {
      const int i = g + q * kSecLanes;
      const bool on = solve && q < nq && i < n && fabsf(w[i]) > defl_thr;
      const float wi = on ? w[i] : 0.f;
      w2[q] = wi * wi;
      const ff di = on ? ff{dhi[i], dlo[i]} : ff{0.f, 0.f};
      dl[q] = on ? ff_sub_to_f(di, lo) : 1.f;
      dh[q] = on ? ff_sub_to_f(di, hi) : 1.f;
    }
    auto f_eval = [&](const float* dd, float tau) -> float {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < kTerms; ++q)
        if (q < nq) s += __fdividef(w2[q], dd[q] - tau);
#pragma unroll
      for (int o = kSecLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      return 1.f + s;
    };
    const float width = last ? wsum : ff_sub_to_f(hi, lo);
    const float half = 0.5f * width;
    const float f_mid = f_eval(dl, half);
    float sgn = 1.f, a = 0.f, b = 0.f;
    bool use_hi = false;
    if (solve) {
      if (last || f_mid > 0.f) {
        b = last ? width : half;
      } else {
        sgn = -1.f;
        b = half;
        use_hi = true;
      }
    }
    const float* dor = use_hi ? dh : dl;
    // In u = sgn * tau the function h(u) = sgn * f(sgn * u) increases from -inf at the near pole
    // (u = 0) and the root lies in (a, b). Each step fits the near-pole model h ~ C - S / u to
    // h and h' at the current u (S = h' u^2, C = h + h' u) and takes its root S / C, falling back
    // to bisection (geometric when the bracket spans decades) whenever that leaves the bracket.
    float u = 0.5f * b;
    for (int it = 0; it < 40; ++it) {
      float fs = 0.f, ds = 0.f;
      if (solve) {
        const float tau_k = sgn * u;
#pragma unroll
        for (int q = 0; q < kTerms; ++q) {
          if (q < nq) {
            const float rq = __fdividef(1.f, dor[q] - tau_k);
            const float t1 = w2[q] * rq;
            fs += t1;
            ds = fmaf(t1, rq, ds);
          }
        }
      }
#pragma unroll
      for (int o = kSecLanes / 2; o > 0; o >>= 1) {
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
      }
      bool done = !solve;
      if (solve) {
        const float h = sgn * (1.f + fs);
        const float hp = ds;  // h'(u) = f'(tau) > 0
        if (h == 0.f) {
          done = true;  // exact root: keep u
        } else {
          if (h < 0.f) a = u;
          else b = u;
          const float C = h + hp * u;
          float un = (C > 0.f) ? hp * u * u / C : -1.f;
          if (!(un > a && un < b)) un = (a > 0.f && b > 4.f * a) ? sqrtf(a) * sqrtf(b) : 0.5f * (a + b);
          done = fabsf(un - u) <= 1e-7f * un || (b - a) <= 2.4e-7f * b;
          u = un;
        }
      }
      if (__all_sync(0xffffffffu, done)) break;
    }
    const float tau = sgn * u;
    if (tau_out) {
      if (live && g == 0) {
        const ff org = use_hi ? hi : lo;
        const ff lam = solve ? ff_add(org, ff{tau, 0.f}) : lo;
        lam_hi[j] = lam.hi;
        lam_lo[j] = lam.lo;
        tau_out[j] = solve ? tau : 0.f;
        org_out[j] = (solve && use_hi) ? nx : j;
      }
      continue;
    }
    float vq[kTerms];
    float nrm2 = 0.f;
#pragma unroll
    for (int q = 0; q < kTerms; ++q) {
      const int i = g + q * kSecLanes;
      float v = 0.f;
      if (q < nq && w2[q] > 0.f) v = w[i] / (dor[q] - tau);
      vq[q] = v;
      nrm2 += v * v;
    }
#pragma unroll
    for (int o = kSecLanes / 2; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
    if (live) {
      const float inv = (solve && nrm2 > 0.f) ? rsqrtf(nrm2) : 0.f;
#pragma unroll
      for (int q = 0; q < kTerms; ++q) {
        const int i = g + q * kSecLanes;
        if (q < nq && i < n) V[(size_t)j * ldv + row[i]] = solve ? vq[q] * inv : (i == j ? 1.f : 0.f);
      }
      if (g == 0) {
        const ff org = use_hi ? hi : lo;
        const ff lam = solve ? ff_add(org, ff{tau, 0.f}) : lo;
        lam_hi[j] = lam.hi;
        lam_lo[j] = lam.lo;
      }
    }
  }
  __syncthreads();
  return true;
}

// Append core vectors from corrected weights (Gu and Eisenstat 1994/95; the construction LAPACK's
// divide-and-conquer SVD uses for its broken-arrow matrices). Given the computed roots lambda_j of
// diag(d) + w w^T (as origin pole + tau), the weights w_hat for which those roots are EXACT
// eigenvalues follow from Loewner's formula
//   w_hat_i^2 = prod_j (lambda_j - d_i) / prod_{l != i} (d_l - d_i)   (non-deflated i, j, l),
// evaluated as a product of ratios, each pairing a root with the pole next to it so that every
// factor is positive and of moderate size. Every difference lambda_j - d_i is taken as
// (d_org(j) - d_i) + tau_j from the float-pair poles, so it keeps its relative accuracy. Then
//   v_j = (w_hat_i / (d_i - lambda_j))_i / norm,   K_hat v_j = (sigma_i v_ji for the Sigma rows; -1),
// the last entry because sum_i w_hat_i^2 / (d_i - lambda_j) = -1 exactly for the modified
// problem. Both vector sets are componentwise accurate and hence orthogonal to working precision,
// whatever the spread of the singular values; K_hat differs from K only by w_hat - w, which is
// checked against tol_bw ||w|| (a failed check, like a deflated rho pole, returns false).
// V: n x n, column j at V + j n, rows in original order (row[]); U: nr x n with column stride nr
// (row i < r is sigma_i's, row r the new row's); sf = float sigma in original order.
static __device__ bool ge_append_vectors(int n, int r, int nr, const float* dhi, const float* dlo, const float* w,
                                  const int* row, const int* nxt, const float* tau, const int* org, const float* sf,
                                  float* what, float* V, float* U, float wn2, float tol_bw, int* s_flag) {
  const int t = threadIdx.x;
  const float thr = 1e-7f * sqrtf(wn2);  // the deflation threshold of secular_cta
  if (t == 0) *s_flag = 0;
  __syncthreads();
  for (int i = t; i < n; i += blockDim.x) {
    float wh = 0.f;
    if (fabsf(w[i]) > thr) {
      const ff di{dhi[i], dlo[i]};
      float prod = 1.f;
      for (int j = 0; j < n; ++j) {
        if (!(fabsf(w[j]) > thr)) continue;
        const int o = org[j];
        const float num = ff_sub_to_f(ff{dhi[o], dlo[o]}, di) + tau[j];  // lambda_j - d_i
        const int nj = nxt[j];
        if (nj < 0) {
          prod *= num;
        } else {
          const int pj = j < i ? j : nj;
          prod *= __fdividef(num, ff_sub_to_f(ff{dhi[pj], dlo[pj]}, di));
        }
      }
      wh = copysignf(sqrtf(fmaxf(prod, 0.f)), w[i]);
      if (!(fabsf(wh - w[i]) <= tol_bw * sqrtf(wn2))) atomicOr(s_flag, 1);
    } else if (row[i] >= r) {
      atomicOr(s_flag, 1);  // rho pole deflated: its left vector is not e_r
    }
    what[i] = wh;
  }
  __syncthreads();
  if (*s_flag) return false;
  // Unnormalised v_j (deflated j: e_j), entry by entry.
  for (int idx = t; idx < n * n; idx += blockDim.x) {
    const int j = idx / n, i = idx - j * n;
    float v;
    if (!(fabsf(w[j]) > thr)) {
      v = (i == j) ? 1.f : 0.f;
    } else if (what[i] == 0.f) {
      v = 0.f;
    } else {
      const int o = org[j];
      const float dl = ff_sub_to_f(ff{dhi[o], dlo[o]}, ff{dhi[i], dlo[i]}) + tau[j];  // lambda_j - d_i
      v = -what[i] / dl;
    }
    V[(size_t)j * n + row[i]] = v;
  }
  __syncthreads();
  // Normalise v_j and form u_j (one warp per column).
  const int warp = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < n; j += nw) {
    float* v = V + (size_t)j * n;
    float* u = U + (size_t)j * nr;
    const bool defl = !(fabsf(w[j]) > thr);
    float sv = 0.f, su = 0.f;
    for (int i = lane; i < n; i += 32) sv += v[i] * v[i];
    for (int i = lane; i < r; i += 32) {
      const float x = sf[i] * v[i];
      su += x * x;
    }
    sv = warp_sum(sv);
    su = warp_sum(su);
    const float iu = defl ? 1.f : rsqrtf(su + 1.f);
    for (int i = lane; i < nr; i += 32) {  // from the unnormalised v
      float x;
      if (defl) x = (i == row[j]) ? 1.f : 0.f;  // deflated sigma pole: u = e_i
      else x = i < r ? sf[i] * v[i] * iu : -iu;
      u[i] = x;
    }
    __syncwarp();
    const float iv = rsqrtf(sv);
    for (int i = lane; i < n; i += 32) v[i] *= iv;
  }
  __syncthreads();
  return true;
}

// C = A B for n x n column-major FP32 matrices in shared memory (ld = n); 4 x 4 register blocks
// so each thread keeps 16 independent accumulators (the loops are latency-bound otherwise).
__device__ __forceinline__ void smem_gemm_nn(int n, const float* A, const float* B, float* Cm) {
  const int nb = (n + 3) / 4;
  for (int blk = threadIdx.x; blk < nb * nb; blk += blockDim.x) {
    const int bc = blk / nb, br = blk - bc * nb;
    const int r0 = 4 * br, c0 = 4 * bc;
    float acc[4][4] = {};
    for (int l = 0; l < n; ++l) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = (r0 + q < n) ? A[(size_t)l * n + r0 + q] : 0.f;
        b[q] = (c0 + q < n) ? B[(size_t)(c0 + q) * n + l] : 0.f;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (r0 + x < n && c0 + y < n) Cm[(size_t)(c0 + y) * n + r0 + x] = acc[x][y];
  }
}

// Inner-index start of a lane in the column sweeps (the Gram products, z = Q1^T u0). The lanes of a
// warp read columns whose starts differ by multiples of the column stride (often a multiple of 32
// words, i.e. one bank); starting each lane's sweep over the inner index at its own offset spreads
// the reads over the banks. The sums are the same terms in a rotated order.
__device__ __forceinline__ int gram_rot(int inner) { return inner > 0 ? (int)(threadIdx.x & 31) % inner : 0; }

// W = K V through K's structure (column-major, W is nr x nc with column stride nr). sf, xf, bf are
// float copies of sigma, p (append) or delta * a (entry), and b (entry); rhof = rho.
__device__ __forceinline__ void structured_kv(const CoreIn& in, int nr, int nc, const float* V, float* W, float* tmp,
                                              const float* sf, const float* xf, const float* bf, float rhof) {
  const int r = in.r;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float* coef = in.kind == kEntry ? bf : xf;
  for (int j = warp; j < nc; j += nw) {  // tmp_j = coef . V[:r, j] (+ rho V[r, j])
    float s = 0.f;
    for (int i = lane; i < r; i += 32) s += coef[i] * V[(size_t)j * nc + i];
    s = warp_sum(s);
    if (lane == 0) tmp[j] = (in.kind != kEntry && in.grew) ? s + rhof * V[(size_t)j * nc + r] : s;
  }
  __syncthreads();
  if (in.kind == kEntry) {
    for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
      const int j = idx / nr, i = idx - j * nr;
      W[idx] = sf[i] * V[(size_t)j * nc + i] + xf[i] * tmp[j];
    }
  } else {
    for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
      const int j = idx / nr, i = idx - j * nr;
      W[idx] = i < r ? sf[i] * V[(size_t)j * nc + i] : tmp[j];
    }
  }
  __syncthreads();
}

// S = W^T W and Q = V^T V in 4 x 4 register blocks over the upper block triangles, one Gram
// matrix per work item (half the shared-memory loads per FMA of the 2 x 2 form below; used where
// n is large enough that the loads, not the latency of each thread's sweep, bound the products).
__device__ __forceinline__ void smem_two_syrk4(int n, int nr, const float* W, const float* V, float* S, float* Q) {
  const int nb = (n + 3) / 4;
  const int npairs = nb * (nb + 1) / 2;
  const int rs = gram_rot(nr), rq = gram_rot(n);
  for (int pidx = threadIdx.x; pidx < 2 * npairs; pidx += blockDim.x) {
    const bool gs = pidx < npairs;
    int ba = 0, rem = gs ? pidx : pidx - npairs;
    while (rem >= nb - ba) {
      rem -= nb - ba;
      ++ba;
    }
    const int bb = ba + rem;
    const int a0 = 4 * ba, b0 = 4 * bb;
    const float* X = gs ? W : V;
    const int inner = gs ? nr : n;  // also the column stride of X
    const int rot = gs ? rs : rq;
    float acc[4][4] = {};
    for (int l0 = 0; l0 < inner; ++l0) {
      const int l = l0 + rot < inner ? l0 + rot : l0 + rot - inner;
      float xa[4], xb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xa[q] = (a0 + q < n) ? X[(size_t)(a0 + q) * inner + l] : 0.f;
        xb[q] = (b0 + q < n) ? X[(size_t)(b0 + q) * inner + l] : 0.f;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(xa[x], xb[y], acc[x][y]);
    }
    float* G = gs ? S : Q;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int a_ = a0 + x, b_ = b0 + y;
        if (a_ < n && b_ < n) {
          G[(size_t)b_ * n + a_] = acc[x][y];
          G[(size_t)a_ * n + b_] = acc[x][y];
        }
      }
  }
}

// S = W^T W and Q = V^T V together (2 x 2 register blocks over the upper block triangle).
__device__ __forceinline__ void smem_two_syrk(int n, int nr, const float* W, const float* V, float* S, float* Q) {
  const int nb = (n + 1) / 2;
  const int npairs = nb * (nb + 1) / 2;
  for (int pidx = threadIdx.x; pidx < npairs; pidx += blockDim.x) {
    int ba = 0, rem = pidx;
    while (rem >= nb - ba) {
      rem -= nb - ba;
      ++ba;
    }
    const int bb = ba + rem;
    const int a0 = 2 * ba, b0 = 2 * bb;
    const bool a1ok = a0 + 1 < n, b1ok = b0 + 1 < n;
    float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f, q00 = 0.f, q01 = 0.f, q10 = 0.f, q11 = 0.f;
    const int rs = gram_rot(nr), rq = gram_rot(n);
    for (int l0 = 0; l0 < nr; ++l0) {
      const int l = l0 + rs < nr ? l0 + rs : l0 + rs - nr;
      const float xa0 = W[(size_t)a0 * nr + l], xa1 = a1ok ? W[(size_t)(a0 + 1) * nr + l] : 0.f;
      const float xb0 = W[(size_t)b0 * nr + l], xb1 = b1ok ? W[(size_t)(b0 + 1) * nr + l] : 0.f;
      s00 += xa0 * xb0;
      s01 += xa0 * xb1;
      s10 += xa1 * xb0;
      s11 += xa1 * xb1;
    }
    for (int l0 = 0; l0 < n; ++l0) {
      const int l = l0 + rq < n ? l0 + rq : l0 + rq - n;
      const float xa0 = V[(size_t)a0 * n + l], xa1 = a1ok ? V[(size_t)(a0 + 1) * n + l] : 0.f;
      const float xb0 = V[(size_t)b0 * n + l], xb1 = b1ok ? V[(size_t)(b0 + 1) * n + l] : 0.f;
      q00 += xa0 * xb0;
      q01 += xa0 * xb1;
      q10 += xa1 * xb0;
      q11 += xa1 * xb1;
    }
    const float sv[4] = {s00, s01, s10, s11}, qv[4] = {q00, q01, q10, q11};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a_ = a0 + (e >> 1), b_ = b0 + (e & 1);
      if (a_ < n && b_ < n) {
        S[(size_t)b_ * n + a_] = sv[e];
        S[(size_t)a_ * n + b_] = sv[e];
        Q[(size_t)b_ * n + a_] = qv[e];
        Q[(size_t)a_ * n + b_] = qv[e];
      }
    }
  }
}

// Largest rank bucket the fast core serves. Its work matrices V, B and W ((n + 1) x n) stay in
// shared memory; the verification's Gram matrix Q = V^T V joins them up to the 64 bucket and
// lives in the caller's global scratch (n x n floats, L2-resident) for the 128 bucket, where four
// n x n float matrices would exceed the 227 KB of shared memory of a CTA.
constexpr int kFastCoreMaxKB = 128;
constexpr int kFastCoreQSmemMaxKB = 64;

template <typename T>
__host__ __device__ inline size_t core_fast_smem_bytes(int kmax) {
  const int n = kmax + 1;
  const int mats = kmax > kFastCoreQSmemMaxKB ? 3 : 4;
  // V, B (Q2 / S / E), W ((n + 1) x n), [Q (n x n)], 18 n floats of vectors, 3 n ints, 2 n doubles
  return (size_t)(mats * n * n + n + 18 * n) * sizeof(float) + (size_t)n * 3 * sizeof(int) +
         (size_t)n * 2 * sizeof(double) + 256;
}

// Fast core SVD (FP32 vectors, FP64-class singular values). Returns k_out >= 0 on success, or -1
// when the verification failed (the caller then runs the Jacobi path). Output as core_svd_cta.
// gq: global scratch of (KB + 1)^2 floats for the Gram matrix of the 128 bucket (unused below).
template <typename T, int KB>
__device__ int core_fast_cta(const CoreIn& in, unsigned char* smem, T* UK, T* VKo, int ldo, double* sig_out,
                             int* iters, float* gq = nullptr) {
  constexpr bool kQGlobal = KB > kFastCoreQSmemMaxKB;
  constexpr int kTerms = (KB + 1 + kSecLanes - 1) / kSecLanes;
  const int r = in.r;
  int nr, nc;
  if (in.kind == kEntry) {
    nr = r;
    nc = r;
  } else {
    nr = r + 1;
    nc = in.grew ? r + 1 : r;
  }
  const int n = nc;
  const int t = threadIdx.x;
  float* V = reinterpret_cast<float*>(smem);   // n x n
  float* B = V + (size_t)n * n;                 // n x n
  float* W = B + (size_t)n * n;                 // (n + 1) x n
  float* vec = W + (size_t)(n + 1) * n + (kQGlobal ? 0 : (size_t)n * n);  // vectors (after Q when in smem)
  float* dhi = vec;
  float* dlo = vec + n;
  float* wv = vec + 2 * n;
  float* tmp = vec + 3 * n;
  float* lhi = vec + 4 * n;
  float* llo = vec + 5 * n;
  float* sig_hi = vec + 6 * n;  // sigma as float pairs (original order)
  float* sig_lo = vec + 7 * n;
  float* u0 = vec + 8 * n;
  float* sf = vec + 15 * n;   // float sigma
  float* xf = vec + 16 * n;   // float p (append) or delta * a (entry)
  float* bf = vec + 17 * n;   // float b (entry)
  int* rowmap = reinterpret_cast<int*>(vec + 18 * n);
  int* nxt = rowmap + n;
  __shared__ int s_flag;
  __shared__ float s_max[2];
  __shared__ float s_sc[4];
  if (nc < 1) return 0;
  if (kQGlobal && gq == nullptr) return -1;
  ISVD_STAMP(0);
  for (int i = t; i < r; i += blockDim.x) {
    const ff si = ff_of(in.sig[i]);
    sig_hi[i] = si.hi;
    sig_lo[i] = si.lo;
    sf[i] = si.hi;
    xf[i] = (float)(in.kind == kEntry ? in.delta * in.a[i] : in.p[i]);
    bf[i] = in.kind == kEntry ? (float)in.b[i] : 0.f;
  }
  const float rhof = (float)in.rho;
  bool ok, ge = false;
  if (in.kind != kEntry) {
    // Ascending poles: (0 for the rho column when grew), sigma_{r-1}^2, ..., sigma_0^2.
    const int off = in.grew ? 1 : 0;
    for (int s_ = t; s_ < n; s_ += blockDim.x) {
      if (in.grew && s_ == 0) {
        dhi[0] = 0.f;
        dlo[0] = 0.f;
        wv[0] = (float)in.rho;
        rowmap[0] = r;
      } else {
        const int i = r - 1 - (s_ - off);
        const ff d2 = ff_of(in.sig[i] * in.sig[i]);
        dhi[s_] = d2.hi;
        dlo[s_] = d2.lo;
        wv[s_] = (float)in.p[i];
        rowmap[s_] = i;
      }
    }
    __syncthreads();
    ISVD_STAMP(1);
    float* tau = vec + 9 * n;
    float* what = vec + 10 * n;
    int* org = reinterpret_cast<int*>(vec + 11 * n);
    ok = secular_cta<kTerms>(n, dhi, dlo, wv, rowmap, V, n, lhi, llo, nxt, s_sc, &s_flag, tau, org);
    ISVD_STAMP(2);
    if (ok) {
      ge = ge_append_vectors(n, r, nr, dhi, dlo, wv, rowmap, nxt, tau, org, sf, what, V, W, s_sc[0],
                             kGeTolEps * Eps<float>::v, &s_flag);
      // Correction rejected: vectors from w, then the Gram verification below.
      if (!ge) ok = secular_cta<kTerms>(n, dhi, dlo, wv, rowmap, V, n, lhi, llo, nxt, s_sc, &s_flag);
    }
  } else {
    // 2 x 2 eigen-split of [[mu, 1], [1, 0]]: K^T K = Sigma^2 + m1 u1 u1^T + m0 u0 u0^T. The FP64
    // scalars are computed once (thread 0) and shared.
    __shared__ double s_m[6];
    if (t < 32) {
      double s_ = 0.0;
      for (int i = t; i < r; i += 32) s_ += in.a[i] * in.a[i];
      s_ = warp_sum(s_);
      if (t == 0) {
        const double mu = in.delta * in.delta * s_;
        const double disc = sqrt(0.25 * mu * mu + 1.0);
        const double m1 = 0.5 * mu + disc, m0 = 0.5 * mu - disc;
        s_m[0] = m1;
        s_m[1] = m0;
        s_m[2] = sqrt(m1 * m1 + 1.0);
        s_m[3] = sqrt(m0 * m0 + 1.0);
        s_m[4] = sqrt(m1);
        s_m[5] = sqrt(-m0);
      }
    }
    __syncthreads();
    const double m1 = s_m[0], m0 = s_m[1], n1 = s_m[2], n0 = s_m[3], sm1 = s_m[4];
    for (int s_ = t; s_ < n; s_ += blockDim.x) {
      const int i = r - 1 - s_;
      const double bi = in.b[i], ci = in.delta * in.sig[i] * in.a[i];
      const ff d2 = ff_of(in.sig[i] * in.sig[i]);
      dhi[s_] = d2.hi;
      dlo[s_] = d2.lo;
      wv[s_] = (float)(sm1 * (bi * m1 + ci) / n1);
      u0[i] = (float)((bi * m0 + ci) / n0);  // weight m0 < 0, original order
      rowmap[s_] = i;
    }
    __syncthreads();
    ok = secular_cta<kTerms>(n, dhi, dlo, wv, rowmap, V, n, lhi, llo, nxt, s_sc, &s_flag);
    if (ok) {
      // Second update in the eigenbasis of the first: diag(lam) + m0 z z^T (z = Q1^T u0), solved
      // as -(diag(-lam) + |m0| z z^T); ascending poles -lam_{n-1}, ..., -lam_0.
      const float sm0 = (float)s_m[5];
      const int rot = gram_rot(n);
      for (int s_ = t; s_ < n; s_ += blockDim.x) {
        const int j = n - 1 - s_;
        float acc = 0.f;
        for (int i0 = 0; i0 < n; ++i0) {
          const int i = i0 + rot < n ? i0 + rot : i0 + rot - n;
          acc += V[(size_t)j * n + i] * u0[i];
        }
        wv[s_] = sm0 * acc;
        dhi[s_] = -lhi[j];
        dlo[s_] = -llo[j];
        rowmap[s_] = j;
      }
      __syncthreads();
      ok = secular_cta<kTerms>(n, dhi, dlo, wv, rowmap, B, n, lhi, llo, nxt, s_sc, &s_flag);
      if (ok) {
        smem_gemm_nn(n, V, B, W);  // Q1 Q2 into W (temporary)
        __syncthreads();
        for (int idx = t; idx < n * n; idx += blockDim.x) V[idx] = W[idx];
        __syncthreads();
      }
    }
  }
  if (!ok) return -1;
  ISVD_STAMP(3);
  // Verification (and at most one first-order polish): off(S) and |I - V^T V| below tolerance.
  const float tol = 8.f * Eps<float>::v * sqrtf((float)(nr > n ? nr : n));
  int pass = 0;
  // S = W^T W and Q = V^T V (R = I - Q): S into B, Q into the scratch area after W.
  float* Qm = kQGlobal ? gq : W + (size_t)(n + 1) * n;  // n x n
  for (; !ge; ++pass) {
    structured_kv(in, nr, n, V, W, tmp, sf, xf, bf, rhof);
    if (t < 2) s_max[t] = 0.f;
    if (KB > kFastCoreQSmemMaxKB) smem_two_syrk4(n, nr, W, V, B, Qm);
    else smem_two_syrk(n, nr, W, V, B, Qm);
    __syncthreads();
    float offm = 0.f, rm = 0.f;
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int a_ = idx / n, b_ = idx - a_ * n;
      const float q = Qm[idx];
      rm = fmaxf(rm, fabsf((a_ == b_ ? 1.f : 0.f) - q));
      if (a_ != b_) {
        const float den = sqrtf(B[(size_t)a_ * n + a_]) * sqrtf(B[(size_t)b_ * n + b_]);
        if (den > 0.f) offm = fmaxf(offm, __fdividef(fabsf(B[idx]), den));
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      offm = fmaxf(offm, __shfl_xor_sync(0xffffffffu, offm, o));
      rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    }
    if ((t & 31) == 0) {
      atomicMax(reinterpret_cast<int*>(&s_max[0]), __float_as_int(offm));
      atomicMax(reinterpret_cast<int*>(&s_max[1]), __float_as_int(rm));
    }
    __syncthreads();
    const float off_all = s_max[0], r_all = s_max[1];
    __syncthreads();
    if (off_all < tol && r_all < tol) break;
    if (pass >= 1 || !(off_all < 0.05f) || !(r_all < 0.05f)) {
      if (t == 0) *iters = -1;
      return -1;
    }
    // First-order correction V <- V + V E (Ogita-Aishima style refinement):
    //   lambda_i = S_ii / (1 - R_ii); E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) (i != j),
    //   E_ii = R_ii / 2.
    for (int idx = t; idx < n * n; idx += blockDim.x) {
      const int j = idx / n, i = idx - j * n;  // E_ij stored column-major in W: W[j * n + i]
      const float Rij = (i == j ? 1.f : 0.f) - Qm[(size_t)j * n + i];
      float e;
      if (i == j) {
        e = 0.5f * Rij;
      } else {
        const float Sij = B[(size_t)j * n + i];
        const float li = B[(size_t)i * n + i] / Qm[(size_t)i * n + i];
        const float lj = B[(size_t)j * n + j] / Qm[(size_t)j * n + j];
        const float gap = lj - li;
        e = (fabsf(gap) > 8.f * fabsf(Sij)) ? (Sij + lj * Rij) / gap : 0.5f * Rij;
      }
      W[(size_t)j * n + i] = e;
    }
    __syncthreads();
    // V + V E -> B, then copy back.
    smem_gemm_nn(n, V, W, B);
    __syncthreads();
    for (int idx = t; idx < n * n; idx += blockDim.x) V[idx] += B[idx];
    __syncthreads();
  }
  if (t == 0) *iters = ge ? 2 : pass;
  ISVD_STAMP(4);
  // W holds K V (Gram path) or the normalised left vectors (corrected-weight path). Column norms of W, and the singular values ||K v_j|| / ||v_j|| in
  // float-float arithmetic through K's structure (FP64-class accuracy on the FP32 pipes).
  const int lane = t & 31, warp = t >> 5;
  double* sref = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(nxt + n) + 15) & ~uintptr_t(15));
  double* nrm = sref + n;
  int* perm = reinterpret_cast<int*>(nrm + n);
  float* x_hi = dhi;  // p (append) or a (entry) as float pairs
  float* x_lo = dlo;
  float* b_hi = wv;
  float* b_lo = u0;
  for (int i = t; i < r; i += blockDim.x) {
    const ff xi = ff_of(in.kind == kEntry ? in.delta * in.a[i] : in.p[i]);
    x_hi[i] = xi.hi;
    x_lo[i] = xi.lo;
    if (in.kind == kEntry) {
      const ff bi = ff_of(in.b[i]);
      b_hi[i] = bi.hi;
      b_lo[i] = bi.lo;
    }
  }
  __syncthreads();
  __shared__ float s_rho[2];
  if (t == 0) {
    const ff q = ff_of(in.rho);
    s_rho[0] = q.hi;
    s_rho[1] = q.lo;
  }
  __syncthreads();
  const ff rho_ff{s_rho[0], s_rho[1]};
  float* acc_hi = vec + 10 * n;  // per-column ||K v||^2 and ||v||^2 as float pairs
  float* acc_lo = vec + 11 * n;
  float* nv_hi = vec + 12 * n;
  float* nv_lo = vec + 13 * n;
  float* inv_nrm = vec + 14 * n;  // 1 / ||W_j||  (declared again below for the output phase)
  {
    const int g = t & (kSecLanes - 1);
    const int ngr = blockDim.x / kSecLanes;
    const int rounds = (n + ngr - 1) / ngr;
    for (int rr = 0; rr < rounds; ++rr) {
      const int j = t / kSecLanes + rr * ngr;
      const bool live = j < n;
      const float* v = V + (size_t)(live ? j : 0) * n;
      float s2 = 0.f;
      ff nv{0.f, 0.f}, acc{0.f, 0.f}, dot{0.f, 0.f};
      if (live) {
        if (!ge)
          for (int row = g; row < nr; row += kSecLanes) s2 += W[(size_t)j * nr + row] * W[(size_t)j * nr + row];
        for (int i = g; i < n; i += kSecLanes) nv = ff_add(nv, two_prod(v[i], v[i]));
      }
      if (in.kind == kEntry) {
        if (live)
          for (int i = g; i < r; i += kSecLanes) dot = ff_add(dot, ff_mul_f(ff{b_hi[i], b_lo[i]}, v[i]));
        dot = ff_group_sum<kSecLanes>(dot);
        if (live) {
          for (int i = g; i < r; i += kSecLanes) {
            const ff sv = ff_mul_f(ff{sig_hi[i], sig_lo[i]}, v[i]);
            ff ad = two_prod(x_hi[i], dot.hi);
            ad.lo = fmaf(x_hi[i], dot.lo, fmaf(x_lo[i], dot.hi, ad.lo));
            acc = ff_add(acc, ff_sqr(ff_add(sv, ad)));
          }
        }
        acc = ff_group_sum<kSecLanes>(acc);
      } else {
        if (live) {
          for (int i = g; i < r; i += kSecLanes) {
            acc = ff_add(acc, ff_sqr(ff_mul_f(ff{sig_hi[i], sig_lo[i]}, v[i])));
            dot = ff_add(dot, ff_mul_f(ff{x_hi[i], x_lo[i]}, v[i]));
          }
        }
        acc = ff_group_sum<kSecLanes>(acc);
        dot = ff_group_sum<kSecLanes>(dot);
        const ff yr = in.grew ? ff_add(dot, ff_mul_f(rho_ff, live ? v[r] : 0.f)) : dot;
        acc = ff_add(acc, ff_sqr(yr));
      }
      nv = ff_group_sum<kSecLanes>(nv);
#pragma unroll
      for (int o = kSecLanes / 2; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (live && g == 0) {
        acc_hi[j] = acc.hi;
        acc_lo[j] = acc.lo;
        nv_hi[j] = nv.hi;
        nv_lo[j] = nv.lo;
        nrm[j] = ge ? 1.0 : (double)sqrtf(s2);
        inv_nrm[j] = ge ? 1.f : (s2 > 0.f ? rsqrtf(s2) : 0.f);
      }
    }
  }
  __syncthreads();
  if (warp == 0) {  // FP64 finish, one column per lane (vectorised, so few FP64 instructions)
    for (int j = lane; j < n; j += 32) {
      const double nvd = (double)nv_hi[j] + (double)nv_lo[j];
      const double ad = (double)acc_hi[j] + (double)acc_lo[j];
      sref[j] = nvd > 0.0 ? sqrt(fmax(ad, 0.0) / nvd) : 0.0;
    }
  }
  __syncthreads();
  ISVD_STAMP(5);
  // Descending order (ties by index) compared exactly as float pairs (no FP64 compares).
  float* key_hi = tmp;
  float* key_lo = lhi;
  for (int j = t; j < n; j += blockDim.x) {
    const ff kj = ff_of(sref[j]);
    key_hi[j] = kj.hi;
    key_lo[j] = kj.lo;
  }
  for (int j = t; j < n; j += blockDim.x) perm[j] = j;  // a NaN key can misorder, never index out of range
  __syncthreads();
  for (int j = t; j < n; j += blockDim.x) {
    const float hj = key_hi[j], lj = key_lo[j];
    int rank = 0;
    for (int l = 0; l < n; ++l) {
      const float hl = key_hi[l], ll = key_lo[l];
      rank += (hl > hj) || (hl == hj && (ll > lj || (ll == lj && l < j)));
    }
    perm[rank] = j;
  }
  __syncthreads();
  const int k_out = in.kt < nc ? in.kt : nc;
  // A kept singular value at the FP32 noise floor has no reliable left vector here (one warp,
  // FP32, on the reciprocal norms: small ||W_j|| <=> large 1 / ||W_j||).
  if (warp == 0 && ge && lane == 0) s_flag = 0;
  if (warp == 0 && !ge) {
    float mx = 0.f;
    for (int j = lane; j < n; j += 32) mx = fmaxf(mx, inv_nrm[j] > 0.f ? 1.f / inv_nrm[j] : 0.f);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int bad = 0;
    for (int jj = lane; jj < k_out; jj += 32) {
      const float nj = inv_nrm[perm[jj]] > 0.f ? 1.f / inv_nrm[perm[jj]] : 0.f;
      bad |= !(nj > mx * 1e-5f);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) s_flag = bad;
  }
  __syncthreads();
  if (s_flag) return -1;
  for (int idx = t; idx < nr * k_out; idx += blockDim.x) {
    const int row = idx / k_out, jj = idx - row * k_out;
    const int j = perm[jj];
    UK[(size_t)row * ldo + jj] = (T)(W[(size_t)j * nr + row] * inv_nrm[j]);
  }
  for (int idx = t; idx < nc * k_out; idx += blockDim.x) {
    const int row = idx / k_out, jj = idx - row * k_out;
    VKo[(size_t)row * ldo + jj] = (T)V[(size_t)perm[jj] * n + row];
  }
  __syncthreads();
  for (int jj = t; jj < k_out; jj += blockDim.x) sig_out[jj] = sref[perm[jj]];
  __syncthreads();
  ISVD_STAMP(6);
  return k_out;
}

}  // namespace isvd
