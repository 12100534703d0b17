// Batched row and column appends (Section 2.2) with ONE WARP per stream update, for streams of
// working-rank capacity up to 32.
//
// The CTA-per-update kernel (pool_kernels.cuh) spends most of its time in block barriers and in
// serial rounds of dependent loads, while its SM is shared with other CTAs doing the same. A warp
// holds everything an update of rank <= 32 needs: the projection side's rows stream through the
// lanes (one row per lane, a whole row in registers), reductions over rows are register
// transposes by shuffles, and the core - a rank-one modification of a diagonal matrix - is solved
// root-per-lane. There are no block barriers and the streams of a tick run in about one wave;
// one launch per rank bucket (8, 16, 32) keeps each kernel's code small enough for the
// instruction caches.
//
// Per update (P = the projection side: V for a row append, U for a column append; Q = the other
// side; x = the new row or column):
//   pass 1      p1 = P^T x, ||x||^2                       (FP32 products, float-float ||x||^2)
//   pass 2      z1 = x - P p1 (float-float per row), p2 = P^T z1, ||z1||^2     (CGS2, one read)
//               p = p1 + p2, rho^2 = ||z1||^2 - ||p2||^2, grew = rho > tol_rel ||x||
//   core        K = [[Sigma, 0], [p, rho]]: K^T K = diag(sigma^2, 0) + w w^T with w = (p, rho);
//               secular roots (one per lane, near-pole rational iteration with a bisection
//               safeguard, poles as float pairs), corrected weights w_hat (Gu-Eisenstat), and
//               both vector sets in closed form from w_hat (see ge_append_vectors); singular
//               values sqrt(lambda) in FP64
//   rotations   P' = [P z_hat] V_K with z_hat = (x - P p) / rho recomputed per row in float-float,
//               Q' = blkdiag(Q, 1) U_K (the new row of Q' is U_K's last row): a separate
//               row-parallel launch (k_pool_rotate in pool_rotate_tma.cuh, two rows per
//               thread) reading V_K, U_K and p from a per-update scratch record, since one warp
//               cannot hide the latency of rotating hundreds of rows.
// An update the warp cannot finish on this path (non-finite input, coinciding poles, a deflated
// rho pole, a rejected weight correction, an empty factorisation) changes nothing and is listed
// for the CTA kernel (k_pool_retry), which has the Jacobi fallback.
#pragma once

#include "core_fast.cuh"
#include "isvd_common.cuh"
#include "pool_kernels.cuh"

namespace isvd {

constexpr int kWarpKB = 32;         // largest rank bucket of the warp kernel
constexpr int kWarpsPerBlock = 4;   // independent warps per block (no block-level sync)

// Per-warp shared memory for rank bucket KB.
template <int KB>
struct alignas(16) WarpSmem {
  float RP[(KB + 1) * 32];  // V_K for P: row c (original order; row r = z_hat's), column jj, stride KB;
                            // during the root search, each lane's shifted poles (pole i at i * 32 + lane)
  float RQ[(KB + 1) * KB];  // U_K for Q: row c (row r = the new row), column jj, stride KB
  float dhi[KB + 1], dlo[KB + 1];  // ascending poles as float pairs
  float w[KB + 1];                 // weights in pole order
  float tau[KB + 1];               // root j = pole org[j] + tau[j]
  float lhi[KB + 1], llo[KB + 1];  // roots as float pairs
  float what[KB + 1];              // w^2 during the root search, then the corrected weights
  float ph[KB], pl[KB];            // p as float pairs (original order)
  float sf[KB];                    // sigma (float, original order)
  int org[KB + 1], row[KB + 1], perm[KB + 1];
};

template <int KB>
constexpr size_t warp_block_smem() {
  return sizeof(WarpSmem<KB>) * kWarpsPerBlock;
}

// What the warp kernel hands to the rotation kernel for one update (global scratch).
template <int KB>
struct alignas(16) RotScratch {
  float RP[(KB + 1) * KB];  // V_K (row stride KB), row r = z_hat's when the rank grew
  float RQ[(KB + 1) * KB];  // U_K (row stride KB)
  float p2[KB];             // p2 = P^T z1, the second projection pass (z = z1 - P p2)
  float inv_rho;
  int r, k_out, grew;       // k_out < 0: the update was handed to the CTA kernel
};
constexpr size_t kRotScratchStride = sizeof(RotScratch<kWarpKB>);  // bytes per update slot

// Warp-wide sums of KB per-lane vectors: returns, on lane L, sum over lanes of v[L % KB]. The
// first log2(KB) rounds exchange half of the remaining entries with the partner lane (a register
// transpose, KB - 1 shuffles), the rest add across lane groups.
template <int KB>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[KB], int lane) {
#pragma unroll
  for (int o = KB / 2; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float s = v[0];
#pragma unroll
  for (int o = KB; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Next non-deflated pole above j (bit set in mask), or -1.
__device__ __forceinline__ int warp_next_pole(uint64_t mask, int j) {
  const uint64_t m = j + 1 < 64 ? (mask >> (j + 1)) : 0ull;
  return m ? j + __ffsll((long long)m) : -1;
}

// One row or column append of one stream by the calling warp. Returns false, with nothing
// written, when the update has to take the CTA kernel instead.
template <int KB>
__device__ bool warp_append(const PoolOp& op, WarpSmem<KB>& S, RotScratch<KB>& RS) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  DevState* st = op.st;
  const int r = st->r;
  const int kt = st->k;
  const bool is_row = op.kind == kRow;
  float* P = is_row ? op.V : op.U;
  float* Q = is_row ? op.U : op.V;
  const int64_t nP = is_row ? op.n : op.m;
  const int64_t nQ = is_row ? op.m : op.n;
  const int64_t ld = op.ld;
  const float* x = op.x;
  if (r < 1 || r > KB || ld != KB) return false;
  ISVD_WSTAMP_INIT(tp);

  // The projection side row by row, one row per lane (rows lane, lane + 32, ...): a lane loads its
  // whole row (KB / 4 float4s; the next row's loads are issued before the current row is used), so
  // every row-wise quantity (the residual z1 in float-float) stays inside the lane, and column sums
  // over rows are per-lane accumulators reduced once at the end (a register transpose). Columns >= r
  // are zeroed (stale values beyond the working rank).
  constexpr int C4 = KB / 4;
  const float4* P4 = reinterpret_cast<const float4*>(P);
  auto load_row = [&](int64_t row, float (&v)[KB], float& xv) {
    const bool ok = row < nP;
#pragma unroll
    for (int q = 0; q < C4; ++q) {
      const float4 a = ok ? P4[row * C4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
      v[4 * q] = 4 * q < r ? a.x : 0.f;
      v[4 * q + 1] = 4 * q + 1 < r ? a.y : 0.f;
      v[4 * q + 2] = 4 * q + 2 < r ? a.z : 0.f;
      v[4 * q + 3] = 4 * q + 3 < r ? a.w : 0.f;
    }
    xv = ok ? x[row] : 0.f;
  };

  // Pass 1: p1 = P^T x and ||x||^2.
  float acc[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) acc[c] = 0.f;
  ff xx{0.f, 0.f};
  {
    float vn[KB], xn;
    load_row(lane, vn, xn);
    for (int64_t row0 = 0; row0 < nP; row0 += 32) {  // warp-uniform trip count
      float v[KB];
#pragma unroll
      for (int c = 0; c < KB; ++c) v[c] = vn[c];
      const float xv = xn;
      if (row0 + 32 < nP) load_row(row0 + 32 + lane, vn, xn);
#pragma unroll
      for (int c = 0; c < KB; ++c) acc[c] = fmaf(v[c], xv, acc[c]);
      xx = ff_add(xx, two_prod(xv, xv));
    }
  }
  const float p1v = warp_transpose_sum<KB>(acc, lane);  // column lane % KB
  xx = ff_group_sum<32>(xx);
  if (lane < KB) S.ph[lane] = lane < r ? p1v : 0.f;
  __syncwarp();
  ISVD_WSTAMP(17, tp);

  // Pass 2 (CGS2): z1 = x - P p1 per row (float-float, inside the row's lane), p2 = P^T z1, ||z1||^2.
  // z1 is also kept for the rotation's z_hat (op.z1).
#pragma unroll
  for (int c = 0; c < KB; ++c) acc[c] = 0.f;
  ff zz{0.f, 0.f};
  {
    float vn[KB], xn;
    load_row(lane, vn, xn);
    for (int64_t row0 = 0; row0 < nP; row0 += 32) {  // warp-uniform trip count
      float v[KB];
#pragma unroll
      for (int c = 0; c < KB; ++c) v[c] = vn[c];
      const float xv = xn;
      const int64_t row = row0 + lane;
      if (row0 + 32 < nP) load_row(row0 + 32 + lane, vn, xn);
      ff d0{0.f, 0.f}, d1{0.f, 0.f};  // two partial dot products (independent chains)
#pragma unroll
      for (int c = 0; c < KB; c += 2) {
        d0 = ff_add(d0, two_prod(v[c], S.ph[c]));
        d1 = ff_add(d1, two_prod(v[c + 1], S.ph[c + 1]));
      }
      const ff d = ff_add(d0, d1);
      const ff zrow = ff_add(ff{xv, 0.f}, ff{-d.hi, -d.lo});
      const float z1 = zrow.hi + zrow.lo;
      if (row < nP) op.z1[row] = z1;
#pragma unroll
      for (int c = 0; c < KB; ++c) acc[c] = fmaf(v[c], z1, acc[c]);
      zz = ff_add(zz, ff_sqr(zrow));
    }
  }
  const float p2v = warp_transpose_sum<KB>(acc, lane);
  zz = ff_group_sum<32>(zz);
  const float p1c_l = (lane < KB && lane < r) ? p1v : 0.f;  // p1[lane]
  const float p2c = (lane < KB && lane < r) ? p2v : 0.f;    // p2[lane]
  double pn = (double)p2c * (double)p2c;
  pn = warp_sum(pn);
  const double xn2 = (double)xx.hi + (double)xx.lo;
  const double rho2 = ((double)zz.hi + (double)zz.lo) - pn;
  ISVD_WSTAMP(18, tp);
  if (!isfinite(xn2) || !isfinite(rho2)) {
    ISVD_WCOUNT(25);
    return false;
  }
  const double rho = sqrt(fmax(rho2, 0.0));
  const double xnorm = sqrt(xn2);
  const bool grew = rho > op.tol_rel * xnorm;
  __syncwarp();
  if (lane < KB) {
    float hi, lo;
    two_sum(p1c_l, p2c, hi, lo);
    S.ph[lane] = lane < r ? hi : 0.f;
    S.pl[lane] = lane < r ? lo : 0.f;
  }
  __syncwarp();

  // Core setup: ascending poles (0 with weight rho when the rank grows), sigma_{r-1}^2 .. sigma_0^2.
  const int nc = grew ? r + 1 : r;
  const int off = grew ? 1 : 0;
  for (int s_ = lane; s_ < nc; s_ += 32) {
    if (grew && s_ == 0) {
      S.dhi[0] = 0.f;
      S.dlo[0] = 0.f;
      S.w[0] = (float)rho;
      S.row[0] = r;
    } else {
      const int i = r - 1 - (s_ - off);
      const double sg = op.sig[i];
      const ff d2 = ff_of(sg * sg);
      S.dhi[s_] = d2.hi;
      S.dlo[s_] = d2.lo;
      S.w[s_] = S.ph[i] + S.pl[i];
      S.row[s_] = i;
    }
  }
  for (int i = lane; i < r; i += 32) S.sf[i] = (float)op.sig[i];
  __syncwarp();
  ff wq{0.f, 0.f};
  for (int s_ = lane; s_ < nc; s_ += 32) wq = ff_add(wq, two_prod(S.w[s_], S.w[s_]));
  wq = ff_group_sum<32>(wq);
  const float wn2 = wq.hi + wq.lo;
  const float thr = 1e-7f * sqrtf(wn2);  // deflation: |w_j| <= thr counts as zero
  const float dscale = fmaxf(fabsf(S.dhi[0]), fabsf(S.dhi[nc - 1]));
  const bool nd0 = lane < nc && fabsf(S.w[lane]) > thr;
  const bool nd1 = lane + 32 < nc && fabsf(S.w[lane + 32]) > thr;
  const uint64_t mask = (uint64_t)__ballot_sync(kFull, nd0) | ((uint64_t)__ballot_sync(kFull, nd1) << 32);
  int bad = 0;
  float ws = 0.f;
  for (int j = lane; j < nc; j += 32) {
    const ff dj{S.dhi[j], S.dlo[j]};
    if (j + 1 < nc && ff_sub_to_f(ff{S.dhi[j + 1], S.dlo[j + 1]}, dj) < 0.f) bad |= 1;  // order
    if ((mask >> j) & 1ull) {
      const int nx = warp_next_pole(mask, j);
      if (nx >= 0 && ff_sub_to_f(ff{S.dhi[nx], S.dlo[nx]}, dj) <= kTieRel * dscale) bad |= 2;  // ties
      ws += S.w[j] * S.w[j];
      S.what[j] = S.w[j] * S.w[j];
    } else {
      S.what[j] = 0.f;
    }
  }
  if (grew && !(mask & 1ull)) bad |= 4;  // deflated rho pole
  if (mask == 0ull) bad |= 8;
  ws = warp_sum(ws) * (1.f + 1e-5f);
  bad = __reduce_or_sync(kFull, bad);
  if (bad) {
    if (bad & 1) ISVD_WCOUNT(26);
    if (bad & 2) ISVD_WCOUNT(27);
    if (bad & 4) ISVD_WCOUNT(28);
    if (bad & 8) ISVD_WCOUNT(29);
    return false;
  }
  __syncwarp();
  ISVD_WSTAMP(19, tp);

  // Roots, one per lane: lambda_j in (d_j, d_next) (the last one in (d_last, d_last + ||w||^2)),
  // in the offset u from the nearer pole. The lane's poles shifted to the origin live in RP
  // (column = lane) while it searches.
  float* sh = S.RP;
  const int nc32 = nc < 32 ? nc : 32;  // roots 0..31 one per lane; root 32 (nc = 33) by the whole warp below
  for (int j = lane; j < nc32; j += 32) {
    if (!((mask >> j) & 1ull)) {
      S.tau[j] = 0.f;
      S.org[j] = j;
      S.lhi[j] = S.dhi[j];
      S.llo[j] = S.dlo[j];
      continue;
    }
    const int nx = warp_next_pole(mask, j);
    const bool last = nx < 0;
    const ff lo{S.dhi[j], S.dlo[j]};
    const ff hi = last ? lo : ff{S.dhi[nx], S.dlo[nx]};
    const float width = last ? ws : ff_sub_to_f(hi, lo);
    const float half = 0.5f * width;
    float fm = 1.f;
    for (int i = 0; i < nc; ++i) {
      const float di = S.what[i] > 0.f ? ff_sub_to_f(ff{S.dhi[i], S.dlo[i]}, lo) : 1e30f;
      sh[i * 32 + lane] = di;
      fm += __fdividef(S.what[i], di - half);
    }
    float sgn = 1.f, b = last ? width : half;
    int o = j;
    if (!last && !(fm > 0.f)) {
      sgn = -1.f;
      b = half;
      o = nx;
      for (int i = 0; i < nc; ++i)
        sh[i * 32 + lane] = S.what[i] > 0.f ? ff_sub_to_f(ff{S.dhi[i], S.dlo[i]}, hi) : 1e30f;
    }
    // h(u) = sgn f(sgn u) rises from -inf at the near pole (u = 0); each step fits
    // h ~ C - S/u to h and h' at u and takes its root, or bisects (geometrically across decades).
    float a = 0.f, u = 0.5f * b;
    for (int it = 0; it < 40; ++it) {
      const float tk = sgn * u;
      float fs = 0.f, ds = 0.f;
      for (int i = 0; i < nc; ++i) {
        const float rq = __fdividef(1.f, sh[i * 32 + lane] - tk);
        const float t1 = S.what[i] * rq;
        fs += t1;
        ds = fmaf(t1, rq, ds);
      }
      const float h = sgn * (1.f + fs);
      if (h == 0.f) break;
      if (h < 0.f) a = u;
      else b = u;
      const float C = h + ds * u;
      float un = (C > 0.f) ? ds * u * u / C : -1.f;
      if (!(un > a && un < b)) un = (a > 0.f && b > 4.f * a) ? sqrtf(a) * sqrtf(b) : 0.5f * (a + b);
      const bool done = fabsf(un - u) <= 1e-7f * un || (b - a) <= 2.4e-7f * b;
      u = un;
      if (done) break;
    }
    const float tau = sgn * u;
    const ff og{S.dhi[o], S.dlo[o]};
    const ff lam = ff_add(og, ff{tau, 0.f});
    S.tau[j] = tau;
    S.org[j] = o;
    S.lhi[j] = lam.hi;
    S.llo[j] = lam.lo;
  }
  if (nc > 32) {
    // Root 32, the largest (above the last pole, nothing above it), by the whole warp: the same
    // iteration as above with the secular sums split over the lanes (pole i on lane i, pole 32 on
    // lane 0) and reduced by shuffles, so every lane runs the identical scalar update.
    const int j = 32;
    if (!((mask >> j) & 1ull)) {
      if (lane == 0) {
        S.tau[j] = 0.f;
        S.org[j] = j;
        S.lhi[j] = S.dhi[j];
        S.llo[j] = S.dlo[j];
      }
    } else {
      const ff lo{S.dhi[j], S.dlo[j]};
      const float d_a = S.what[lane] > 0.f ? ff_sub_to_f(ff{S.dhi[lane], S.dlo[lane]}, lo) : 1e30f;
      const float w_a = S.what[lane];
      const float d_b = lane == 0 && S.what[32] > 0.f ? ff_sub_to_f(ff{S.dhi[32], S.dlo[32]}, lo) : 1e30f;
      const float w_b = lane == 0 ? S.what[32] : 0.f;
      float a = 0.f, b = ws, u = 0.5f * ws;
      for (int it = 0; it < 40; ++it) {
        float rq = __fdividef(1.f, d_a - u);
        float t1 = w_a * rq;
        float fs = t1, ds = t1 * rq;
        rq = __fdividef(1.f, d_b - u);
        t1 = w_b * rq;
        fs += t1;
        ds = fmaf(t1, rq, ds);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fs += __shfl_xor_sync(kFull, fs, o);
          ds += __shfl_xor_sync(kFull, ds, o);
        }
        fs = __shfl_sync(kFull, fs, 0);  // lane 0's sums everywhere: bit-identical control flow
        ds = __shfl_sync(kFull, ds, 0);
        const float h = 1.f + fs;
        if (h == 0.f) break;
        if (h < 0.f) a = u;
        else b = u;
        const float C = h + ds * u;
        float un = (C > 0.f) ? ds * u * u / C : -1.f;
        if (!(un > a && un < b)) un = (a > 0.f && b > 4.f * a) ? sqrtf(a) * sqrtf(b) : 0.5f * (a + b);
        const bool done = fabsf(un - u) <= 1e-7f * un || (b - a) <= 2.4e-7f * b;
        u = un;
        if (done) break;
      }
      if (lane == 0) {
        const ff lam = ff_add(lo, ff{u, 0.f});
        S.tau[j] = u;
        S.org[j] = j;
        S.lhi[j] = lam.hi;
        S.llo[j] = lam.lo;
      }
    }
  }
  __syncwarp();
  ISVD_WSTAMP(20, tp);

  // Corrected weights: w_hat_i^2 = prod_j (lambda_j - d_i) / prod_{l != i} (d_l - d_i), each
  // root paired with its neighbouring pole; rejected when |w_hat - w| > kGeTolEps eps ||w||.
  const float tol = kGeTolEps * Eps<float>::v * sqrtf(wn2);
  int badge = 0;
  for (int i = lane; i < nc32; i += 32) {
    float wh = 0.f;
    if ((mask >> i) & 1ull) {
      const ff di{S.dhi[i], S.dlo[i]};
      float prod = 1.f;
      for (int j = 0; j < nc; ++j) {
        if (!((mask >> j) & 1ull)) continue;
        const int o = S.org[j];
        const float num = ff_sub_to_f(ff{S.dhi[o], S.dlo[o]}, di) + S.tau[j];
        const int nj = warp_next_pole(mask, j);
        if (nj < 0) {
          prod *= num;
        } else {
          const int pj = j < i ? j : nj;
          prod *= __fdividef(num, ff_sub_to_f(ff{S.dhi[pj], S.dlo[pj]}, di));
        }
      }
      wh = copysignf(sqrtf(fmaxf(prod, 0.f)), S.w[i]);
      if (!(fabsf(wh - S.w[i]) <= tol)) badge = 1;
    }
    S.what[i] = wh;
  }
  if (nc > 32) {
    // w_hat_32 by the whole warp: factor j on lane j (and j = 32 on lane 0), a product butterfly.
    const int i = 32;
    const bool live = (mask >> i) & 1ull;
    const ff di{S.dhi[i], S.dlo[i]};
    auto factor = [&](int j) -> float {
      if (!((mask >> j) & 1ull)) return 1.f;
      const int o = S.org[j];
      const float num = ff_sub_to_f(ff{S.dhi[o], S.dlo[o]}, di) + S.tau[j];
      const int nj = warp_next_pole(mask, j);
      if (nj < 0) return num;
      const int pj = j < i ? j : nj;
      return __fdividef(num, ff_sub_to_f(ff{S.dhi[pj], S.dlo[pj]}, di));
    };
    float prod = live ? factor(lane) * (lane == 0 ? factor(32) : 1.f) : 1.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) prod *= __shfl_xor_sync(kFull, prod, o);
    prod = __shfl_sync(kFull, prod, 0);
    __syncwarp();
    if (lane == 0) {
      float wh = 0.f;
      if (live) {
        wh = copysignf(sqrtf(fmaxf(prod, 0.f)), S.w[i]);
        if (!(fabsf(wh - S.w[i]) <= tol)) badge = 1;
      }
      S.what[i] = wh;
    }
  }
  if (__any_sync(kFull, badge)) {
    ISVD_WCOUNT(30);
    return false;
  }

  // Descending order of the roots (compared as float pairs, ties by index). Every slot must be
  // filled exactly once; anything else (a NaN root) hands the update back.
  for (int j = lane; j < nc; j += 32) S.perm[j] = -1;
  __syncwarp();
  for (int j = lane; j < nc32; j += 32) {
    const float hj = S.lhi[j], lj = S.llo[j];
    int rk = 0;
    for (int l = 0; l < nc; ++l) {
      const float hl = S.lhi[l], ll = S.llo[l];
      rk += (hl > hj) || (hl == hj && (ll > lj || (ll == lj && l < j)));
    }
    if (rk < nc) S.perm[rk] = j;
  }
  if (nc > 32) {
    // rank of root 32 by the whole warp: lane l compares root l (root 32 never outranks itself)
    const int j = 32;
    const float hj = S.lhi[j], lj = S.llo[j];
    const float hl = S.lhi[lane], ll = S.llo[lane];
    const bool beats = (hl > hj) || (hl == hj && (ll > lj || (ll == lj && lane < j)));
    const int rk = __popc(__ballot_sync(kFull, beats));
    if (lane == 0 && rk < nc) S.perm[rk] = j;
  }
  __syncwarp();
  int unset = 0;
  for (int j = lane; j < nc; j += 32) unset |= S.perm[j] < 0;
  if (__any_sync(kFull, unset)) return false;
  const int k_out = kt < nc ? kt : nc;
  ISVD_WSTAMP(21, tp);

  // Vectors of output column jj = lane: v_j = (w_hat_i / (d_i - lambda_j))_i / norm into RP,
  // u_j = (sigma_i v_ji ; -1) / norm into RQ; a deflated pole keeps e_j on both sides.
  if (lane < k_out) {
    const int jj = lane, j = S.perm[jj];
    if (!((mask >> j) & 1ull)) {
      const int cj = S.row[j];
      for (int c = 0; c < nc; ++c) S.RP[c * KB + jj] = c == cj ? 1.f : 0.f;
      for (int c = 0; c <= r; ++c) S.RQ[c * KB + jj] = c == cj ? 1.f : 0.f;
    } else {
      const int o = S.org[j];
      const ff dor{S.dhi[o], S.dlo[o]};
      const float tj = S.tau[j];
      float sv = 0.f, su = 0.f;
      for (int i = 0; i < nc; ++i) {
        const int c = S.row[i];
        const float wh = S.what[i];
        const float v = wh != 0.f ? -wh / (ff_sub_to_f(dor, ff{S.dhi[i], S.dlo[i]}) + tj) : 0.f;
        S.RP[c * KB + jj] = v;
        sv = fmaf(v, v, sv);
        if (c < r) {
          const float uv = S.sf[c] * v;
          su = fmaf(uv, uv, su);
        }
      }
      const float iv = rsqrtf(sv), iu = rsqrtf(su + 1.f);
      for (int c = 0; c < nc; ++c) {
        const float v = S.RP[c * KB + jj];
        if (c < r) S.RQ[c * KB + jj] = S.sf[c] * v * iu;
        S.RP[c * KB + jj] = v * iv;
      }
      S.RQ[r * KB + jj] = -iu;
    }
    op.sig[jj] = sqrt((double)S.lhi[j] + (double)S.llo[j]);
  }
  __syncwarp();

  ISVD_WSTAMP(22, tp);
  // Hand V_K, U_K and p to the rotation kernel (rows beyond r zero: it sums over all KB rows);
  // the new row of Q is U_K's last row.
  for (int idx = lane; idx < (KB + 1) * KB; idx += 32) {
    const bool in = idx < (r + 1) * KB;
    RS.RP[idx] = in ? S.RP[idx] : 0.f;
    RS.RQ[idx] = in ? S.RQ[idx] : 0.f;
  }
  if (lane < KB) RS.p2[lane] = p2c;  // zero beyond r
  if (lane == 0) {
    RS.inv_rho = grew ? (float)(1.0 / rho) : 0.f;
    RS.r = r;
    RS.k_out = k_out;
    RS.grew = grew ? 1 : 0;
  }
  if (lane < k_out) Q[nQ * ld + lane] = S.RQ[r * KB + lane];
  // The dense matrix gains x as its new row / column.
  for (int64_t c = lane; c < nP; c += 32) {
    if (is_row) op.A[op.m * op.lda + c] = x[c];
    else op.A[c * op.lda + op.n] = x[c];
  }
  // Successive-subspace angles: squared norms of the kept rows r of U_K and V_K (warp sums).
  float cq = 0.f, cp = 0.f;
  if (k_out <= r && lane < k_out) {
    const float a = S.RQ[r * KB + lane], b = grew ? S.RP[r * KB + lane] : 0.f;
    cq = a * a;
    cp = b * b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cq += __shfl_xor_sync(kFull, cq, o);
    cp += __shfl_xor_sync(kFull, cp, o);
  }
  if (lane == 0) {
    st->rho = rho;
    st->grew = grew ? 1 : 0;
    st->novelty = xnorm > 0.0 ? rho / xnorm : 0.0;
    st->xnorm2 = xn2;
    st->N += xn2;
    st->r_in = r;
    st->k_out = k_out;
    st->r = k_out;
    st->sweeps = 102;
    append_signals_sums<float>(st, is_row, cq, cp, grew, kt);
  }
  ISVD_WSTAMP(23, tp);
  return true;
}

// ops[0 .. count): row/column appends of streams in rank bucket KB, one warp each. Updates that
// need the CTA kernel are listed in retry[] as base + index (count in *retry_n), untouched.
// Also fills block_op[chunk_start[e] + i] = e for the update's rotation blocks (rot_rows rows of
// one side per block: 256 for the FP32-pipe rotation, 128 for the tensor-core one), checking that
// they fall inside the run's table of nblocks entries (else the pool's check word gets code 6).
constexpr int kPoolRotThreads = 128;
constexpr int kPoolRotRows = 2 * kPoolRotThreads;  // rows per rotation block (two per thread)
template <int KB>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, KB <= 8 ? 6 : KB <= 16 ? 5 : 3)
    k_pool_warp(const PoolOp* __restrict__ ops, int count, int base, int* __restrict__ retry,
                int* __restrict__ retry_n, RotScratch<KB>* __restrict__ scratch, const int* __restrict__ chunk_start,
                int* __restrict__ block_op, int rot_rows, int nblocks, int* __restrict__ kcheck) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wid = threadIdx.x >> 5;
  const int e = blockIdx.x * kWarpsPerBlock + wid;
  if (e >= count) return;
  WarpSmem<KB>& S = reinterpret_cast<WarpSmem<KB>*>(smem)[wid];
  const PoolOp op = ops[e];
  {
    const int64_t nP = op.kind == kRow ? op.n : op.m, nQ = op.kind == kRow ? op.m : op.n;
    const int nb = (int)((nP + rot_rows - 1) / rot_rows + (nQ + rot_rows - 1) / rot_rows);
    const int c0 = chunk_start[e];
    if (c0 < 0 || c0 + nb > nblocks) {  // self-check: the host's table sizes disagree with the shapes
      if ((threadIdx.x & 31) == 0 && atomicCAS(&kcheck[0], 0, 6) == 0) kcheck[1] = e;
    } else {
      for (int i = threadIdx.x & 31; i < nb; i += 32) block_op[c0 + i] = e;
    }
  }
  const bool ok = warp_append<KB>(op, S, scratch[e]);
  if (!ok && (threadIdx.x & 31) == 0) {
    scratch[e].k_out = -1;
    retry[atomicAdd(retry_n, 1)] = base + e;
  }
}

}  // namespace isvd
