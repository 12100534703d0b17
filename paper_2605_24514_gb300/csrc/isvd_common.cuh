// Shared device-side definitions of libisvd (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace isvd {

// Largest supported working-rank capacity (columns of U and V).
constexpr int kKmaxLimit = 128;
// Partial-sum slots per projection pass (blocks of the projection kernels).
constexpr int kMaxProjBlocks = 256;

// Sticky device status bits (mapped to isvd_status on the host).
constexpr int kStNotConv = 1;
constexpr int kStNonFinite = 2;
constexpr int kStTimeout = 4;
constexpr int kStLayout = 8;  // a kernel's shared-memory layout did not fit its launch (nothing done)

// Update kinds (Section 2.1).
constexpr int kRow = 0;
constexpr int kCol = 1;
constexpr int kEntry = 2;
// Entry update in the rank-increasing form (the core gains the two residual directions); core
// kernels only, never a pool op kind.
constexpr int kEntryX = 3;

// Device-resident scalar state of one stream; read and written only by kernels, so a
// sequence of updates needs no host round trip.
struct DevState {
  int32_t r;          // maintained rank r_t
  int32_t k;          // working rank k_t
  int32_t status;     // sticky error bits
  int32_t grew;       // last append kept its new direction (rho > tol)
  int32_t r_in;       // rank before the last core SVD
  int32_t k_out;      // rank after it
  int32_t sweeps;     // Jacobi sweeps of the last core SVD
  int32_t defer_rows; // deferred rotations: columns of the stored U0, V0 (rows of R_U, R_V)
  double N;           // N_t = ||A_t||_F^2
  double xnorm2;      // ||x||^2 of the last append
  double rho;         // residual norm of the last append
  double novelty;     // rho / ||x||
  unsigned int counter;   // last-block-done counter of the projection kernels
  unsigned int pad1;
  // Loss-of-orthogonality monitor of the batched path: max|U^T U - I|, max|V^T V - I| at its last
  // run and the re-orthogonalisations it performed.
  double orth_u;
  double orth_v;
  int32_t reorths;
  int32_t orth_runs;
  // Local angular signals of the last update (Section 3.3): the largest principal angle between
  // span(U_{t-1}) and span(U_t), and between span(V_{t-1}) and span(V_t).
  double ang_u;
  double ang_v;
  // Novelty rank rule (Eq. novelty-rank-rule): after an append with rho > eta_nov ||x||,
  // k <- min(k + 1, kcap_nov) for the next update; kcap_nov = 0: off.
  double eta_nov;
  int32_t kcap_nov;
  int32_t pad2;
};

// The successive-subspace angles of an append from its core factors, and the novelty rule.
// QK: the factor of the side that gained the new row (U_K for a row append), PK: the side that
// gained z_hat (V_K), both with row stride ld, row r the new row / z_hat's; the kept columns are
// 0 .. k_out - 1. With [B; c^T] the kept block of an orthogonal factor (B its first r rows),
// B^T B = I - c c^T, so the cosines of the principal angles between the old span (extended by a
// zero row) and the new one are 1 but one, sqrt(1 - ||c||^2), when k_out <= r; when k_out > r the
// old span lies inside the new one. The side that gained no direction keeps its span.
// The sums and the arcsine run in the factors' own precision (T). append_signals_sums takes the
// squared norms ||c||^2 of the two kept rows already summed (zero when k_out > r).
template <typename T>
__device__ inline void append_signals_sums(DevState* st, bool kind_row, T cq, T cp, bool grew, int kt) {
  const T one = T(1);
  const T aq = asin(sqrt(cq) < one ? sqrt(cq) : one), ap = grew ? asin(sqrt(cp) < one ? sqrt(cp) : one) : T(0);
  st->ang_u = (double)(kind_row ? aq : ap);
  st->ang_v = (double)(kind_row ? ap : aq);
  if (st->kcap_nov > 0 && st->novelty > st->eta_nov) st->k = min(kt + 1, st->kcap_nov);
}
template <typename T>
__device__ inline void append_signals(DevState* st, bool kind_row, const T* QK, const T* PK, int64_t ld, int r,
                                      int k_out, bool grew, int kt) {
  T cq = T(0), cp = T(0);
  if (k_out <= r) {
    for (int j = 0; j < k_out; ++j) {
      const T a = QK[(int64_t)r * ld + j];
      cq += a * a;
      if (grew) {
        const T b = PK[(int64_t)r * ld + j];
        cp += b * b;
      }
    }
  }
  append_signals_sums<T>(st, kind_row, cq, cp, grew, kt);
}

// Optional phase timing (compile with -DISVD_CORE_TIMING): thread 0 of each CTA stores its
// clock64() stamp i into isvd_core_clock[i] and adds it to isvd_core_clock_sum[i], so that for
// many CTAs (sum[b] - sum[a]) / CTAs is the mean time between stamps a and b. Stamps 0-15 are
// the core's, 16-31 the pool tick's.
#ifdef ISVD_CORE_TIMING
__device__ long long isvd_core_clock[32];
__device__ unsigned long long isvd_core_clock_sum[32];
#define ISVD_STAMP(i)                                                              \
  do {                                                                             \
    __syncthreads();                                                               \
    if (threadIdx.x == 0) {                                                        \
      const long long c_ = clock64();                                              \
      isvd_core_clock[(i)] = c_;                                                   \
      atomicAdd(&isvd_core_clock_sum[(i)], (unsigned long long)c_);               \
    }                                                                              \
  } while (0)
// Warp-level phase timing: lane 0 adds the cycles since the warp's previous stamp to
// isvd_core_clock_sum[i] and counts the hit in isvd_core_clock_cnt[i].
__device__ unsigned long long isvd_core_clock_cnt[32];
#define ISVD_WSTAMP_INIT(tp) long long tp = clock64()
#define ISVD_WSTAMP(i, tp)                                                         \
  do {                                                                             \
    const long long c_ = clock64();                                                \
    if ((threadIdx.x & 31) == 0) {                                                 \
      atomicAdd(&isvd_core_clock_sum[(i)], (unsigned long long)(c_ - (tp)));       \
      atomicAdd(&isvd_core_clock_cnt[(i)], 1ull);                                  \
    }                                                                              \
    (tp) = c_;                                                                     \
  } while (0)
#define ISVD_WCOUNT(i)                                                               \
  do {                                                                               \
    if ((threadIdx.x & 31) == 0) atomicAdd(&isvd_core_clock_cnt[(i)], 1ull);       \
  } while (0)
#else
#define ISVD_WCOUNT(i) \
  do {                 \
  } while (0)
#define ISVD_STAMP(i) \
  do {                \
  } while (0)
#define ISVD_WSTAMP_INIT(tp) \
  do {                       \
  } while (0)
#define ISVD_WSTAMP(i, tp) \
  do {                     \
  } while (0)
#endif

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T half_sum(T v) {  // sum over aligned groups of 16 lanes
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 5.9604645e-8f; };
template <> struct Eps<double> { static constexpr double v = 1.1102230246251565e-16; };

__device__ __forceinline__ bool is_finite_d(double x) { return isfinite(x); }

}  // namespace isvd
