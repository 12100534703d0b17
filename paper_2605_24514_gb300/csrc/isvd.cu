// libisvd host side: the C ABI declared in include/isvd.h.
//
// One handle = one stream of updates on one GPU. Device state (U, V, A, sigma, N_t, rank) is
// resident in HBM and only kernels touch it, so consecutive updates queue back to back on the
// handle's CUDA stream with no host round trip; the host synchronises only for metrics, policy
// checks and explicit reads.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda.h>

#include "../../include/isvd.h"
#include "launch.cuh"
#include "pool_kernels.cuh"
#include "pool_reorth.cuh"
#include "pool_warp.cuh"
#include "refresh_kernels.cuh"
#include "update_kernels.cuh"

using namespace isvd;

struct isvd_ctx {
  // Fields a batched submit reads or advances for every op, packed into the first two cache
  // lines (a pool touches thousands of these per tick).
  int64_t m = 0, n = 0, t = 0, row_cap = 0, col_cap = 0;
  int kmax = 0, ld = 0;
  double tol_rel = 1e-10;
  void* U = nullptr;
  void* V = nullptr;
  void* A = nullptr;
  DevState* st = nullptr;
  double* sig = nullptr;
  int sticky = ISVD_OK;
  int prec = ISVD_FP64;
  size_t es = 8;
  int dev = 0;
  cudaStream_t stream = nullptr;
  int k_host = 0;
  double orth_tol = 1e-12;
  int64_t orth_every = 0, since_orth = 0;
  int orth_on_device = 0;  // the batched path's monitor (DevState orth_u/v, reorths) runs this stream
  int64_t since_rank = 0;  // the batched path's adaptive-rank cadence
  // finance layer scratch: weights (n, storage type) and the r x r Grams / vectors (FP64)
  void* wbuf = nullptr;
  int64_t wbuf_cap = 0;
  double* riskbuf = nullptr;
  int64_t risk_cap = 0;
  void* Uref = nullptr;
  int64_t m_ref = 0, uref_cap = 0;
  int r_ref = 0;
  double* p = nullptr;
  double* px = nullptr;  // rank-increasing entry update: p, q (stride kKmaxLimit + 2), alpha, beta
  // Deferred rotations (isvd_set_deferred_rotations): U = U0 R_U, V = V0 R_V with R_U, R_V kmax x ld
  // in the storage type; pending: entry updates have been applied to R_U, R_V and not yet to U, V.
  void* RU = nullptr;
  void* RV = nullptr;
  int defer = 0, defer_pending = 0;
  float* gq = nullptr;  // (kKmaxLimit + 1)^2 floats: the 128-bucket fast core's Gram matrix
  double* part = nullptr;
  void* UK = nullptr;
  void* VK = nullptr;
  void* xbuf = nullptr;
  int64_t xbuf_cap = 0;
  // refresh / metrics workspace
  double* G = nullptr;
  int64_t G_cap = 0;
  double* small = nullptr;  // several (kKmaxLimit+1)^2 FP64 scratch matrices
  double* evals = nullptr;
  double* inv = nullptr;
  double* scal = nullptr;  // scalars: [0] E_inc^2, [1] tail, [2] max offident, ...
  int* info = nullptr;
  void* Rtmp = nullptr;
  void* Uopt = nullptr;
  int64_t uopt_cap = 0;
  void* Vopt = nullptr;
  int64_t vopt_cap = 0;
  double* sig_opt = nullptr;
  double* Cbuf = nullptr;
  int64_t cbuf_cap = 0;
  // randomized refresh workspace
  void* Yb = nullptr;
  int64_t yb_cap = 0;
  void* Om = nullptr;
  int64_t om_cap = 0;
  double* Zd = nullptr;
  int64_t zd_cap = 0;
  void* Rl = nullptr;
  int64_t rl_cap = 0;
  int rsvd_p = 16, rsvd_q = 2;
  int64_t opt_t = -1;  // t at which Uopt/Vopt/sig_opt hold the truncated SVD of A_t
  int opt_rank = 0;
  uint64_t seed = 0;
  int64_t rsvd_calls = 0;
  isvd_policy pol{};
  int has_pol = 0;
  int64_t t_last = 0, refreshes = 0, reorths = 0, launches = 0;
  double orth_err_u = 0, orth_err_v = 0;
  isvd_metrics_t last_check{};
  std::string err;
  // profiling (events around launches; per-update stamps)
  int prof = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Span {
    int cls;
    size_t a, b;
    double bytes;
  };
  std::vector<Span> spans;
  std::vector<size_t> stamps;  // event index at the end of each update
  int cur_cls = -1;
  size_t cur_a = 0;
  double cur_bytes = 0;
  double cls_ms[ISVD_NUM_KCLASS] = {0};
  double cls_bytes[ISVD_NUM_KCLASS] = {0};
  int64_t cls_n[ISVD_NUM_KCLASS] = {0};
  std::vector<double> lat_us;
};

namespace {

constexpr int kSmall = (kKmaxLimit + 1) * (kKmaxLimit + 1);

// ---- profiling helpers ----------------------------------------------------------------------

size_t prof_event(isvd_ctx* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  cudaEventRecord(h->ev_pool[h->ev_used], h->stream);
  return h->ev_used++;
}

// Marks the start of a launch of kernel class cls moving `bytes` algorithmic bytes.
void prof_begin(isvd_ctx* h, int cls, double bytes) {
  if (!h->prof) return;
  h->cur_cls = cls;
  h->cur_a = prof_event(h);
  h->cur_bytes = bytes;
}

void prof_end(isvd_ctx* h) {
  if (!h->prof || h->cur_cls < 0) return;
  const size_t b = prof_event(h);
  h->spans.push_back({h->cur_cls, h->cur_a, b, h->cur_bytes});
  h->cur_cls = -1;
}

void prof_stamp(isvd_ctx* h) {
  if (!h->prof) return;
  h->stamps.push_back(prof_event(h));
}

// Resolves recorded events into per-class totals and per-update latencies (synchronises).
void prof_flush(isvd_ctx* h) {
  if (h->ev_used == 0) return;
  cudaEventSynchronize(h->ev_pool[h->ev_used - 1]);
  for (const auto& sp : h->spans) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev_pool[sp.a], h->ev_pool[sp.b]);
    h->cls_ms[sp.cls] += ms;
    h->cls_bytes[sp.cls] += sp.bytes;
    h->cls_n[sp.cls] += 1;
  }
  for (size_t i = 1; i < h->stamps.size(); ++i) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev_pool[h->stamps[i - 1]], h->ev_pool[h->stamps[i]]);
    h->lat_us.push_back(ms * 1e3);
  }
  size_t keep = h->stamps.empty() ? 0 : h->stamps.back();
  h->spans.clear();
  if (!h->stamps.empty()) {
    // keep the last stamp as the origin of the next update's latency
    std::swap(h->ev_pool[0], h->ev_pool[keep]);
    h->stamps.assign(1, 0);
    h->ev_used = 1;
  } else {
    h->ev_used = 0;
  }
}

isvd_status fail(isvd_ctx* h, isvd_status s, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (s == ISVD_ECUDA || s == ISVD_ENOTCONV || s == ISVD_ENONFINITE || s == ISVD_ETIMEOUT) h->sticky = s;
  }
  return s;
}

#define CK(h, x)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return fail((h), ISVD_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));      \
  } while (0)

#define CKL(h)                                                                            \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      return fail((h), ISVD_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    (h)->launches++;                                                                      \
  } while (0)

int kb_bucket(int k) { return k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128; }
int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <typename T>
size_t core_kernel_smem(int kmax) {
  size_t b = core_smem_bytes<T>(kmax);
  if (sizeof(T) == sizeof(float) && kb_bucket(kmax) <= kFastCoreMaxKB) b = std::max(b, core_fast_smem_bytes<T>(kmax));
  return 2 * (kKmaxLimit + 1) * sizeof(double) + b;
}

int core_threads(int kmax) {
  // Enough 8-lane groups for one root per group in the secular solver (kmax + 1 roots), which
  // also covers the Jacobi pairs; capped by the kernel's launch bound.
  const int nc = kmax + 1;
  int warps = (nc * kSecLanes + 31) / 32;
  const int cap = core_max_threads(kb_bucket(kmax)) / 32;
  warps = std::max(2, std::min(cap, warps));
  return warps * 32;
}

// True iff no element is Inf or NaN. Those are exactly the IEEE values whose exponent field is all
// ones, so the scan tests that field branch-free over fixed-size blocks (a constant trip count the
// host compiler vectorises at -O2) and stops after the first block holding a non-finite value.
template <typename T>
bool host_finite(const T* v, int64_t len) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "float or double");
  using B = typename std::conditional<sizeof(T) == 4, uint32_t, uint64_t>::type;
  constexpr B kExp = sizeof(T) == 4 ? (B)0x7f800000u : (B)0x7ff0000000000000ull;
  constexpr int64_t kBlock = 4096;
  int64_t b = 0;
  for (; b + kBlock <= len; b += kBlock) {
    B bad = 0;
    for (int64_t i = 0; i < kBlock; ++i) {
      B u;
      std::memcpy(&u, v + b + i, sizeof u);
      bad |= (B)((u & kExp) == kExp);
    }
    if (bad) return false;
  }
  B bad = 0;
  for (; b < len; ++b) {
    B u;
    std::memcpy(&u, v + b, sizeof u);
    bad |= (B)((u & kExp) == kExp);
  }
  return bad == 0;
}

// One launch of the core SVD kernel (single CTA), templated on the rank bucket.
template <typename T>
isvd_status launch_core(isvd_ctx* h, int kind, int64_t i, int64_t j, double delta) {
  const size_t cs = core_kernel_smem<T>(h->kmax);
  const int th = core_threads(h->kmax);
  const bool via_r = kind == kEntry && h->defer_pending;
  CK(h, core_launch<T>(kb_bucket(h->kmax), th, cs, h->stream, kind, h->st, h->sig, h->p, (T*)h->U, (T*)h->V, h->ld, i,
                       j, delta, (T*)h->A, h->col_cap, (T*)h->UK, (T*)h->VK, h->ld, h->px, h->tol_rel,
                       via_r ? (const T*)h->RU : nullptr, via_r ? (const T*)h->RV : nullptr, h->ld, h->gq));
  CKL(h);
  return ISVD_OK;
}

template <typename T, int KB>
isvd_status set_rot_attr(isvd_ctx* h) {
  CK(h, cudaFuncSetAttribute(k_rotate<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rot_smem_bytes<T, KB>()));
  return ISVD_OK;
}

template <typename T>
isvd_status set_attrs(isvd_ctx* h) {
  isvd_status s;
  if ((s = set_rot_attr<T, 16>(h)) || (s = set_rot_attr<T, 32>(h)) || (s = set_rot_attr<T, 64>(h)) ||
      (s = set_rot_attr<T, 128>(h)))
    return s;
  // The attribute is process-wide per template, so each bucket gets the shared memory of the
  // largest k_max it serves (handles with different k_max share one instantiation).
  const int kcap = sizeof(T) == sizeof(double) ? 96 : kKmaxLimit;
  const size_t core_smem[4] = {core_kernel_smem<T>(16), core_kernel_smem<T>(32), core_kernel_smem<T>(64),
                                core_kernel_smem<T>(kcap)};
  CK(h, core_set_attrs<T>(core_smem));
  CK(h, cudaFuncSetAttribute(k_sym_eig<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
  CK(h, cudaFuncSetAttribute(k_sym_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
  CK(h, cudaFuncSetAttribute(k_chol_rinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kKmaxLimit + 1) * (kKmaxLimit + 1) * sizeof(double))));
  CK(h, cudaFuncSetAttribute(k_resid_norm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kKmaxLimit * (kResTile + 1) * sizeof(T))));
  return ISVD_OK;
}

template <typename T>
isvd_status launch_rotate(isvd_ctx* h, const RotSide& s0, const RotSide& s1, int kb, const T* xz, const double* p) {
  // Side 0 always gets at least one block (its new row may be the only work).
  const int64_t t0e = std::max<int64_t>(1, (s0.rows + kRotRows - 1) / kRotRows);
  const int64_t t1 = s1.rows > 0 ? (s1.rows + kRotRows - 1) / kRotRows : 0;
  const int64_t tiles = t0e + t1;
  switch (kb) {
    case 16:
      k_rotate<T, 16><<<(unsigned)tiles, kRotThreads, rot_smem_bytes<T, 16>(), h->stream>>>(s0, s1, (int)t0e, xz, p, h->st);
      break;
    case 32:
      k_rotate<T, 32><<<(unsigned)tiles, kRotThreads, rot_smem_bytes<T, 32>(), h->stream>>>(s0, s1, (int)t0e, xz, p, h->st);
      break;
    case 64:
      k_rotate<T, 64><<<(unsigned)tiles, kRotThreads, rot_smem_bytes<T, 64>(), h->stream>>>(s0, s1, (int)t0e, xz, p, h->st);
      break;
    default:
      k_rotate<T, 128><<<(unsigned)tiles, kRotThreads, rot_smem_bytes<T, 128>(), h->stream>>>(s0, s1, (int)t0e, xz, p, h->st);
      break;
  }
  CKL(h);
  return ISVD_OK;
}

// ---- memory ------------------------------------------------------------------------------

isvd_status dmalloc(isvd_ctx* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, ISVD_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return ISVD_OK;
}

isvd_status ensure_rows(isvd_ctx* h, int64_t need) {
  if (need <= h->row_cap) return ISVD_OK;
  const int64_t cap = std::max(need, h->row_cap * 2);
  void *U2 = nullptr, *A2 = nullptr;
  isvd_status s;
  if ((s = dmalloc(h, &U2, (size_t)cap * h->ld * h->es))) return s;
  if ((s = dmalloc(h, &A2, (size_t)cap * h->col_cap * h->es))) {
    cudaFree(U2);
    return s;
  }
  CK(h, cudaMemcpyAsync(U2, h->U, (size_t)h->m * h->ld * h->es, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(A2, h->A, (size_t)h->m * h->col_cap * h->es, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  cudaFree(h->U);
  cudaFree(h->A);
  h->U = U2;
  h->A = A2;
  h->row_cap = cap;
  return ISVD_OK;
}

isvd_status ensure_cols(isvd_ctx* h, int64_t need) {
  if (need <= h->col_cap) return ISVD_OK;
  const int64_t cap = std::max(need, h->col_cap * 2);
  void *V2 = nullptr, *A2 = nullptr;
  isvd_status s;
  if ((s = dmalloc(h, &V2, (size_t)cap * h->ld * h->es))) return s;
  if ((s = dmalloc(h, &A2, (size_t)h->row_cap * cap * h->es))) {
    cudaFree(V2);
    return s;
  }
  CK(h, cudaMemcpyAsync(V2, h->V, (size_t)h->n * h->ld * h->es, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpy2DAsync(A2, cap * h->es, h->A, h->col_cap * h->es, h->n * h->es, h->m, cudaMemcpyDeviceToDevice,
                          h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  cudaFree(h->V);
  cudaFree(h->A);
  h->V = V2;
  h->A = A2;
  h->col_cap = cap;
  return ISVD_OK;
}

isvd_status ensure_buf(isvd_ctx* h, void** buf, int64_t* cap, int64_t need_bytes) {
  if (need_bytes <= *cap) return ISVD_OK;
  if (*buf) {
    CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(*buf);
    *buf = nullptr;
  }
  const int64_t c = std::max(need_bytes, *cap * 2);
  isvd_status s = dmalloc(h, buf, (size_t)c);
  if (s) {
    *cap = 0;
    return s;
  }
  *cap = c;
  return ISVD_OK;
}

// ---- single update ------------------------------------------------------------------------

int proj_blocks(int64_t rows) {
  int64_t b = (rows + 63) / 64;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, kMaxProjBlocks));
}

// Deferred rotations: fold the pending R_U, R_V into the tall factors, U <- U0 R_U and
// V <- V0 R_V (one pass of the rotation kernel over both sides, rows defer_rows -> r columns).
// Every operation that reads U or V calls this first; a no-op when nothing is pending.
template <typename T>
isvd_status materialize(isvd_ctx* h) {
  if (!h->defer_pending) return ISVD_OK;
  RotSide su{}, sv{};
  su.X = su.Y = h->U;
  su.rows = h->m;
  su.ldx = su.ldy = h->ld;
  su.R = h->RU;
  su.ldr = h->ld;
  su.c_in = -2;
  su.k_out = -2;
  sv = su;
  sv.X = sv.Y = h->V;
  sv.rows = h->n;
  sv.R = h->RV;
  prof_begin(h, ISVD_KCLASS_ROTATE, 2.0 * (h->m + h->n) * (double)h->k_host * h->es);
  isvd_status s = launch_rotate<T>(h, su, sv, kb_bucket(h->kmax), (const T*)nullptr, h->p);
  if (s) return s;
  prof_end(h);
  h->defer_pending = 0;
  return ISVD_OK;
}

isvd_status materialize_any(isvd_ctx* h) {
  return h->prec == ISVD_FP64 ? materialize<double>(h) : materialize<float>(h);
}

// Row append (kind kRow, x over the n columns) or column append (kind kCol, x over the m rows),
// x already on the device. Section 2.2 Steps 1-3 / Algorithms A1, A2.
template <typename T>
isvd_status do_append(isvd_ctx* h, int kind, const T* x) {
  isvd_status s;
  if ((s = materialize<T>(h))) return s;
  if (kind == kRow) {
    if ((s = ensure_rows(h, h->m + 1))) return s;
  } else {
    if ((s = ensure_cols(h, h->n + 1))) return s;
  }
  T* U = (T*)h->U;
  T* V = (T*)h->V;
  T* A = (T*)h->A;
  const int64_t lda = h->col_cap;
  // Projection side X: V for a row append (x over columns), U for a column append.
  const T* X = kind == kRow ? V : U;
  const int64_t rows = kind == kRow ? h->n : h->m;
  T* dst = kind == kRow ? A + h->m * lda : A + h->n;
  const int64_t dst_stride = kind == kRow ? 1 : lda;
  const int nb = proj_blocks(rows);
  const double kk = (double)h->k_host;
  prof_begin(h, ISVD_KCLASS_PROJ, (double)rows * (kk + 2) * h->es);  // X, x read; x written into A
  k_proj1<T><<<nb, kProjThreads, 0, h->stream>>>(X, h->ld, rows, x, h->st, h->part, h->p, dst, dst_stride);
  CKL(h);
  prof_end(h);
  prof_begin(h, ISVD_KCLASS_PROJ, (double)rows * (kk + 1) * h->es);  // X, x read
  if (sizeof(T) == sizeof(float)) {
    k_proj2<T, true><<<nb, kProjThreads, 0, h->stream>>>(X, h->ld, rows, x, h->st, h->part, h->p, h->tol_rel);
  } else {
    k_proj2<T, false><<<nb, kProjThreads, 0, h->stream>>>(X, h->ld, rows, x, h->st, h->part, h->p, h->tol_rel);
  }
  CKL(h);
  prof_end(h);
  prof_begin(h, ISVD_KCLASS_CORE, 2.0 * (kk + 1) * kk * h->es);
  if ((s = launch_core<T>(h, kind, 0, 0, 0.0))) return s;
  prof_end(h);
  // Rotations. Row append: U side uses U_K plus the new row, V side uses V_K plus z_hat.
  // Column append (transpose): U side uses V_K plus z_hat, V side uses U_K plus the new row.
  RotSide su{}, sv{};
  su.X = su.Y = U;
  su.rows = h->m;
  su.ldx = su.ldy = h->ld;
  su.ldr = h->ld;
  su.c_in = -1;
  su.k_out = -1;
  sv = su;
  sv.X = sv.Y = V;
  sv.rows = h->n;
  if (kind == kRow) {
    su.R = h->UK;
    su.newrow = 1;
    sv.R = h->VK;
    sv.zhat = 1;
  } else {
    su.R = h->VK;
    su.zhat = 1;
    sv.R = h->UK;
    sv.newrow = 1;
  }
  // U and V read and written once, plus the z_hat source vector.
  prof_begin(h, ISVD_KCLASS_ROTATE, (2.0 * (h->m + h->n) * kk + (double)rows) * h->es);
  if ((s = launch_rotate<T>(h, su, sv, kb_bucket(h->kmax), x, h->p))) return s;
  prof_end(h);
  if (kind == kRow) h->m += 1;
  else h->n += 1;
  return ISVD_OK;
}

// Rank-1 entry update, Section 2.3 / Algorithm A3. With deferred rotations on, the core gathers
// U0[i, :] R_U and V0[j, :] R_V and its factors go into R_U, R_V (k x k products); the tall factors
// are left alone until the next fold.
template <typename T>
isvd_status do_entry(isvd_ctx* h, int64_t i, int64_t j, double delta) {
  T* U = (T*)h->U;
  T* V = (T*)h->V;
  const double kk = (double)h->k_host;
  if (h->defer) {
    if (!h->defer_pending) {
      k_defer_init<T><<<std::max(1, std::min(148, h->kmax)), 256, 0, h->stream>>>((T*)h->RU, (T*)h->RV, h->ld, h->kmax,
                                                                                 h->st);
      CKL(h);
      h->defer_pending = 1;
    }
    prof_begin(h, ISVD_KCLASS_CORE, 2.0 * kk * kk * h->es);
    isvd_status s0 = launch_core<T>(h, kEntry, i, j, delta);
    if (s0) return s0;
    prof_end(h);
    prof_begin(h, ISVD_KCLASS_ROTATE, 4.0 * kk * kk * h->es);  // R_U, R_V read and written
    k_defer_compose<T><<<dim3((unsigned)h->kmax, 2), 128, 0, h->stream>>>((T*)h->RU, (T*)h->RV, h->ld,
                                                                           (const T*)h->UK, (const T*)h->VK, h->ld,
                                                                           h->st);
    CKL(h);
    prof_end(h);
    return ISVD_OK;
  }
  prof_begin(h, ISVD_KCLASS_CORE, 2.0 * kk * kk * h->es);
  isvd_status s0 = launch_core<T>(h, kEntry, i, j, delta);
  if (s0) return s0;
  prof_end(h);
  RotSide su{}, sv{};
  su.X = su.Y = U;
  su.rows = h->m;
  su.ldx = su.ldy = h->ld;
  su.ldr = h->ld;
  su.c_in = -1;
  su.k_out = -1;
  su.R = h->UK;
  sv = su;
  sv.X = sv.Y = V;
  sv.rows = h->n;
  sv.R = h->VK;
  prof_begin(h, ISVD_KCLASS_ROTATE, 2.0 * (h->m + h->n) * kk * h->es);
  isvd_status s = launch_rotate<T>(h, su, sv, kb_bucket(h->kmax), (const T*)nullptr, h->p);
  prof_end(h);
  return s;
}

// Rank-1 entry update in the rank-increasing form: the core is diag(sigma, 0) + delta [p; alpha]
// [q; beta]^T and each side gains its residual direction, P = (e_i - U p) / alpha and
// Q = (e_j - V q) / beta, formed row by row in the rotations.
template <typename T>
isvd_status do_entry_exact(isvd_ctx* h, int64_t i, int64_t j, double delta) {
  isvd_status sm = materialize<T>(h);
  if (sm) return sm;
  T* U = (T*)h->U;
  T* V = (T*)h->V;
  const double kk = (double)h->k_host;
  prof_begin(h, ISVD_KCLASS_CORE, 2.0 * (kk + 1) * (kk + 1) * h->es);
  isvd_status s0 = launch_core<T>(h, kEntryX, i, j, delta);
  if (s0) return s0;
  prof_end(h);
  RotSide su{}, sv{};
  su.X = su.Y = U;
  su.rows = h->m;
  su.ldx = su.ldy = h->ld;
  su.ldr = h->ld;
  su.c_in = -1;
  su.k_out = -1;
  su.R = h->UK;
  su.zhat = 1;
  su.zp = h->px;
  su.zrho = h->px + 2 * (kKmaxLimit + 2);
  su.zunit = i;
  sv = su;
  sv.X = sv.Y = V;
  sv.rows = h->n;
  sv.R = h->VK;
  sv.zp = h->px + (kKmaxLimit + 2);
  sv.zrho = h->px + 2 * (kKmaxLimit + 2) + 1;
  sv.zunit = j;
  prof_begin(h, ISVD_KCLASS_ROTATE, 2.0 * (h->m + h->n) * kk * h->es);
  isvd_status s = launch_rotate<T>(h, su, sv, kb_bucket(h->kmax), (const T*)nullptr, h->p);
  prof_end(h);
  return s;
}

// ---- truncated SVD of A (refresh and metrics) ----------------------------------------------

// C (rc x cc, FP64) = X^T Y over `rows` rows.
template <typename T>
isvd_status gemm_tn(isvd_ctx* h, const T* X, int64_t ldx, int cx, const T* Y, int64_t ldy, int cy, int64_t rows,
                    double* C, bool exact = false) {
  CK(h, cudaMemsetAsync(C, 0, (size_t)cx * cy * 8, h->stream));
  if (rows <= 0) return ISVD_OK;
  const int64_t splits_target = 304;
  int64_t rps = (rows + splits_target - 1) / splits_target;
  rps = std::max<int64_t>(kTnChunk, (rps + kTnChunk - 1) / kTnChunk * kTnChunk);
  dim3 grid((unsigned)((cx + kTnTile - 1) / kTnTile), (unsigned)((cy + kTnTile - 1) / kTnTile),
            (unsigned)((rows + rps - 1) / rps));
  if (exact) k_gemm_tn<T, true><<<grid, 256, 0, h->stream>>>(X, ldx, cx, Y, ldy, cy, rows, rps, C, cy);
  else k_gemm_tn<T><<<grid, 256, 0, h->stream>>>(X, ldx, cx, Y, ldy, cy, rows, rps, C, cy);
  CKL(h);
  return ISVD_OK;
}

// Eigendecomposition of an FP64 symmetric matrix: FP64 Jacobi (rotations in shared memory up to
// n = 80, beyond that in the n x n FP64 scratch vk), or (fp64 = 0) FP32 Jacobi with FP64
// Rayleigh-quotient eigenvalues.
template <typename T>
isvd_status sym_eig(isvd_ctx* h, const double* G, int n, double* evals, double* evecs, int fp64, double* vk) {
  const int threads = core_threads(std::max(n - 1, 1));
  if (fp64 && n <= 80) {
    const size_t sm = (size_t)2 * n * n * sizeof(double) + (size_t)n * 12 + 64;
    k_sym_eig<double><<<1, threads, sm, h->stream>>>(G, n, evals, evecs, h->info, nullptr);
  } else if (fp64) {
    const size_t sm = (size_t)n * n * sizeof(double) + (size_t)n * 12 + 64;
    k_sym_eig<double><<<1, threads, sm, h->stream>>>(G, n, evals, evecs, h->info, vk);
  } else {
    const size_t sm = (size_t)2 * n * n * sizeof(float) + (size_t)n * 12 + 64;
    k_sym_eig<float><<<1, threads, sm, h->stream>>>(G, n, evals, evecs, h->info, nullptr);
  }
  CKL(h);
  return ISVD_OK;
}

// Columns of a freshly formed factor side Q = A W diag(1 / sigma) (rows x r, row stride ldq)
// whose singular value is at the rounding floor are seeded with pseudo-random values, then the
// side is re-orthonormalised by shifted CholeskyQR3 (the leading columns barely move; the
// seeded ones become an orthonormal completion).
template <typename T>
isvd_status finish_side(isvd_ctx* h, T* Q, int64_t rows, int r, const double* sig);


isvd_status read_state(isvd_ctx* h, DevState* out) {
  CK(h, cudaMemcpyAsync(out, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (out->status & kStNonFinite) return fail(h, ISVD_ENONFINITE, "non-finite value in a device input");
  if (out->status & kStNotConv) return fail(h, ISVD_ENOTCONV, "core Jacobi SVD did not converge");
  if (out->status & kStTimeout) return fail(h, ISVD_ETIMEOUT, "device wait timed out");
  if (out->status & kStLayout) return fail(h, ISVD_ECUDA, "kernel shared-memory layout did not fit its launch");
  return ISVD_OK;
}

// In-place orthonormalisation of the columns of Q (rows x l, row stride l) by Cholesky-QR: a
// first pass with a small diagonal shift (robust when Q is rank deficient), then two plain
// passes (Fukaya et al.'s shifted CholeskyQR3).
template <typename T>
isvd_status orth_cols(isvd_ctx* h, T* Q, int64_t rows, int l, int64_t ldq = -1) {
  isvd_status s;
  if (ldq < 0) ldq = l;
  double* B = h->small + 4 * kSmall;
  if ((s = ensure_buf(h, &h->Rl, &h->rl_cap, (int64_t)l * l * (int64_t)h->es * 2))) return s;
  for (int pass = 0; pass < 3; ++pass) {
    if ((s = gemm_tn<T>(h, Q, ldq, l, Q, ldq, l, rows, B))) return s;
    if (pass == 0) {
      k_add_diag<<<1, 128, 0, h->stream>>>(B, l, sizeof(T) == 8 ? 1e-13 : 1e-5);
      CKL(h);
    }
    k_chol_rinv<T><<<1, 128, (size_t)l * l * sizeof(double), h->stream>>>(B, l, h->small + 5 * kSmall, (T*)h->Rl, l,
                                                                          h->info);
    CKL(h);
    RotSide sq{};
    sq.X = sq.Y = Q;
    sq.rows = rows;
    sq.ldx = sq.ldy = ldq;
    sq.R = h->Rl;
    sq.ldr = l;
    sq.c_in = l;
    sq.k_out = l;
    RotSide none{};
    if ((s = launch_rotate<T>(h, sq, none, kb_bucket(l), (const T*)nullptr, nullptr))) return s;
  }
  return ISVD_OK;
}

// One-sided finish of a truncated SVD (Gram or randomized path). Given B = A W (or A^T W) for the
// computed orthonormal basis W of the other side (rows x r, storage TB, row stride ldb), the
// singular values are taken as the column norms ||B_j|| (FP64 sums): accurate down to the
// rounding level of A, where sqrt of the Gram eigenvalue only reaches sqrt(eps) sigma_1. Columns
// are sorted by them; outB = B diag(1 / sigma) and W are permuted alike, and outB is finished by
// finish_side (seed + re-orthonormalisation).
template <typename T, typename TB>
isvd_status one_sided_finish(isvd_ctx* h, const TB* B, int64_t ldb, T* outB, int64_t rows, T* W, int64_t rows_w,
                             int r, double* sig_o) {
  double* sq = h->small + 5 * kSmall;
  int* perm = reinterpret_cast<int*>(sq + 256);
  CK(h, cudaMemsetAsync(sq, 0, (size_t)r * 8, h->stream));
  const int64_t splits = std::min<int64_t>(256, std::max<int64_t>(1, rows / 512));
  const int64_t rps = (rows + splits - 1) / splits;
  const dim3 gs((unsigned)((r + 31) / 32), (unsigned)splits);
  k_col_sumsq<TB><<<gs, 256, 0, h->stream>>>(B, rows, ldb, r, rps, sq);
  CKL(h);
  k_sort_norms<<<1, 128, 0, h->stream>>>(sq, r, sig_o, perm, h->inv);
  CKL(h);
  k_permute_cols<TB, T><<<(unsigned)((rows + 7) / 8), 256, 0, h->stream>>>(B, ldb, outB, h->ld, rows, r, perm, h->inv);
  CKL(h);
  k_permute_cols<T, T><<<(unsigned)((rows_w + 7) / 8), 256, 0, h->stream>>>(W, h->ld, W, h->ld, rows_w, r, perm, nullptr);
  CKL(h);
  return finish_side<T>(h, outB, rows, r, sig_o);
}

template <typename T>
isvd_status finish_side(isvd_ctx* h, T* Q, int64_t rows, int r, const double* sig) {
  if (r < 1 || rows < r) return ISVD_OK;
  const double rel = sizeof(T) == sizeof(double) ? 1e-13 : 1e-5;  // ~64 eps: B_j is rounding there
  const int64_t tot = rows * r;
  k_seed_small_cols<T><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(Q, rows, h->ld, sig, r, rel,
                                                                             h->seed ^ 0x5EEDC0151ull);
  CKL(h);
  return orth_cols<T>(h, Q, rows, r, h->ld);
}

// Randomized truncated SVD of A (Halko, Martinsson and Tropp 2011) at rank kr: l = kr + p
// columns (capped at 128 and min(m, n)), test matrix warm-started with the current V (the
// maintained right subspace) and completed with Gaussian columns, q power iterations with
// re-orthonormalisation between passes, then the small SVD of B = Q^T A through the Gram
// B B^T = Z^T Z (Z = A^T Q). The tail energy is not formed here: the metrics take E_opt as the
// residual ||A - U S V^T||_F of the computed factorisation (no N_t - sum sigma^2 cancellation).
template <typename T>
isvd_status tsvd_randomized(isvd_ctx* h, int kr, T* Uo, double* sig_o, T* Vo, int warm) {
  const int64_t m = h->m, n = h->n, lda = h->col_cap;
  const T* A = (const T*)h->A;
  isvd_status s;
  const int l = (int)std::min<int64_t>(std::min<int64_t>(kr + h->rsvd_p, kKmaxLimit), std::min(m, n));
  if (l < kr) return fail(h, ISVD_EINVAL, "randomized refresh: rank exceeds the sketch size");
  if ((s = ensure_buf(h, &h->Yb, &h->yb_cap, m * l * (int64_t)h->es))) return s;
  if ((s = ensure_buf(h, &h->Om, &h->om_cap, n * l * (int64_t)h->es))) return s;
  if ((s = ensure_buf(h, (void**)&h->Zd, &h->zd_cap, n * l * 8))) return s;
  if ((s = ensure_buf(h, &h->Rl, &h->rl_cap, (int64_t)l * l * (int64_t)h->es * 2))) return s;
  T* Y = (T*)h->Yb;
  T* Om = (T*)h->Om;
  T* Rl2 = (T*)h->Rl + (int64_t)l * l;
  int c0 = 0;
  if (warm) {
    DevState ds;
    if ((s = read_state(h, &ds))) return s;
    c0 = std::min(ds.r, l);
  }
  const uint64_t seed = h->seed * 0x9E3779B97F4A7C15ull + (uint64_t)(++h->rsvd_calls);
  k_fill_omega<T><<<(unsigned)((n * l + 255) / 256), 256, 0, h->stream>>>(Om, n, l, l, (const T*)h->V, h->ld, c0, seed);
  CKL(h);
  const dim3 gy((unsigned)((m + kGemmBM - 1) / kGemmBM), (unsigned)((l + kGemmBN - 1) / kGemmBN));
  k_gemm_nn<T><<<gy, 256, 0, h->stream>>>(A, lda, m, n, Om, l, l, Y, l);
  CKL(h);
  if ((s = orth_cols<T>(h, Y, m, l))) return s;
  for (int it = 0; it <= h->rsvd_q; ++it) {
    // Z = A^T Q (n x l, FP64)
    if ((s = gemm_tn<T>(h, A, lda, (int)n, Y, l, l, m, h->Zd))) return s;
    if (it == h->rsvd_q) break;
    k_scale_cast<T><<<(unsigned)((n * l + 255) / 256), 256, 0, h->stream>>>(h->Zd, n, l, l, nullptr, Om, l);
    CKL(h);
    if ((s = orth_cols<T>(h, Om, n, l))) return s;
    k_gemm_nn<T><<<gy, 256, 0, h->stream>>>(A, lda, m, n, Om, l, l, Y, l);
    CKL(h);
    if ((s = orth_cols<T>(h, Y, m, l))) return s;
  }
  double* GB = h->small + 3 * kSmall;
  double* evecs = h->small + 2 * kSmall;
  if ((s = gemm_tn<double>(h, h->Zd, l, l, h->Zd, l, l, n, GB))) return s;
  if ((s = sym_eig<T>(h, GB, l, h->evals, evecs, 1, h->small + kSmall))) return s;
  k_eig_to_factors<T><<<1, 256, 0, h->stream>>>(h->evals, evecs, l, kr, sig_o, h->inv, Rl2, l, h->scal + 3);
  CKL(h);
  RotSide su{};
  su.X = Y;
  su.Y = Uo;
  su.rows = m;
  su.ldx = l;
  su.ldy = h->ld;
  su.R = Rl2;
  su.ldr = l;
  su.c_in = l;
  su.k_out = kr;
  RotSide none{};
  if ((s = launch_rotate<T>(h, su, none, kb_bucket(l), (const T*)nullptr, nullptr))) return s;
  // B = A^T U = Z E[:, :kr] (FP64), then the one-sided finish of V.
  if ((s = ensure_buf(h, (void**)&h->Cbuf, &h->cbuf_cap, n * kr * 8))) return s;
  k_small_gemm_cast<double><<<(unsigned)((n * kr + 255) / 256), 256, 0, h->stream>>>(h->Zd, n, l, evecs, kr, nullptr,
                                                                                     h->Cbuf, kr);
  CKL(h);
  return one_sided_finish<T, double>(h, h->Cbuf, kr, Vo, n, Uo, m, kr, sig_o);
}

// Truncated SVD of the stored A_t at rank kr (Algorithm 1 "TruncatedSVD", Section 2.4):
// Uo (m x kr, row stride ld), sig_o (kr), Vo (n x kr, row stride ld); on the exact path (through
// the Gram matrix of the short side) also the tail energy sum_{j > kr} s_j^2 in h->scal[1].
template <typename T>
isvd_status tsvd(isvd_ctx* h, int kr, T* Uo, double* sig_o, T* Vo, int warm = 1) {
  const int64_t m = h->m, n = h->n;
  const int64_t lda = h->col_cap;
  const T* A = (const T*)h->A;
  // The small symmetric eigenproblem runs in FP64 for both storage types: with FP32 Jacobi the
  // eigenvectors of nearly equal eigenvalues (a noise bulk at the truncation boundary) were off by
  // eps * ||G|| / gap, far above the FP32 path's tolerance.
  const int fp64 = 1;
  if (std::min(m, n) > kKmaxLimit) return tsvd_randomized<T>(h, kr, Uo, sig_o, Vo, warm);
  isvd_status s;
  const int q = (int)std::min(m, n);
  if ((s = ensure_buf(h, (void**)&h->G, &h->G_cap, (int64_t)q * q * 8 * 3))) return s;
  double* G = h->G;
  double* evecs = h->G + (int64_t)q * q;
  double* vk = h->G + (int64_t)2 * q * q;
  if (n <= m) {
    if ((s = gemm_tn<T>(h, A, lda, (int)n, A, lda, (int)n, m, G, true))) return s;
    if ((s = sym_eig<T>(h, G, q, h->evals, evecs, fp64, vk))) return s;
    k_eig_to_factors<T><<<1, 256, 0, h->stream>>>(h->evals, evecs, q, kr, sig_o, h->inv, Vo, h->ld, h->scal + 1);
    CKL(h);
    RotSide su{};
    su.X = A;
    su.Y = Uo;
    su.rows = m;
    su.ldx = lda;
    su.ldy = h->ld;
    su.R = Vo;
    su.ldr = h->ld;
    su.c_in = (int)n;
    su.k_out = kr;
    su.colscale = nullptr;  // B = A V; sigma and the scaling come from its column norms
    RotSide none{};
    none.rows = 0;
    none.c_in = 0;
    none.k_out = 0;
    if ((s = launch_rotate<T>(h, su, none, kb_bucket(std::max<int>((int)n, kr)), (const T*)nullptr, nullptr))) return s;
    if ((s = one_sided_finish<T, T>(h, Uo, h->ld, Uo, m, Vo, n, kr, sig_o))) return s;
  } else {
    CK(h, cudaMemsetAsync(G, 0, (size_t)q * q * 8, h->stream));
    const int64_t e = (int64_t)m * m;
    k_gram_rows<T><<<(unsigned)((e + 7) / 8), 256, 0, h->stream>>>(A, lda, (int)m, n, G);
    CKL(h);
    if ((s = sym_eig<T>(h, G, q, h->evals, evecs, fp64, vk))) return s;
    k_eig_to_factors<T><<<1, 256, 0, h->stream>>>(h->evals, evecs, q, kr, sig_o, h->inv, Uo, h->ld, h->scal + 1);
    CKL(h);
    // V = A^T U S^-1.
    if ((s = ensure_buf(h, (void**)&h->Cbuf, &h->cbuf_cap, n * kr * 8))) return s;
    CK(h, cudaMemsetAsync(h->Cbuf, 0, (size_t)n * kr * 8, h->stream));
    const int64_t rps = std::max<int64_t>(kTnChunk, m);
    dim3 grid((unsigned)((n + kTnTile - 1) / kTnTile), (unsigned)((kr + kTnTile - 1) / kTnTile), 1);
    k_gemm_tn<T><<<grid, 256, 0, h->stream>>>(A, lda, (int)n, Uo, h->ld, kr, m, rps, h->Cbuf, kr);
    CKL(h);
    if ((s = one_sided_finish<T, double>(h, h->Cbuf, kr, Vo, n, Uo, m, kr, sig_o))) return s;
  }
  return ISVD_OK;
}

template <typename T>
isvd_status set_rank(isvd_ctx* h, int r) {
  CK(h, cudaMemcpyAsync(&h->st->r, &r, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return ISVD_OK;
}

template <typename T>
isvd_status store_ref(isvd_ctx* h, int r) {
  isvd_status s;
  if ((s = ensure_buf(h, &h->Uref, &h->uref_cap, h->m * h->ld * (int64_t)h->es))) return s;
  CK(h, cudaMemcpyAsync(h->Uref, h->U, (size_t)h->m * h->ld * h->es, cudaMemcpyDeviceToDevice, h->stream));
  h->m_ref = h->m;
  h->r_ref = r;
  return ISVD_OK;
}

template <typename T>
isvd_status do_refresh(isvd_ctx* h, int store) {
  isvd_status s;
  if ((s = materialize<T>(h))) return s;
  {
    // The working rank may have been grown on the device (novelty rule, the pool's rank rule).
    DevState ds;
    if ((s = read_state(h, &ds))) return s;
    h->k_host = ds.k;
  }
  const int kr = (int)std::min<int64_t>(h->k_host, std::min(h->m, h->n));
  if (h->opt_t == h->t && h->opt_rank == kr && h->Uopt && h->Vopt) {
    // The policy check at this same t already computed TruncatedSVD(A_t, kr) for its metrics.
    CK(h, cudaMemcpyAsync(h->U, h->Uopt, (size_t)h->m * h->ld * h->es, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->V, h->Vopt, (size_t)h->n * h->ld * h->es, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->sig, h->sig_opt, (size_t)kr * 8, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    if ((s = tsvd<T>(h, kr, (T*)h->U, h->sig, (T*)h->V))) return s;
  }
  if ((s = set_rank<T>(h, kr))) return s;
  if (store && (s = store_ref<T>(h, kr))) return s;
  h->t_last = h->t;
  h->refreshes++;
  return ISVD_OK;
}

// ---- metrics ----------------------------------------------------------------------------

// Largest principal angle between span(Q1) (rows1 x r1) and span(Q2) (rows2 x r2), rows1 <= rows2
// (Q1 embedded with zero rows), Eq. (theta-max). Computed as arcsin(sqrt(lambda_max(E))) with
// E = Q_b^T (I - P_a) Q_b for the side b with fewer columns, which equals
// arccos(sigma_min(Q1^T Q2)) for orthonormal bases and keeps small angles accurate.
template <typename T>
isvd_status max_angle(isvd_ctx* h, const T* Q1, int64_t rows1, int r1, const T* Q2, int r2, double* theta) {
  isvd_status s;
  double* C = h->small;              // r1 x r2
  double* B = h->small + kSmall;     // q x q
  double* E = h->small + 2 * kSmall; // q x q
  double* evecs = h->small + 3 * kSmall;
  if ((s = gemm_tn<T>(h, Q1, h->ld, r1, Q2, h->ld, r2, rows1, C))) return s;
  const int tr = r1 <= r2 ? 1 : 0;  // E on the Q1 side when it has fewer columns
  const int q = tr ? r1 : r2;
  if (tr) {
    if ((s = gemm_tn<T>(h, Q1, h->ld, r1, Q1, h->ld, r1, rows1, B))) return s;
  } else {
    if ((s = gemm_tn<T>(h, Q2, h->ld, r2, Q2, h->ld, r2, h->m, B))) return s;
  }
  k_angle_matrix<<<1, 256, 0, h->stream>>>(B, C, r1, r2, tr, E);
  CKL(h);
  if ((s = sym_eig<T>(h, E, q, h->evals, evecs, sizeof(T) == sizeof(double), h->small + 4 * kSmall))) return s;
  double lam = 0;
  CK(h, cudaMemcpyAsync(&lam, h->evals, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  lam = std::min(1.0, std::max(0.0, lam));
  *theta = std::asin(std::sqrt(lam));
  return ISVD_OK;
}

template <typename T>
isvd_status do_metrics(isvd_ctx* h, int flags, isvd_metrics_t* mt) {
  isvd_status s;
  if ((s = materialize<T>(h))) return s;
  DevState ds;
  if ((s = read_state(h, &ds))) return s;
  const int r = ds.r;
  std::vector<double> sg(r);
  CK(h, cudaMemcpy(sg.data(), h->sig, r * 8, cudaMemcpyDeviceToHost));
  memset(mt, 0, sizeof(*mt));
  mt->t = h->t;
  mt->m = h->m;
  mt->n = h->n;
  mt->r = r;
  mt->k = ds.k;
  double ss = 0;
  for (double v : sg) ss += v * v;
  mt->N = ds.N;
  mt->evr = ds.N > 0 ? ss / ds.N : NAN;
  mt->rho_last = ds.rho;
  mt->novelty_last = ds.novelty;
  mt->angle_succ_u = ds.ang_u;
  mt->angle_succ_v = ds.ang_v;
  mt->orth_err_u = h->orth_on_device && ds.orth_runs > 0 ? ds.orth_u : h->orth_err_u;
  mt->orth_err_v = h->orth_on_device && ds.orth_runs > 0 ? ds.orth_v : h->orth_err_v;
  mt->refreshes = h->refreshes;
  mt->reorths = h->reorths + ds.reorths;
  mt->t_last = h->t_last;
  mt->core_sweeps = ds.sweeps;
  const double nan = std::nan("");
  mt->frob_error = mt->frob_opt = mt->frob_gap = mt->frob_ratio = mt->angle = mt->angle_to_opt = nan;
  if (!(flags & ISVD_METRICS_FULL)) return ISVD_OK;
  // E_inc
  CK(h, cudaMemsetAsync(h->scal, 0, 8, h->stream));
  {
    dim3 grid((unsigned)((h->n + kResTile - 1) / kResTile), (unsigned)((h->m + kResTile - 1) / kResTile));
    const size_t sm = (size_t)2 * std::max(r, 1) * (kResTile + 1) * sizeof(T);
    k_resid_norm<T><<<grid, 256, sm, h->stream>>>((const T*)h->A, h->col_cap, h->m, h->n, (const T*)h->U,
                                                  (const T*)h->V, h->ld, h->sig, h->st, h->scal);
    CKL(h);
  }
  // optimal rank-r factorisation
  if ((s = ensure_buf(h, &h->Uopt, &h->uopt_cap, h->m * h->ld * (int64_t)h->es))) return s;
  if ((s = ensure_buf(h, &h->Vopt, &h->vopt_cap, h->n * h->ld * (int64_t)h->es))) return s;
  if ((s = tsvd<T>(h, r, (T*)h->Uopt, h->sig_opt, (T*)h->Vopt))) return s;
  h->opt_t = h->t;
  h->opt_rank = r;
  if (std::min(h->m, h->n) > kKmaxLimit) {
    // Randomized path: E_opt = ||A - U_opt S_opt V_opt^T||_F of the computed rank-r factorisation,
    // summed entry by entry in FP64 (an upper bound of the optimum that needs no tail spectrum).
    CK(h, cudaMemsetAsync(h->scal + 1, 0, 8, h->stream));
    dim3 grid((unsigned)((h->n + kResTile - 1) / kResTile), (unsigned)((h->m + kResTile - 1) / kResTile));
    const size_t sm = (size_t)2 * std::max(r, 1) * (kResTile + 1) * sizeof(T);
    k_resid_norm<T><<<grid, 256, sm, h->stream>>>((const T*)h->A, h->col_cap, h->m, h->n, (const T*)h->Uopt,
                                                  (const T*)h->Vopt, h->ld, h->sig_opt, h->st, h->scal + 1, r);
    CKL(h);
  }
  double sc[2];
  CK(h, cudaMemcpyAsync(sc, h->scal, 16, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const double e_inc = std::sqrt(std::max(sc[0], 0.0));
  const double e_opt = std::sqrt(std::max(sc[1], 0.0));
  mt->frob_error = e_inc;
  mt->frob_opt = e_opt;
  mt->frob_gap = e_inc - e_opt;
  mt->frob_ratio = (e_opt <= 1e-12 * std::sqrt(std::max(ds.N, 0.0))) ? nan : e_inc / e_opt;
  double th = nan;
  if ((s = max_angle<T>(h, (const T*)h->Uopt, h->m, r, (const T*)h->U, r, &th))) return s;
  mt->angle_to_opt = th;
  if (h->Uref && h->r_ref > 0) {
    if ((s = max_angle<T>(h, (const T*)h->Uref, h->m_ref, h->r_ref, (const T*)h->U, r, &th))) return s;
    mt->angle = th;
  }
  return ISVD_OK;
}

// ---- finance layer: low-rank covariance and portfolio risk (Section 5.3) --------------------

template <typename T>
isvd_status do_risk(isvd_ctx* h, const void* w, int w_dev, int flags, isvd_risk_t* out) {
  isvd_status s;
  if ((s = materialize<T>(h))) return s;
  DevState ds;
  if ((s = read_state(h, &ds))) return s;
  const int r = ds.r;
  const int64_t n = h->n;
  memset(out, 0, sizeof(*out));
  out->t = h->m;
  out->r = r;
  if (r < 1 || h->m < 2) return fail(h, ISVD_ESHAPE, "risk needs at least two rows and one component");
  const T* wd = (const T*)w;
  if (!w || !w_dev) {
    if ((s = ensure_buf(h, &h->wbuf, &h->wbuf_cap, n * (int64_t)h->es))) return s;
    if (!w) {
      k_fill<T><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>((T*)h->wbuf, n, (T)(1.0 / (double)n));
      CKL(h);
    } else {
      CK(h, cudaMemcpyAsync(h->wbuf, w, (size_t)n * h->es, cudaMemcpyHostToDevice, h->stream));
    }
    wd = (const T*)h->wbuf;
  }
  const int full = (flags & ISVD_RISK_FULL) != 0;
  if (full && !(h->opt_t == h->t && h->opt_rank == r && h->Uopt && h->Vopt)) {
    if ((s = ensure_buf(h, &h->Uopt, &h->uopt_cap, h->m * h->ld * (int64_t)h->es))) return s;
    if ((s = ensure_buf(h, &h->Vopt, &h->vopt_cap, h->n * h->ld * (int64_t)h->es))) return s;
    if ((s = tsvd<T>(h, r, (T*)h->Uopt, h->sig_opt, (T*)h->Vopt))) return s;
    h->opt_t = h->t;
    h->opt_rank = r;
  }
  const int64_t need = (int64_t)(3 * r * r + 2 * r + 8) * 8;
  if ((s = ensure_buf(h, (void**)&h->riskbuf, &h->risk_cap, need))) return s;
  double* G1 = h->riskbuf;
  double* G2 = G1 + r * r;
  double* Cx = G2 + r * r;
  double* g = Cx + r * r;
  double* gopt = g + r;
  double* res = gopt + r;
  const T* V = (const T*)h->V;
  if ((s = gemm_tn<T>(h, V, h->ld, r, wd, 1, 1, n, g, true))) return s;
  if ((s = gemm_tn<T>(h, V, h->ld, r, V, h->ld, r, n, G1, true))) return s;
  if (full) {
    const T* Vo = (const T*)h->Vopt;
    if ((s = gemm_tn<T>(h, Vo, h->ld, r, wd, 1, 1, n, gopt, true))) return s;
    if ((s = gemm_tn<T>(h, Vo, h->ld, r, Vo, h->ld, r, n, G2, true))) return s;
    if ((s = gemm_tn<T>(h, V, h->ld, r, Vo, h->ld, r, n, Cx, true))) return s;
  }
  k_risk_finish<<<1, 256, 0, h->stream>>>(h->sig, h->sig_opt, g, gopt, G1, G2, Cx, r, 1.0 / (double)(h->m - 1), full,
                                          res);
  CKL(h);
  double v[5];
  CK(h, cudaMemcpyAsync(v, res, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  out->vol = v[0];
  out->vol_opt = v[1];
  out->risk_error = v[2];
  out->cov_error = v[3];
  out->cov_norm = v[4];
  return ISVD_OK;
}

// ---- re-orthogonalisation -----------------------------------------------------------------

template <typename T>
isvd_status orth_err(isvd_ctx* h, const T* Q, int64_t rows, int r, double* err) {
  isvd_status s;
  double* B = h->small + 4 * kSmall;
  // Exact FP64 products: the measurement error stays far below the FP32 orthogonality level.
  if ((s = gemm_tn<T>(h, Q, h->ld, r, Q, h->ld, r, rows, B, true))) return s;
  k_max_offident<<<1, 256, 0, h->stream>>>(B, r, h->scal + 2);
  CKL(h);
  CK(h, cudaMemcpyAsync(err, h->scal + 2, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return ISVD_OK;
}

// One Cholesky-QR pass Q <- Q R^-1 with R^T R = Q^T Q (B must hold Q^T Q).
template <typename T>
isvd_status cholqr_pass(isvd_ctx* h, T* Q, int64_t rows, int r) {
  isvd_status s;
  double* B = h->small + 4 * kSmall;
  if ((s = gemm_tn<T>(h, Q, h->ld, r, Q, h->ld, r, rows, B))) return s;
  k_chol_rinv<T><<<1, 128, (size_t)r * r * sizeof(double), h->stream>>>(B, r, h->small + 5 * kSmall, (T*)h->Rtmp,
                                                                          h->ld, h->info);
  CKL(h);
  RotSide sq{};
  sq.X = sq.Y = Q;
  sq.rows = rows;
  sq.ldx = sq.ldy = h->ld;
  sq.R = h->Rtmp;
  sq.ldr = h->ld;
  sq.c_in = r;
  sq.k_out = r;
  RotSide none{};
  return launch_rotate<T>(h, sq, none, kb_bucket(h->kmax), (const T*)nullptr, nullptr);
}

template <typename T>
isvd_status do_reorth(isvd_ctx* h, int force, double* eu, double* ev) {
  isvd_status s;
  if ((s = materialize<T>(h))) return s;
  DevState ds;
  if ((s = read_state(h, &ds))) return s;
  const int r = ds.r;
  if ((s = orth_err<T>(h, (const T*)h->U, h->m, r, &h->orth_err_u))) return s;
  if ((s = orth_err<T>(h, (const T*)h->V, h->n, r, &h->orth_err_v))) return s;
  if (std::isnan(h->orth_err_u) || std::isnan(h->orth_err_v))
    return fail(h, ISVD_ENONFINITE, "non-finite values in U or V (orthogonality monitor)");
  if (force || h->orth_err_u > h->orth_tol || h->orth_err_v > h->orth_tol) {
    for (int pass = 0; pass < 2; ++pass) {
      if ((s = cholqr_pass<T>(h, (T*)h->U, h->m, r))) return s;
      if ((s = cholqr_pass<T>(h, (T*)h->V, h->n, r))) return s;
    }
    h->reorths++;
  }
  if (eu) *eu = h->orth_err_u;
  if (ev) *ev = h->orth_err_v;
  h->since_orth = 0;
  return ISVD_OK;
}

// ---- policy (Section 3), evaluated after every update -------------------------------------

template <typename T>
isvd_status after_update(isvd_ctx* h) {
  h->t += 1;
  h->since_orth += 1;
  isvd_status s;
  bool fire = false;
  if (h->has_pol) {
    const isvd_policy& pol = h->pol;
    if ((pol.kind & ISVD_POLICY_PERIODIC) && pol.T_refresh > 0 && h->t % pol.T_refresh == 0) fire = true;
    if (pol.check_every > 0 && h->t % pol.check_every == 0) {
      isvd_metrics_t mt;
      prof_begin(h, ISVD_KCLASS_CHECK, 0.0);
      if ((s = do_metrics<T>(h, ISVD_METRICS_FULL, &mt))) return s;
      prof_end(h);
      const bool spaced = (h->t - h->t_last) >= pol.T_min;
      if ((pol.kind & ISVD_POLICY_ERROR) && spaced && std::isfinite(mt.frob_ratio) && mt.frob_ratio > pol.gamma)
        fire = true;
      if ((pol.kind & ISVD_POLICY_ANGLE) && spaced && std::isfinite(mt.angle_to_opt) &&
          mt.angle_to_opt > pol.theta_max_rad)
        fire = true;
      h->k_host = mt.k;  // the device's working rank (the novelty rule may have grown it)
      if ((pol.kind & ISVD_POLICY_ADAPTIVE_RANK) && std::isfinite(mt.evr) && mt.evr < pol.tau_evr) {
        const int kcap = pol.k_max > 0 ? std::min(pol.k_max, h->kmax) : h->kmax;
        const int knew = std::min(h->k_host + 1, kcap);
        if (knew != h->k_host) {
          h->k_host = knew;
          CK(h, cudaMemcpyAsync(&h->st->k, &h->k_host, sizeof(int), cudaMemcpyHostToDevice, h->stream));
          CK(h, cudaStreamSynchronize(h->stream));
        }
      } else if ((pol.kind & ISVD_POLICY_RANK_SHRINK) && h->k_host > std::max(pol.k_min, 1) && mt.N > 0.0) {
        // The shrink side: the leading k - 1 maintained components against N_t.
        const int keep = std::min(h->k_host - 1, (int)mt.r);
        std::vector<double> sg(keep);
        if (keep > 0) CK(h, cudaMemcpy(sg.data(), h->sig, 8 * (size_t)keep, cudaMemcpyDeviceToHost));
        double ss = 0.0;
        for (double v : sg) ss += v * v;
        if (ss / mt.N >= pol.tau_shrink) {
          h->k_host -= 1;
          const int rnew = std::min((int)mt.r, h->k_host);
          CK(h, cudaMemcpyAsync(&h->st->k, &h->k_host, sizeof(int), cudaMemcpyHostToDevice, h->stream));
          CK(h, cudaMemcpyAsync(&h->st->r, &rnew, sizeof(int), cudaMemcpyHostToDevice, h->stream));
          CK(h, cudaStreamSynchronize(h->stream));
        }
      }
      h->last_check = mt;
    }
  }
  if (fire) {
    prof_begin(h, ISVD_KCLASS_REFRESH, 0.0);
    if ((s = do_refresh<T>(h, h->has_pol ? h->pol.store_initial_subspace : 0))) return s;
    prof_end(h);
    if (h->has_pol && h->pol.check_every > 0 && h->t % h->pol.check_every == 0) h->last_check.t_last = h->t;
  }
  if (h->orth_every > 0 && h->since_orth >= h->orth_every) {
    prof_begin(h, ISVD_KCLASS_REORTH, 0.0);
    if ((s = do_reorth<T>(h, 0, nullptr, nullptr))) return s;
    prof_end(h);
  }
  prof_stamp(h);
  return ISVD_OK;
}

// ---- host vector staging ------------------------------------------------------------------

isvd_status stage(isvd_ctx* h, const void* src, int64_t len, int on_device, const void** out) {
  if (on_device) {
    *out = src;
    return ISVD_OK;
  }
  isvd_status s;
  // The previous update may still read xbuf: wait for the stream before overwriting it.
  const int64_t bytes = len * (int64_t)h->es;
  if (bytes > h->xbuf_cap) {
    if ((s = ensure_buf(h, &h->xbuf, &h->xbuf_cap, bytes))) return s;
  }
  CK(h, cudaMemcpyAsync(h->xbuf, src, (size_t)bytes, cudaMemcpyHostToDevice, h->stream));
  *out = h->xbuf;
  return ISVD_OK;
}

template <typename T>
isvd_status create_impl(isvd_ctx* h, const void* A0, int64_t m0, int64_t n0, int64_t lda0, int k, int on_dev,
                        const void* U0 = nullptr, const double* S0 = nullptr, const void* V0 = nullptr) {
  isvd_status s;
  if ((s = set_attrs<T>(h))) return s;
  if ((s = dmalloc(h, &h->U, (size_t)h->row_cap * h->ld * h->es))) return s;
  if ((s = dmalloc(h, &h->V, (size_t)h->col_cap * h->ld * h->es))) return s;
  if ((s = dmalloc(h, &h->A, (size_t)h->row_cap * h->col_cap * h->es))) return s;
  if ((s = dmalloc(h, (void**)&h->st, sizeof(DevState)))) return s;
  if ((s = dmalloc(h, (void**)&h->sig, (kKmaxLimit + 2) * 8))) return s;
  if ((s = dmalloc(h, (void**)&h->p, (kKmaxLimit + 2) * 8))) return s;
  if ((s = dmalloc(h, (void**)&h->px, (2 * (kKmaxLimit + 2) + 2) * 8))) return s;
  if (h->kmax > kFastCoreQSmemMaxKB &&
      (s = dmalloc(h, (void**)&h->gq, (size_t)(kKmaxLimit + 1) * (kKmaxLimit + 1) * sizeof(float))))
    return s;
  if ((s = dmalloc(h, (void**)&h->part, (size_t)kMaxProjBlocks * kPartStride * 8))) return s;
  if ((s = dmalloc(h, &h->UK, (size_t)(kKmaxLimit + 2) * h->ld * h->es))) return s;
  if ((s = dmalloc(h, &h->VK, (size_t)(kKmaxLimit + 2) * h->ld * h->es))) return s;
  if ((s = dmalloc(h, (void**)&h->small, (size_t)6 * kSmall * 8))) return s;
  if ((s = dmalloc(h, (void**)&h->evals, (kKmaxLimit + 2) * 8 * 2))) return s;
  if ((s = dmalloc(h, (void**)&h->inv, (kKmaxLimit + 2) * 8))) return s;
  if ((s = dmalloc(h, (void**)&h->sig_opt, (kKmaxLimit + 2) * 8))) return s;
  if ((s = dmalloc(h, (void**)&h->scal, 64))) return s;
  if ((s = dmalloc(h, (void**)&h->info, 64))) return s;
  if ((s = dmalloc(h, &h->Rtmp, (size_t)(kKmaxLimit + 2) * h->ld * h->es))) return s;
  CK(h, cudaMemsetAsync(h->U, 0, (size_t)h->row_cap * h->ld * h->es, h->stream));
  CK(h, cudaMemsetAsync(h->V, 0, (size_t)h->col_cap * h->ld * h->es, h->stream));
  CK(h, cudaMemcpy2DAsync(h->A, h->col_cap * h->es, A0, lda0 * h->es, n0 * h->es, m0,
                          on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  h->m = m0;
  h->n = n0;
  // N_0 = ||A0||_F^2 (Section 2.4): the trace of the Gram of A0 through the same product kernel.
  DevState ds{};
  ds.k = k;
  ds.ang_u = ds.ang_v = NAN;  // no update yet
  CK(h, cudaMemcpyAsync(h->st, &ds, sizeof(ds), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemsetAsync(h->scal, 0, 64, h->stream));
  {
    // sum of squares via the residual kernel with r = 0 (E = ||A - 0||).
    dim3 grid((unsigned)((n0 + kResTile - 1) / kResTile), (unsigned)((m0 + kResTile - 1) / kResTile));
    k_resid_norm<T><<<grid, 256, (size_t)2 * (kResTile + 1) * sizeof(T), h->stream>>>(
        (const T*)h->A, h->col_cap, m0, n0, (const T*)h->U, (const T*)h->V, h->ld, h->sig, h->st, h->scal);
    CKL(h);
  }
  CK(h, cudaMemcpyAsync(&h->st->N, h->scal, 8, cudaMemcpyDeviceToDevice, h->stream));
  const int r0 = (int)std::min<int64_t>(k, std::min(m0, n0));
  if (U0) {
    // Caller-supplied initial factors (U0 m0 x r0, sigma0 r0, V0 n0 x r0, row stride r0).
    const cudaMemcpyKind kd = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(h, cudaMemcpy2DAsync(h->U, h->ld * h->es, U0, r0 * h->es, r0 * h->es, m0, kd, h->stream));
    CK(h, cudaMemcpy2DAsync(h->V, h->ld * h->es, V0, r0 * h->es, r0 * h->es, n0, kd, h->stream));
    CK(h, cudaMemcpyAsync(h->sig, S0, r0 * 8, kd, h->stream));
  } else {
    if ((s = tsvd<T>(h, r0, (T*)h->U, h->sig, (T*)h->V, 0))) return s;
  }
  if ((s = set_rank<T>(h, r0))) return s;
  if ((s = store_ref<T>(h, r0))) return s;
  CK(h, cudaStreamSynchronize(h->stream));
  return read_state(h, &ds);
}

}  // namespace

// ---- C ABI ----------------------------------------------------------------------------------

extern "C" {

const char* isvd_status_string(isvd_status s) {
  switch (s) {
    case ISVD_OK: return "ok";
    case ISVD_EINVAL: return "invalid argument";
    case ISVD_ESHAPE: return "shape mismatch";
    case ISVD_EBOUNDS: return "index out of bounds";
    case ISVD_ENOMEM: return "out of device memory";
    case ISVD_EBUDGET: return "memory budget exceeded";
    case ISVD_ENOTCONV: return "core SVD did not converge";
    case ISVD_ETIMEOUT: return "device wait timed out";
    case ISVD_ECUDA: return "CUDA error";
    case ISVD_ENONFINITE: return "non-finite input";
  }
  return "unknown status";
}

static isvd_status create_common(const isvd_config* cfg, const void* A0, int64_t m0, int64_t n0, int64_t lda, int k,
                                 int on_dev, const void* U0, const double* S0, const void* V0, int r0, isvd_t* out) {
  if (!cfg || !A0 || !out) return ISVD_EINVAL;
  *out = nullptr;
  if (m0 < 1 || n0 < 1 || lda < n0 || k < 1) return ISVD_ESHAPE;
  if (cfg->prec != ISVD_FP64 && cfg->prec != ISVD_FP32) return ISVD_EINVAL;
  const int kmax = cfg->k_max > 0 ? cfg->k_max : k;
  if (kmax < k || kmax > kKmaxLimit) return ISVD_EINVAL;
  if (cfg->prec == ISVD_FP64 && kmax > 96) return ISVD_EINVAL;  // FP64 core shared memory
  if (U0 && (!S0 || !V0 || r0 != (int)std::min<int64_t>(k, std::min(m0, n0)))) return ISVD_ESHAPE;
  isvd_ctx* h = new isvd_ctx();
  h->prec = cfg->prec;
  h->es = cfg->prec == ISVD_FP64 ? 8 : 4;
  h->stream = (cudaStream_t)cfg->cuda_stream;
  cudaGetDevice(&h->dev);
  h->kmax = kmax;
  h->ld = round_up(kmax, 4);
  h->k_host = k;
  h->tol_rel = cfg->tol_rel > 0 ? cfg->tol_rel : (cfg->prec == ISVD_FP64 ? 1e-10 : 3e-6);
  h->orth_tol = cfg->orth_tol > 0 ? cfg->orth_tol : (cfg->prec == ISVD_FP64 ? 1e-12 : 1e-5);
  h->orth_every = cfg->orth_every > 0 ? cfg->orth_every : (cfg->prec == ISVD_FP64 ? 0 : 256);
  h->row_cap = std::max<int64_t>(cfg->row_cap > 0 ? cfg->row_cap : 2 * m0, m0 + 1);
  h->col_cap = std::max<int64_t>(cfg->col_cap > 0 ? cfg->col_cap : 2 * n0, n0 + 1);
  h->rsvd_p = cfg->rsvd_oversample > 0 ? cfg->rsvd_oversample : 16;
  h->rsvd_q = cfg->rsvd_power_iters >= 0 ? cfg->rsvd_power_iters : 2;
  h->seed = cfg->seed;
  if (!on_dev) {
    bool ok = true;
    for (int64_t i = 0; i < m0 && ok; ++i)
      ok = h->prec == ISVD_FP64 ? host_finite((const double*)A0 + i * lda, n0) : host_finite((const float*)A0 + i * lda, n0);
    if (!ok) {
      delete h;
      return ISVD_ENONFINITE;
    }
  }
  isvd_status s = h->prec == ISVD_FP64 ? create_impl<double>(h, A0, m0, n0, lda, k, on_dev, U0, S0, V0)
                                       : create_impl<float>(h, A0, m0, n0, lda, k, on_dev, U0, S0, V0);
  if (s != ISVD_OK) {
    fprintf(stderr, "isvd_create: %s\n", h->err.c_str());
    isvd_destroy(h);
    return s;
  }
  *out = h;
  return ISVD_OK;
}

isvd_status isvd_create(const isvd_config* cfg, const void* A0, int64_t m0, int64_t n0, int64_t lda, int k,
                        int a0_on_device, isvd_t* out) {
  return create_common(cfg, A0, m0, n0, lda, k, a0_on_device, nullptr, nullptr, nullptr, 0, out);
}

isvd_status isvd_create_from_factors(const isvd_config* cfg, const void* A0, int64_t m0, int64_t n0, int64_t lda,
                                     const void* U0, const double* sigma0, const void* V0, int r0, int k,
                                     int on_device, isvd_t* out) {
  if (!U0) return ISVD_EINVAL;
  return create_common(cfg, A0, m0, n0, lda, k, on_device, U0, sigma0, V0, r0, out);
}

void isvd_destroy(isvd_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  void* bufs[] = {h->U, h->V, h->A, h->Uref, h->st, h->sig, h->p, h->part, h->UK, h->VK, h->xbuf, h->G,
                  h->small, h->evals, h->inv, h->scal, h->info, h->Rtmp, h->Uopt, h->Vopt, h->sig_opt, h->Cbuf,
                  h->Yb, h->Om, h->Zd, h->Rl, h->wbuf, h->riskbuf, h->RU, h->RV, h->gq};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

static isvd_status append_common(isvd_t h, int kind, const void* v, int64_t len, int on_device) {
  if (!h || !v) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  const int64_t want = kind == kRow ? h->n : h->m;
  if (len != want) return fail(h, ISVD_ESHAPE, "vector length " + std::to_string(len) + " != " + std::to_string(want));
  if (!on_device) {
    const bool ok = h->prec == ISVD_FP64 ? host_finite((const double*)v, len) : host_finite((const float*)v, len);
    if (!ok) return fail(h, ISVD_ENONFINITE, "non-finite value in the appended vector");
  }
  const void* dv = nullptr;
  isvd_status s = stage(h, v, len, on_device, &dv);
  if (s) return s;
  s = h->prec == ISVD_FP64 ? do_append<double>(h, kind, (const double*)dv) : do_append<float>(h, kind, (const float*)dv);
  if (s) return s;
  return h->prec == ISVD_FP64 ? after_update<double>(h) : after_update<float>(h);
}

isvd_status isvd_append_row(isvd_t h, const void* x, int64_t n, int on_device) {
  return append_common(h, kRow, x, n, on_device);
}

isvd_status isvd_append_col(isvd_t h, const void* y, int64_t m, int on_device) {
  return append_common(h, kCol, y, m, on_device);
}

isvd_status isvd_update_entry(isvd_t h, int64_t i, int64_t j, double delta) {
  if (!h) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  if (i < 0 || i >= h->m || j < 0 || j >= h->n) return fail(h, ISVD_EBOUNDS, "entry index out of range");
  if (!std::isfinite(delta)) return fail(h, ISVD_ENONFINITE, "non-finite delta");
  isvd_status s = h->prec == ISVD_FP64 ? do_entry<double>(h, i, j, delta) : do_entry<float>(h, i, j, delta);
  if (s) return s;
  return h->prec == ISVD_FP64 ? after_update<double>(h) : after_update<float>(h);
}

isvd_status isvd_update_entry_exact(isvd_t h, int64_t i, int64_t j, double delta) {
  if (!h) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  if (i < 0 || i >= h->m || j < 0 || j >= h->n) return fail(h, ISVD_EBOUNDS, "entry index out of range");
  if (!std::isfinite(delta)) return fail(h, ISVD_ENONFINITE, "non-finite delta");
  isvd_status s = h->prec == ISVD_FP64 ? do_entry_exact<double>(h, i, j, delta) : do_entry_exact<float>(h, i, j, delta);
  if (s) return s;
  return h->prec == ISVD_FP64 ? after_update<double>(h) : after_update<float>(h);
}

isvd_status isvd_set_deferred_rotations(isvd_t h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  if (h->orth_on_device) return fail(h, ISVD_EINVAL, "deferred rotations serve single streams, not pool streams");
  isvd_status s;
  if (!enable) {
    if ((s = materialize_any(h))) return s;
    h->defer = 0;
    return ISVD_OK;
  }
  if (!h->RU) {
    const size_t bytes = (size_t)h->kmax * h->ld * h->es;
    if ((s = dmalloc(h, &h->RU, bytes))) return s;
    if ((s = dmalloc(h, &h->RV, bytes))) {
      cudaFree(h->RU);
      h->RU = nullptr;
      return s;
    }
  }
  h->defer = 1;
  return ISVD_OK;
}

int isvd_deferred_pending(isvd_t h) { return h ? h->defer_pending : 0; }

isvd_status isvd_apply_events(isvd_t h, const isvd_event* ev, int64_t nev, const void* payload, int64_t payload_len,
                              int payload_on_device) {
  if (!h || (nev > 0 && !ev)) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  isvd_status s;
  const char* base = (const char*)payload;
  if (!payload_on_device && payload_len > 0) {
    // One host-to-device copy of the whole payload; the events then read it in place.
    const bool ok = h->prec == ISVD_FP64 ? host_finite((const double*)payload, payload_len)
                                         : host_finite((const float*)payload, payload_len);
    if (!ok) return fail(h, ISVD_ENONFINITE, "non-finite value in the event payload");
    if ((s = ensure_buf(h, &h->xbuf, &h->xbuf_cap, payload_len * (int64_t)h->es))) return s;
    CK(h, cudaMemcpyAsync(h->xbuf, payload, (size_t)payload_len * h->es, cudaMemcpyHostToDevice, h->stream));
    base = (const char*)h->xbuf;
  }
  for (int64_t e = 0; e < nev; ++e) {
    const isvd_event& E = ev[e];
    if (E.kind == kEntry) {
      if ((s = isvd_update_entry(h, E.i, E.j, E.delta))) return s;
      continue;
    }
    if (E.kind != kRow && E.kind != kCol) return fail(h, ISVD_EINVAL, "unknown event kind");
    const int64_t want = E.kind == kRow ? h->n : h->m;
    if (E.len != want) return fail(h, ISVD_ESHAPE, "event vector length mismatch");
    if (E.off < 0 || E.off + E.len > payload_len) return fail(h, ISVD_EBOUNDS, "event payload out of range");
    const void* dv = base + E.off * (int64_t)h->es;
    s = h->prec == ISVD_FP64 ? do_append<double>(h, E.kind, (const double*)dv) : do_append<float>(h, E.kind, (const float*)dv);
    if (s) return s;
    if ((s = (h->prec == ISVD_FP64 ? after_update<double>(h) : after_update<float>(h)))) return s;
  }
  return ISVD_OK;
}

isvd_status isvd_set_policy(isvd_t h, const isvd_policy* pol) {
  if (!h) return ISVD_EINVAL;
  if (!pol) {
    if (h->has_pol && (h->pol.kind & ISVD_POLICY_NOVELTY_RANK)) {
      const int32_t off = 0;
      CK(h, cudaMemcpyAsync(&h->st->kcap_nov, &off, sizeof off, cudaMemcpyHostToDevice, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
    }
    h->has_pol = 0;
    return ISVD_OK;
  }
  if (pol->T_refresh < 0 || pol->T_min < 0 || pol->check_every < 0) return ISVD_EINVAL;
  if (pol->kind & ~(ISVD_POLICY_PERIODIC | ISVD_POLICY_ERROR | ISVD_POLICY_ANGLE | ISVD_POLICY_ADAPTIVE_RANK |
                    ISVD_POLICY_NOVELTY_RANK | ISVD_POLICY_RANK_SHRINK))
    return fail(h, ISVD_EINVAL, "unknown policy kind bit");
  if ((pol->kind & ISVD_POLICY_RANK_SHRINK) && !(pol->tau_shrink > 0.0 && pol->tau_shrink <= 1.0))
    return fail(h, ISVD_EINVAL, "shrink threshold tau_shrink not in (0, 1]");
  if (pol->k_max > h->kmax) return fail(h, ISVD_EINVAL, "policy k_max exceeds the handle's k_max");
  const bool nov = (pol->kind & ISVD_POLICY_NOVELTY_RANK) != 0;
  if (nov && !(pol->eta > 0.0 && pol->eta < 1.0)) return fail(h, ISVD_EINVAL, "novelty threshold eta not in (0, 1)");
  // The novelty rule is decided on the device, right after each append's core.
  const double eta = nov ? pol->eta : 0.0;
  const int32_t kcap = nov ? (pol->k_max > 0 ? pol->k_max : h->kmax) : 0;
  CK(h, cudaMemcpyAsync(&h->st->eta_nov, &eta, sizeof eta, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(&h->st->kcap_nov, &kcap, sizeof kcap, cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->pol = *pol;
  h->has_pol = 1;
  return ISVD_OK;
}

isvd_status isvd_refresh(isvd_t h, int store_initial_subspace) {
  if (!h) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  return h->prec == ISVD_FP64 ? do_refresh<double>(h, store_initial_subspace) : do_refresh<float>(h, store_initial_subspace);
}

isvd_status isvd_metrics(isvd_t h, int flags, isvd_metrics_t* out) {
  if (!h || !out) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  if (flags & ~ISVD_METRICS_FULL) return ISVD_EINVAL;
  return h->prec == ISVD_FP64 ? do_metrics<double>(h, flags, out) : do_metrics<float>(h, flags, out);
}

isvd_status isvd_last_check_metrics(isvd_t h, isvd_metrics_t* out) {
  if (!h || !out) return ISVD_EINVAL;
  *out = h->last_check;
  return ISVD_OK;
}

isvd_status isvd_get_shape(isvd_t h, int64_t* m, int64_t* n, int32_t* r, int32_t* k) {
  if (!h) return ISVD_EINVAL;
  DevState ds;
  isvd_status s = read_state(h, &ds);
  if (s) return s;
  if (m) *m = h->m;
  if (n) *n = h->n;
  if (r) *r = ds.r;
  if (k) *k = ds.k;
  return ISVD_OK;
}

isvd_status isvd_get_factors(isvd_t h, void* U, double* sigma, void* V, int to_device) {
  if (!h) return ISVD_EINVAL;
  DevState ds;
  isvd_status s = (U || V) ? materialize_any(h) : ISVD_OK;
  if (s) return s;
  if ((s = read_state(h, &ds))) return s;
  const int r = ds.r;
  const cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (U) CK(h, cudaMemcpy2DAsync(U, r * h->es, h->U, h->ld * h->es, r * h->es, h->m, kind, h->stream));
  if (V) CK(h, cudaMemcpy2DAsync(V, r * h->es, h->V, h->ld * h->es, r * h->es, h->n, kind, h->stream));
  if (sigma) CK(h, cudaMemcpyAsync(sigma, h->sig, r * 8, to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return ISVD_OK;
}

isvd_status isvd_get_matrix(isvd_t h, void* A, int to_device) {
  if (!h || !A) return ISVD_EINVAL;
  const cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(h, cudaMemcpy2DAsync(A, h->n * h->es, h->A, h->col_cap * h->es, h->n * h->es, h->m, kind, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return ISVD_OK;
}

isvd_status isvd_reorthogonalize(isvd_t h, int force, double* err_u, double* err_v) {
  if (!h) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  return h->prec == ISVD_FP64 ? do_reorth<double>(h, force, err_u, err_v) : do_reorth<float>(h, force, err_u, err_v);
}

isvd_status isvd_risk(isvd_t h, const void* w, int w_on_device, int flags, isvd_risk_t* out) {
  if (!h || !out || (flags & ~ISVD_RISK_FULL)) return ISVD_EINVAL;
  if (h->sticky) return (isvd_status)h->sticky;
  if (w && !w_on_device) {
    const bool ok = h->prec == ISVD_FP64 ? host_finite((const double*)w, h->n) : host_finite((const float*)w, h->n);
    if (!ok) return fail(h, ISVD_ENONFINITE, "non-finite portfolio weight");
  }
  return h->prec == ISVD_FP64 ? do_risk<double>(h, w, w_on_device, flags, out)
                              : do_risk<float>(h, w, w_on_device, flags, out);
}

isvd_status isvd_sync(isvd_t h) {
  if (!h) return ISVD_EINVAL;
  DevState ds;
  return read_state(h, &ds);
}

int64_t isvd_kernel_launches(isvd_t h) { return h ? h->launches : 0; }

#ifdef ISVD_CORE_TIMING
int isvd_debug_core_clock(long long* out) {
  return (int)cudaMemcpyFromSymbol(out, isvd_core_clock, sizeof(long long) * 16);
}
int isvd_debug_clock_sums(unsigned long long* out, int reset) {
  int e = (int)cudaMemcpyFromSymbol(out, isvd_core_clock_sum, sizeof(unsigned long long) * 32);
  if (!e) e = (int)cudaMemcpyFromSymbol(out + 32, isvd_core_clock_cnt, sizeof(unsigned long long) * 32);
  if (!e && reset) {
    unsigned long long z[32] = {};
    e = (int)cudaMemcpyToSymbol(isvd_core_clock_sum, z, sizeof(z));
    if (!e) e = (int)cudaMemcpyToSymbol(isvd_core_clock_cnt, z, sizeof(z));
  }
  return e;
}
#endif

isvd_status isvd_profile(isvd_t h, int enable) {
  if (!h) return ISVD_EINVAL;
  prof_flush(h);
  h->prof = enable ? 1 : 0;
  for (int c = 0; c < ISVD_NUM_KCLASS; ++c) {
    h->cls_ms[c] = 0;
    h->cls_bytes[c] = 0;
    h->cls_n[c] = 0;
  }
  h->lat_us.clear();
  h->stamps.clear();
  h->spans.clear();
  h->ev_used = 0;
  if (h->prof) prof_stamp(h);
  return ISVD_OK;
}

isvd_status isvd_profile_read(isvd_t h, int cls, double* total_ms, double* bytes, int64_t* launches) {
  if (!h || cls < 0 || cls >= ISVD_NUM_KCLASS) return ISVD_EINVAL;
  prof_flush(h);
  if (total_ms) *total_ms = h->cls_ms[cls];
  if (bytes) *bytes = h->cls_bytes[cls];
  if (launches) *launches = h->cls_n[cls];
  return ISVD_OK;
}

isvd_status isvd_latencies(isvd_t h, double* us, int64_t cap, int64_t* count) {
  if (!h || !count) return ISVD_EINVAL;
  prof_flush(h);
  const int64_t n = (int64_t)h->lat_us.size();
  *count = n;
  if (us) memcpy(us, h->lat_us.data(), sizeof(double) * (size_t)std::min(n, cap));
  return ISVD_OK;
}

const char* isvd_last_error(isvd_t h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"

// ---- batched pool of streams ----------------------------------------------------------------

struct isvd_pool_ctx {
  int kmax = 32, kb = 32;
  int flags = 0;
  int64_t orth_every = 256;  // <= 0: no monitor
  double orth_tol = 1e-5;
  PoolReorthOp* reorth_dev = nullptr;  // per submit: the monitor's stream list of every tick
  // Completion records (ISVD_POOL_COMPLETIONS): written per tick into comp_dev, copied per submit
  // into a pinned batch; isvd_pool_poll hands out batches whose event has completed.
  int64_t seq_next = 0;
  PoolCompletion* comp_dev = nullptr;
  int64_t comp_cap = 0;
  struct CompBatch {
    PoolCompletion* host = nullptr;
    int64_t cap = 0, count = 0, taken = 0;
    cudaEvent_t ev = nullptr;
  };
  std::deque<CompBatch> comp_q;
  std::vector<CompBatch> comp_free;
  // Per-slot device tables of the streams' sigma and state pointers (sigma gather); released
  // slots point at zeroed stand-ins.
  const double** tab_sig = nullptr;
  const DevState** tab_st = nullptr;
  int64_t tab_cap = 0;
  double* zero_sig = nullptr;
  DevState* zero_st = nullptr;
  double* gather_dev = nullptr;
  int64_t gather_cap = 0;
  int* status_dev = nullptr;   // every slot's status word (isvd_pool_sync), device and pinned host
  int* status_host = nullptr;
  int64_t status_cap = 0;
  int* kcheck = nullptr;       // the pool kernels' self-check word: first failing check (code, detail)
  int* kcheck_host = nullptr;  // its pinned copy, read at isvd_pool_sync
  // Tensor maps (CUtensorMap, 128 bytes) of every slot's U and V for the tensor-core rotations
  // (TMA loads of 128-row boxes, swizzled), rebuilt when a stream's U or V is reallocated.
  CUtensorMap* tmaps_dev = nullptr;
  int64_t tmaps_cap = 0;  // slots
  std::vector<const void*> tmap_u, tmap_v;  // the base addresses the maps were built for
  int64_t reorth_cap = 0;
  int64_t reorth_runs = 0;
  // Streams whose monitor is due; checked together once a full wave of them has gathered (or one
  // of them is overdue by a whole cadence), so that the check costs one short launch per wave.
  std::vector<int32_t> reorth_pending;
  // Adaptive rank (rank_every > 0): streams due after each tick of a submit.
  int64_t rank_every = 0;
  double tau_evr = 0.9;
  double eta_nov = 0.0;  // novelty rank rule threshold (0: off)
  double tau_shrink = 0.0;  // shrink side of the rank rule (0: off)
  std::vector<PoolRankOp> v_rank;
  std::vector<int64_t> v_rank_start;
  PoolRankOp* rank_dev = nullptr;
  int64_t rank_cap = 0;
  std::vector<int64_t> reorth_due_t;  // per slot: pool tick at which the stream became due (-1: none)
  cudaStream_t stream = nullptr;
  int64_t budget = 0, used = 0, max_streams = 0;
  double tol_rel = 3e-6;
  isvd_config cfg{};
  std::vector<isvd_ctx*> streams;
  std::vector<int64_t> bytes;
  PoolOp* ops_dev = nullptr;
  int64_t ops_cap = 0;
  // Host staging of a submit's descriptors, double-buffered: a submit fills one slot while the
  // previous submit's copies from the other may still be pending, so the host waits only when it
  // runs two submits ahead of the device.
  struct Stage {
    PoolOp* ops = nullptr;
    int* chunks = nullptr;
    int64_t cap = 0;
    PoolReorthOp* reorth = nullptr;
    int64_t reorth_cap = 0;
    PoolRankOp* rank = nullptr;
    int64_t rank_cap = 0;
    cudaEvent_t copied = nullptr;
  } stage[2];
  int stage_cur = 0;
  void* payload = nullptr;
  int64_t payload_cap = 0;
  float* zbuf = nullptr;      // first-pass residuals of the appends' projection sides (PoolOp::z1)
  int64_t zbuf_cap = 0;       // elements
  int* retry_list = nullptr;  // per-tick list of warp-path updates handed to the CTA kernel
  int64_t retry_cap = 0;
  int* retry_n = nullptr;     // one counter per tick of a submit
  int64_t retry_n_cap = 0;
  void* rot_scratch = nullptr;  // per-update records from the warp kernel to the rotation kernel
  int64_t rot_cap = 0;          // updates
  int* chunks_dev = nullptr;  // first rotation block of each update (per bucket run)
  int64_t chunks_cap = 0;
  int* block_op = nullptr;  // rotation block -> update, written by the warp kernels
  int64_t block_op_cap = 0;
  // The rank buckets of a tick run concurrently on side streams (fork/join through events).
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_r[3] = {nullptr, nullptr, nullptr};
  int num_sms = 152;
  // Per-stream scratch of a submit (valid where s_gen == gen), so that a submit touches only the
  // streams it names, and each stream's fused-kernel bucket (set at admission).
  std::vector<int64_t> s_m, s_n;
  std::vector<uint32_t> s_gen;
  std::vector<int32_t> s_seen;
  std::vector<uint8_t> s_bucket;
  uint32_t gen = 0;
  std::vector<int32_t> touched;
  // Reused host scratch of a submit (no allocation per call once grown).
  std::vector<int32_t> v_tick_of;
  std::vector<int64_t> v_order, v_tick_start, v_tmp, v_fill, v_run_boff, v_reorth_start;
  std::vector<uint8_t> v_key;
  std::vector<char> v_fused;
  std::vector<int> v_run_blocks;
  std::vector<PoolReorthOp> v_reorth;
  int64_t launches = 0, ticks = 0, fused_ops = 0, fallback_ops = 0, warp_ops = 0;
  // Host time of submits by phase (validate, order, stage, enqueue), while profiling.
  double host_us[4] = {0, 0, 0, 0};
  int64_t host_submits = 0;
  // Optional per-class launch timing (isvd_pool_profile).
  int prof = 0;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
  std::vector<std::pair<int, size_t>> prof_spans;  // (class, index of the first of two events)
  std::string err;
};

namespace {

isvd_status pool_fail(isvd_pool_ctx* p, isvd_status s, const std::string& m) {
  p->err = m;
  return s;
}

// Profiling: an event pair around one launch on stream cs (nothing when profiling is off).
cudaEvent_t pool_prof_event(isvd_pool_ctx* p) {
  if (p->prof_used == p->prof_ev.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->prof_ev.push_back(e);
  }
  return p->prof_ev[p->prof_used++];
}
void pool_prof_begin(isvd_pool_ctx* p, cudaStream_t cs, int cls) {
  if (!p->prof) return;
  const size_t a = p->prof_used;
  cudaEvent_t e0 = pool_prof_event(p), e1 = pool_prof_event(p);
  if (!e0 || !e1) return;
  cudaEventRecord(e0, cs);
  p->prof_spans.push_back({cls, a});
}
void pool_prof_end(isvd_pool_ctx* p, cudaStream_t cs) {
  if (!p->prof || p->prof_spans.empty()) return;
  cudaEventRecord(p->prof_ev[p->prof_spans.back().second + 1], cs);
}

template <int KB>
isvd_status pool_launch(isvd_pool_ctx* p, const PoolOp* ops, int count) {
  pool_prof_begin(p, p->stream, ISVD_POOL_KCLASS_CTA);
  cudaError_t e = pool_tick_launch<KB>(count, p->stream, ops);
  pool_prof_end(p, p->stream);
  if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool tick launch: ") + cudaGetErrorString(e));
  p->launches++;
  return ISVD_OK;
}

// One warp-per-update launch over ops[0 .. count) of rank bucket KB: scr is the run's rotation
// scratch, hand-backs are listed in retry (as indexes into ops) and counted in *retry_n.
template <int KB>
isvd_status pool_launch_warp(isvd_pool_ctx* p, cudaStream_t cs, const PoolOp* ops, int count, void* scr, int* retry,
                             int* retry_n, const int* chunks, int* block_op, int nblocks) {
  pool_prof_begin(p, cs, KB == 8 ? ISVD_POOL_KCLASS_WARP8 : KB == 16 ? ISVD_POOL_KCLASS_WARP16 : ISVD_POOL_KCLASS_WARP32);
  cudaError_t e = pool_warp_launch(KB, count, cs, ops, 0, retry, retry_n, scr, chunks, block_op,
                                   pool_rot_rows(KB, (p->flags & ISVD_POOL_TC_ROTATIONS) != 0), nblocks, p->kcheck);
  pool_prof_end(p, cs);
  if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool warp launch: ") + cudaGetErrorString(e));
  p->launches++;
  return ISVD_OK;
}

// Row-parallel rotations of a bucket run (chunks = its first-block table, nblocks in total).
template <int KB>
isvd_status pool_launch_rotate(isvd_pool_ctx* p, cudaStream_t cs, const PoolOp* ops, const void* scr, const int* chunks,
                               const int* block_op, int nblocks, int count) {
  pool_prof_begin(p, cs, KB == 8 ? ISVD_POOL_KCLASS_ROT8 : KB == 16 ? ISVD_POOL_KCLASS_ROT16 : ISVD_POOL_KCLASS_ROT32);
  cudaError_t e = pool_rotate_launch(KB, nblocks, cs, ops, scr, chunks, block_op, (p->flags & ISVD_POOL_TC_ROTATIONS) != 0,
                                     p->tmaps_dev, count, (int)(2 * p->tmaps_cap), p->kcheck);
  pool_prof_end(p, cs);
  if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool rotate launch: ") + cudaGetErrorString(e));
  p->launches++;
  return ISVD_OK;
}

// The CTA kernel over the updates a warp launch handed back (ops = that launch's ops, retry and
// retry_n its hand-back list and count), on the launch's stream.
isvd_status pool_launch_retry(isvd_pool_ctx* p, cudaStream_t cs, const PoolOp* ops, int count, const int* retry,
                              const int* retry_n) {
  const int rblocks = std::min(count, p->num_sms);
  pool_prof_begin(p, cs, ISVD_POOL_KCLASS_RETRY);
  cudaError_t e = pool_retry_launch(rblocks, cs, ops, retry, retry_n);
  pool_prof_end(p, cs);
  if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool retry launch: ") + cudaGetErrorString(e));
  p->launches++;
  return ISVD_OK;
}

// Points slot id of the sigma-gather tables at (sig, st), growing the tables as needed.
isvd_status pool_set_slot(isvd_pool_ctx* p, int64_t id, const double* sig, const DevState* st) {
  if (id >= p->tab_cap) {
    const int64_t cap = std::max<int64_t>(id + 1, 2 * p->tab_cap);
    const double** ts = nullptr;
    const DevState** tt = nullptr;
    if (cudaMalloc((void**)&ts, sizeof(void*) * cap) != cudaSuccess ||
        cudaMalloc((void**)&tt, sizeof(void*) * cap) != cudaSuccess) {
      if (ts) cudaFree(ts);
      return pool_fail(p, ISVD_ENOMEM, "pool slot tables");
    }
    std::vector<const void*> zs(cap, p->zero_sig), zt(cap, p->zero_st);
    cudaStreamSynchronize(p->stream);
    if (p->tab_cap > 0) {
      cudaMemcpy(zs.data(), p->tab_sig, sizeof(void*) * p->tab_cap, cudaMemcpyDeviceToHost);
      cudaMemcpy(zt.data(), p->tab_st, sizeof(void*) * p->tab_cap, cudaMemcpyDeviceToHost);
    }
    cudaMemcpy(ts, zs.data(), sizeof(void*) * cap, cudaMemcpyHostToDevice);
    cudaMemcpy(tt, zt.data(), sizeof(void*) * cap, cudaMemcpyHostToDevice);
    if (p->tab_sig) cudaFree(p->tab_sig);
    if (p->tab_st) cudaFree(p->tab_st);
    p->tab_sig = ts;
    p->tab_st = tt;
    p->tab_cap = cap;
  }
  // Stream-ordered, so gathers queued earlier still see the old entry.
  if (cudaMemcpyAsync(p->tab_sig + id, &sig, sizeof(void*), cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(p->tab_st + id, &st, sizeof(void*), cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool slot tables");
  return ISVD_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time dependency).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

// A map over a rows x ld FP32 matrix (row-major) with boxes of kRowBoxRows rows of the full row
// width, swizzled by the row width (32-, 64- or 128-byte rows: the rank buckets 8, 16, 32 the
// rotation kernels serve) so that a thread reading its own staged row meets no bank conflicts;
// zeroed for other widths (never used).
bool encode_rows_map(CUtensorMap* m, const void* base, int64_t rows, int ld) {
  memset(m, 0, sizeof(*m));
  if (ld != 8 && ld != 16 && ld != 32) return true;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)ld, (cuuint32_t)kRowBoxRows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUtensorMapSwizzle sw = ld == 32   ? CU_TENSOR_MAP_SWIZZLE_128B
                                : ld == 16 ? CU_TENSOR_MAP_SWIZZLE_64B
                                           : CU_TENSOR_MAP_SWIZZLE_32B;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// (Re)builds slot id's two maps if its U or V moved; the pool's stream must be idle for this slot
// (admission, or right after a reallocation, which synchronises).
isvd_status pool_set_maps(isvd_pool_ctx* p, int64_t id, const isvd_ctx* h) {
  if (id >= p->tmaps_cap) {
    const int64_t cap = std::max<int64_t>(id + 1, 2 * p->tmaps_cap);
    CUtensorMap* d = nullptr;
    if (cudaMalloc((void**)&d, sizeof(CUtensorMap) * 2 * (size_t)cap) != cudaSuccess)
      return pool_fail(p, ISVD_ENOMEM, "pool tensor maps");
    cudaStreamSynchronize(p->stream);
    if (p->tmaps_dev) {
      cudaMemcpy(d, p->tmaps_dev, sizeof(CUtensorMap) * 2 * (size_t)p->tmaps_cap, cudaMemcpyDeviceToDevice);
      cudaFree(p->tmaps_dev);
    }
    p->tmaps_dev = d;
    p->tmaps_cap = cap;
    p->tmap_u.resize(cap, nullptr);
    p->tmap_v.resize(cap, nullptr);
  }
  if (p->tmap_u[id] == h->U && p->tmap_v[id] == h->V) return ISVD_OK;
  CUtensorMap m[2];
  if (!encode_rows_map(&m[0], h->U, h->row_cap, h->ld) || !encode_rows_map(&m[1], h->V, h->col_cap, h->ld))
    return pool_fail(p, ISVD_ECUDA, "cuTensorMapEncodeTiled failed");
  if (cudaMemcpy(p->tmaps_dev + 2 * id, m, sizeof m, cudaMemcpyHostToDevice) != cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool tensor map copy");
  p->tmap_u[id] = h->U;
  p->tmap_v[id] = h->V;
  return ISVD_OK;
}

int64_t stream_footprint(int64_t row_cap, int64_t col_cap, int ld) {
  // U, V, U_ref and A in FP32 plus the handle's fixed workspace (the 128 bucket's core scratch
  // included: ld > 64).
  const int64_t fixed = (int64_t)6 * (kKmaxLimit + 1) * (kKmaxLimit + 1) * 8 + (int64_t)kMaxProjBlocks * kPartStride * 8 +
                        (int64_t)4 * (kKmaxLimit + 2) * ld * 4 +
                        (ld > kFastCoreQSmemMaxKB ? (int64_t)(kKmaxLimit + 1) * (kKmaxLimit + 1) * 4 : 0);
  return (2 * row_cap * ld + col_cap * ld + row_cap * col_cap) * 4 + fixed;
}

}  // namespace

extern "C" {

isvd_status isvd_pool_create(const isvd_pool_config* cfg, isvd_pool_t* out) {
  if (!cfg || !out) return ISVD_EINVAL;
  *out = nullptr;
  if (cfg->k_max < 1 || cfg->k_max > kKmaxLimit) return ISVD_EINVAL;
  if (cfg->flags & ~(ISVD_POOL_TC_ROTATIONS | ISVD_POOL_COMPLETIONS | ISVD_POOL_DEVICE_CHECKS)) return ISVD_EINVAL;
  if (!(cfg->eta_novelty == 0.0 || (cfg->eta_novelty > 0.0 && cfg->eta_novelty < 1.0))) return ISVD_EINVAL;
  if (!(cfg->tau_shrink == 0.0 || (cfg->tau_shrink > cfg->tau_evr && cfg->tau_shrink <= 1.0))) return ISVD_EINVAL;
  isvd_pool_ctx* p = new isvd_pool_ctx();
  p->kmax = cfg->k_max;
  p->kb = kb_bucket(cfg->k_max);
  p->stream = (cudaStream_t)cfg->cuda_stream;
  p->budget = cfg->hbm_budget_bytes;
  p->max_streams = cfg->max_streams > 0 ? cfg->max_streams : (int64_t)1 << 30;
  p->tol_rel = cfg->tol_rel > 0 ? cfg->tol_rel : 3e-6;
  p->flags = cfg->flags;
  p->orth_every = cfg->orth_every == 0 ? 256 : cfg->orth_every;
  p->orth_tol = cfg->orth_tol > 0 ? cfg->orth_tol : 1e-5;
  p->rank_every = cfg->rank_every > 0 ? cfg->rank_every : 0;
  p->tau_evr = cfg->tau_evr;
  p->eta_nov = cfg->eta_novelty;
  p->tau_shrink = cfg->tau_shrink;
  p->cfg.prec = ISVD_FP32;
  p->cfg.k_max = p->kmax;
  p->cfg.tol_rel = p->tol_rel;
  p->cfg.cuda_stream = cfg->cuda_stream;
  p->cfg.orth_every = (int64_t)1 << 62;  // the pool path runs no monitor; isvd_reorthogonalize on demand
  p->cfg.rsvd_power_iters = -1;
  cudaError_t e = pool_tick_set_attr<8>();
  if (e == cudaSuccess) e = pool_tick_set_attr<16>();
  if (e == cudaSuccess) e = pool_tick_set_attr<32>();
  if (e == cudaSuccess) e = pool_tick_set_attr<64>();
  if (e == cudaSuccess) e = pool_retry_set_attr();
  if (e == cudaSuccess) e = pool_warp_set_attrs();
  if (e == cudaSuccess) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_r[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->stage[i].copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->zero_sig, 8 * (kKmaxLimit + 2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->zero_st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemset(p->zero_sig, 0, 8 * (kKmaxLimit + 2));
  if (e == cudaSuccess) e = cudaMemset(p->zero_st, 0, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->kcheck, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->kcheck, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->kcheck_host, 2 * sizeof(int));
  if (e != cudaSuccess) {
    delete p;
    return ISVD_ECUDA;
  }
  *out = p;
  return ISVD_OK;
}

void isvd_pool_destroy(isvd_pool_t p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  for (isvd_ctx* h : p->streams)
    if (h) isvd_destroy(h);
  if (p->ops_dev) cudaFree(p->ops_dev);
  if (p->retry_list) cudaFree(p->retry_list);
  if (p->retry_n) cudaFree(p->retry_n);
  if (p->rot_scratch) cudaFree(p->rot_scratch);
  if (p->block_op) cudaFree(p->block_op);
  for (int i = 0; i < 3; ++i) {
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
    if (p->ev_r[i]) cudaEventDestroy(p->ev_r[i]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
  if (p->chunks_dev) cudaFree(p->chunks_dev);
  if (p->reorth_dev) cudaFree(p->reorth_dev);
  if (p->comp_dev) cudaFree(p->comp_dev);
  if (p->rank_dev) cudaFree(p->rank_dev);
  for (auto& b : p->comp_q) {
    if (b.host) cudaFreeHost(b.host);
    if (b.ev) cudaEventDestroy(b.ev);
  }
  for (auto& b : p->comp_free) {
    if (b.host) cudaFreeHost(b.host);
    if (b.ev) cudaEventDestroy(b.ev);
  }
  if (p->tab_sig) cudaFree(p->tab_sig);
  if (p->tab_st) cudaFree(p->tab_st);
  if (p->zero_sig) cudaFree(p->zero_sig);
  if (p->zero_st) cudaFree(p->zero_st);
  if (p->gather_dev) cudaFree(p->gather_dev);
  if (p->status_dev) cudaFree(p->status_dev);
  if (p->status_host) cudaFreeHost(p->status_host);
  if (p->kcheck) cudaFree(p->kcheck);
  if (p->kcheck_host) cudaFreeHost(p->kcheck_host);
  if (p->tmaps_dev) cudaFree(p->tmaps_dev);
  for (auto& sg : p->stage) {
    if (sg.ops) cudaFreeHost(sg.ops);
    if (sg.chunks) cudaFreeHost(sg.chunks);
    if (sg.reorth) cudaFreeHost(sg.reorth);
    if (sg.rank) cudaFreeHost(sg.rank);
    if (sg.copied) cudaEventDestroy(sg.copied);
  }
  if (p->payload) cudaFree(p->payload);
  if (p->zbuf) cudaFree(p->zbuf);
  delete p;
}

isvd_status isvd_pool_admit(isvd_pool_t p, const void* A0, int64_t m0, int64_t n0, int64_t lda, int k,
                            int64_t row_cap, int64_t col_cap, const void* U0, const double* sigma0, const void* V0,
                            int on_device, int32_t* stream_id) {
  if (!p || !A0 || !stream_id || k < 1 || k > p->kmax) return ISVD_EINVAL;
  int64_t live = 0;
  for (isvd_ctx* h : p->streams) live += h != nullptr;
  if (live >= p->max_streams) return pool_fail(p, ISVD_EBUDGET, "pool: stream slots exhausted");
  isvd_config c = p->cfg;
  // The stream's rank capacity is its fused-kernel bucket (8, 16, 32 or 64): U and V rows are then
  // exactly one bucket wide, which the batched kernels read as contiguous float4 arrays. The
  // working rank stays k.
  c.k_max = pool_bucket(k);
  c.row_cap = std::max<int64_t>(row_cap, m0 + 1);
  c.col_cap = std::max<int64_t>(col_cap, n0 + 1);
  const int64_t need = stream_footprint(c.row_cap, c.col_cap, c.k_max);
  if (p->budget > 0 && p->used + need > p->budget)
    return pool_fail(p, ISVD_EBUDGET, "pool: HBM budget exceeded (" + std::to_string(p->used + need) + " > " +
                                          std::to_string(p->budget) + " bytes)");
  isvd_t h = nullptr;
  const int r0 = (int)std::min<int64_t>(k, std::min(m0, n0));
  isvd_status s = U0 ? isvd_create_from_factors(&c, A0, m0, n0, lda, U0, sigma0, V0, r0, k, on_device, &h)
                     : isvd_create(&c, A0, m0, n0, lda, k, on_device, &h);
  if (s) return s;
  int32_t id = -1;
  for (size_t i = 0; i < p->streams.size(); ++i)
    if (!p->streams[i]) {
      id = (int32_t)i;
      break;
    }
  if (id < 0) {
    id = (int32_t)p->streams.size();
    p->streams.push_back(nullptr);
    p->bytes.push_back(0);
  }
  p->streams[id] = h;
  p->bytes[id] = need;
  // The batched monitor: streams start at staggered points of the cadence, so that admissions
  // made together are not all checked in the same tick.
  h->orth_on_device = 1;
  h->since_orth = p->orth_every > 0 ? ((int64_t)id * 37) % p->orth_every : 0;
  if ((s = pool_set_slot(p, id, h->sig, h->st))) return s;
  if ((s = pool_set_maps(p, id, h))) return s;
  if (p->s_gen.size() < p->streams.size()) {
    const size_t ns = p->streams.size();
    p->s_m.resize(ns);
    p->s_n.resize(ns);
    p->s_gen.resize(ns, 0);
    p->s_seen.resize(ns);
    p->s_bucket.resize(ns);
  }
  p->s_gen[id] = 0;
  p->s_bucket[id] = (uint8_t)pool_bucket(k);
  if (p->eta_nov > 0.0) {
    // The novelty rank rule, decided on the device after each append, up to the stream's capacity.
    const double eta = p->eta_nov;
    const int32_t kcap = std::min<int32_t>(p->s_bucket[id], p->kmax);
    if (cudaMemcpyAsync(&h->st->eta_nov, &eta, sizeof eta, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(&h->st->kcap_nov, &kcap, sizeof kcap, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool novelty rule");
  }
  p->used += need;
  *stream_id = id;
  return ISVD_OK;
}

isvd_status isvd_pool_release(isvd_pool_t p, int32_t sid) {
  if (!p || sid < 0 || sid >= (int32_t)p->streams.size() || !p->streams[sid]) return ISVD_EINVAL;
  cudaStreamSynchronize(p->stream);
  isvd_destroy(p->streams[sid]);
  p->streams[sid] = nullptr;
  pool_set_slot(p, sid, p->zero_sig, p->zero_st);
  if (sid < (int64_t)p->tmap_u.size()) p->tmap_u[sid] = p->tmap_v[sid] = nullptr;
  if (sid < (int32_t)p->reorth_due_t.size() && p->reorth_due_t[sid] >= 0) {
    p->reorth_due_t[sid] = -1;
    p->reorth_pending.erase(std::find(p->reorth_pending.begin(), p->reorth_pending.end(), sid));
  }
  p->used -= p->bytes[sid];
  p->bytes[sid] = 0;
  return ISVD_OK;
}

isvd_t isvd_pool_stream(isvd_pool_t p, int32_t sid) {
  if (!p || sid < 0 || sid >= (int32_t)p->streams.size()) return nullptr;
  return p->streams[sid];
}

int64_t isvd_pool_bytes_used(isvd_pool_t p) { return p ? p->used : 0; }

int64_t isvd_pool_kernel_launches(isvd_pool_t p) { return p ? p->launches : 0; }

isvd_status isvd_pool_profile(isvd_pool_t p, int enable) {
  if (!p) return ISVD_EINVAL;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return pool_fail(p, ISVD_ECUDA, "pool profile");
  p->prof = enable ? 1 : 0;
  if (enable) {
    p->prof_used = 0;
    p->prof_spans.clear();
    for (double& v : p->host_us) v = 0.0;
    p->host_submits = 0;
  }
  return ISVD_OK;
}

isvd_status isvd_pool_host_profile(isvd_pool_t p, double* us_out, int n, int64_t* submits) {
  if (!p || !us_out || n < 0 || n > 4) return ISVD_EINVAL;
  for (int i = 0; i < n; ++i) us_out[i] = p->host_us[i];
  if (submits) *submits = p->host_submits;
  return ISVD_OK;
}

isvd_status isvd_pool_profile_read(isvd_pool_t p, double* ms_out, int64_t* launches_out, int n) {
  if (!p || !ms_out || !launches_out || n < 0 || n > ISVD_POOL_NUM_KCLASS) return ISVD_EINVAL;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return pool_fail(p, ISVD_ECUDA, "pool profile read");
  for (int c = 0; c < n; ++c) {
    ms_out[c] = 0.0;
    launches_out[c] = 0;
  }
  for (const auto& sp : p->prof_spans) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->prof_ev[sp.second], p->prof_ev[sp.second + 1]) != cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool profile read");
    if (sp.first < n) {
      ms_out[sp.first] += ms;
      launches_out[sp.first] += 1;
    }
  }
  return ISVD_OK;
}

isvd_status isvd_pool_submit(isvd_pool_t p, const isvd_op* ops, int64_t nops, const void* payload,
                             int64_t payload_len, int payload_on_device) {
  if (!p || (nops > 0 && !ops)) return ISVD_EINVAL;
  if (nops == 0) return ISVD_OK;
  const size_t es = 4;
  using clk = std::chrono::steady_clock;
  const auto h0 = clk::now();
  // Validate every op against the shapes it will see (per-stream order), before any work. Only
  // the streams named by the ops are read (their shapes into the pool's per-stream scratch).
  if (++p->gen == 0) {
    std::fill(p->s_gen.begin(), p->s_gen.end(), 0u);
    p->gen = 1;
  }
  const uint32_t gen = p->gen;
  std::vector<int64_t>& mm = p->s_m;
  std::vector<int64_t>& nn = p->s_n;
  std::vector<int32_t>& seen = p->s_seen;
  p->touched.clear();
  std::vector<int32_t>& tick_of = p->v_tick_of;
  tick_of.resize(nops);
  int32_t nticks = 0;
  for (int64_t e = 0; e < nops; ++e) {
    const isvd_op& o = ops[e];
    if (o.stream < 0 || o.stream >= (int32_t)p->streams.size() || !p->streams[o.stream])
      return pool_fail(p, ISVD_EINVAL, "pool op " + std::to_string(e) + ": unknown stream");
    const int32_t sid = o.stream;
    if (p->s_gen[sid] != gen) {
      const isvd_ctx* h = p->streams[sid];
      if (h->sticky) return (isvd_status)h->sticky;
      p->s_gen[sid] = gen;
      mm[sid] = h->m;
      nn[sid] = h->n;
      seen[sid] = 0;
      p->touched.push_back(sid);
    }
    if (o.kind == kEntry) {
      if (o.i < 0 || o.i >= mm[sid] || o.j < 0 || o.j >= nn[sid] || !std::isfinite(o.delta))
        return pool_fail(p, ISVD_EBOUNDS, "pool op " + std::to_string(e) + ": entry out of range");
    } else if (o.kind == kRow || o.kind == kCol) {
      const int64_t want = o.kind == kRow ? nn[sid] : mm[sid];
      if (o.len != want) return pool_fail(p, ISVD_ESHAPE, "pool op " + std::to_string(e) + ": length mismatch");
      if (o.off < 0 || o.off + o.len > payload_len) return pool_fail(p, ISVD_EBOUNDS, "pool op payload out of range");
      if (o.kind == kRow) mm[sid]++;
      else nn[sid]++;
    } else {
      return pool_fail(p, ISVD_EINVAL, "pool op: unknown kind");
    }
    tick_of[e] = seen[sid]++;
    nticks = std::max(nticks, tick_of[e] + 1);
  }
  if (!payload_on_device && payload_len > 0 && !(p->flags & ISVD_POOL_DEVICE_CHECKS) &&
      !host_finite((const float*)payload, payload_len))
    return pool_fail(p, ISVD_ENONFINITE, "pool payload has non-finite values");
  const float* pay = (const float*)payload;
  if (!payload_on_device && payload_len > 0) {
    if (payload_len * (int64_t)es > p->payload_cap) {
      cudaStreamSynchronize(p->stream);
      if (p->payload) cudaFree(p->payload);
      p->payload = nullptr;
      p->payload_cap = std::max(payload_len * (int64_t)es, 2 * p->payload_cap);
      if (cudaMalloc(&p->payload, (size_t)p->payload_cap) != cudaSuccess) {
        p->payload_cap = 0;
        return pool_fail(p, ISVD_ENOMEM, "pool payload buffer");
      }
    }
    if (cudaMemcpyAsync(p->payload, payload, (size_t)payload_len * es, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool payload copy");
    pay = (const float*)p->payload;
  }
  if (payload_len > p->zbuf_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->zbuf) cudaFree(p->zbuf);
    p->zbuf = nullptr;
    p->zbuf_cap = std::max(payload_len, 2 * p->zbuf_cap);
    if (cudaMalloc((void**)&p->zbuf, sizeof(float) * (size_t)p->zbuf_cap) != cudaSuccess) {
      p->zbuf_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool residual buffer");
    }
  }
  const auto h1 = clk::now();
  // Order ops by tick (stable), build descriptors, then one descriptor copy for all ticks.
  std::vector<int64_t>& order = p->v_order;
  std::vector<int64_t>& tick_start = p->v_tick_start;
  order.resize(nops);
  tick_start.assign(nticks + 1, 0);
  for (int64_t e = 0; e < nops; ++e) tick_start[tick_of[e] + 1]++;
  for (int32_t t = 0; t < nticks; ++t) tick_start[t + 1] += tick_start[t];
  {
    std::vector<int64_t>& fill = p->v_fill;
    fill.assign(tick_start.begin(), tick_start.end() - 1);
    for (int64_t e = 0; e < nops; ++e) order[fill[tick_of[e]]++] = e;
    // Within a tick: first the appends of rank capacity <= 32 (one warp-per-update launch, the
    // widest buckets first so the longest updates start first), then the CTA kernel's updates
    // grouped by rank bucket (one launch per bucket, the narrowest instance that fits).
    // Counting sort (stable) on a small key: 0-2 warp buckets 32/16/8, 3-6 CTA buckets 8-64, 7
    // bucket 128 (single-stream kernels).
    std::vector<uint8_t>& key = p->v_key;
    key.resize(nops);
    for (int64_t e = 0; e < nops; ++e) {
      const int b = p->s_bucket[ops[e].stream];
      const int lb = b == 8 ? 0 : b == 16 ? 1 : b == 32 ? 2 : b == 64 ? 3 : 4;
      key[e] = (uint8_t)((ops[e].kind != kEntry && b <= kWarpKB) ? 2 - lb : 3 + lb);
    }
    std::vector<int64_t>& tmp = p->v_tmp;
    tmp.resize(nops);
    for (int32_t t = 0; t < nticks; ++t) {
      int64_t cnt[9] = {};
      for (int64_t z = tick_start[t]; z < tick_start[t + 1]; ++z) cnt[key[order[z]] + 1]++;
      for (int k = 1; k < 9; ++k) cnt[k] += cnt[k - 1];
      for (int64_t z = tick_start[t]; z < tick_start[t + 1]; ++z) tmp[tick_start[t] + cnt[key[order[z]]]++] = order[z];
      std::copy(tmp.begin() + tick_start[t], tmp.begin() + tick_start[t + 1], order.begin() + tick_start[t]);
    }
  }
  const auto h2 = clk::now();
  // This submit's staging slot: its previous user's copies (two submits ago) must have finished.
  isvd_pool_ctx::Stage& sg = p->stage[p->stage_cur];
  p->stage_cur ^= 1;
  cudaEventSynchronize(sg.copied);
  if (nops > sg.cap) {
    if (sg.ops) cudaFreeHost(sg.ops);
    if (sg.chunks) cudaFreeHost(sg.chunks);
    sg.ops = nullptr;
    sg.chunks = nullptr;
    sg.cap = std::max<int64_t>(nops, 2 * sg.cap);
    if (cudaMallocHost((void**)&sg.ops, sizeof(PoolOp) * (size_t)sg.cap) != cudaSuccess ||
        cudaMallocHost((void**)&sg.chunks, sizeof(int) * (size_t)sg.cap) != cudaSuccess) {
      sg.cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool pinned descriptors");
    }
  }
  if (nops > p->ops_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->ops_dev) cudaFree(p->ops_dev);
    p->ops_cap = std::max<int64_t>(nops, 2 * p->ops_cap);
    if (cudaMalloc((void**)&p->ops_dev, sizeof(PoolOp) * (size_t)p->ops_cap) != cudaSuccess) {
      p->ops_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool descriptors");
    }
  }
  int64_t tick_max = 0;
  for (int32_t t = 0; t < nticks; ++t) tick_max = std::max(tick_max, tick_start[t + 1] - tick_start[t]);
  if (tick_max > p->retry_cap || 3 * nticks > p->retry_n_cap) {
    cudaStreamSynchronize(p->stream);
    if (tick_max > p->retry_cap) {
      if (p->retry_list) cudaFree(p->retry_list);
      p->retry_list = nullptr;
      p->retry_cap = std::max<int64_t>(tick_max, 2 * p->retry_cap);
      if (cudaMalloc((void**)&p->retry_list, 3 * sizeof(int) * (size_t)p->retry_cap) != cudaSuccess) {
        p->retry_cap = 0;
        return pool_fail(p, ISVD_ENOMEM, "pool retry list");
      }
    }
    if (3 * nticks > p->retry_n_cap) {
      if (p->retry_n) cudaFree(p->retry_n);
      p->retry_n = nullptr;
      p->retry_n_cap = std::max<int64_t>(3 * nticks, 2 * p->retry_n_cap);
      if (cudaMalloc((void**)&p->retry_n, sizeof(int) * (size_t)p->retry_n_cap) != cudaSuccess) {
        p->retry_n_cap = 0;
        return pool_fail(p, ISVD_ENOMEM, "pool retry counters");
      }
    }
  }
  if (tick_max > p->rot_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->rot_scratch) cudaFree(p->rot_scratch);
    p->rot_scratch = nullptr;
    p->rot_cap = std::max<int64_t>(tick_max, 2 * p->rot_cap);
    if (cudaMalloc(&p->rot_scratch, 3 * kRotScratchStride * (size_t)p->rot_cap) != cudaSuccess) {
      p->rot_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool rotation scratch");
    }
  }
  if (nops > p->chunks_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->chunks_dev) cudaFree(p->chunks_dev);
    p->chunks_dev = nullptr;
    p->chunks_cap = std::max<int64_t>(nops, 2 * p->chunks_cap);
    if (cudaMalloc((void**)&p->chunks_dev, sizeof(int) * (size_t)p->chunks_cap) != cudaSuccess) {
      p->chunks_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool rotation tables");
    }
  }
  isvd_status s;
  // Grow every named stream to its final shape for this submit BEFORE building descriptors, so
  // that no reallocation can invalidate a descriptor or copy data ahead of queued work.
  for (const int32_t sid : p->touched) {
    isvd_ctx* h = p->streams[sid];
    if ((s = ensure_rows(h, mm[sid] + 1))) return s;
    if ((s = ensure_cols(h, nn[sid] + 1))) return s;
    // a reallocation moved U or V (and synchronised the stream): rebuild the slot's maps
    if ((p->tmap_u[sid] != h->U || p->tmap_v[sid] != h->V) && (s = pool_set_maps(p, sid, h))) return s;
  }
  std::vector<char>& fused = p->v_fused;
  fused.assign(nops, 0);
  // Streams whose monitor is due, per tick (checked after that tick's updates).
  std::vector<PoolReorthOp>& reorth = p->v_reorth;
  std::vector<int64_t>& reorth_start = p->v_reorth_start;
  reorth.clear();
  reorth_start.assign(nticks + 1, 0);
  if ((int64_t)p->reorth_due_t.size() < (int64_t)p->streams.size()) p->reorth_due_t.resize(p->streams.size(), -1);
  std::vector<PoolRankOp>& rank = p->v_rank;
  std::vector<int64_t>& rank_start = p->v_rank_start;
  rank.clear();
  rank_start.assign(nticks + 1, 0);
  for (int32_t t = 0; t < nticks; ++t) {
    reorth_start[t] = (int64_t)reorth.size();
    rank_start[t] = (int64_t)rank.size();
    for (int64_t q = tick_start[t]; q < tick_start[t + 1]; ++q) {
      const int64_t e = order[q];
      const isvd_op& o = ops[e];
      isvd_ctx* h = p->streams[o.stream];
      const int bk = p->s_bucket[o.stream];
      if (o.kind != kEntry && bk <= kWarpKB) fused[q] = 2;  // warp per update
      else fused[q] = bk <= 64 ? 1 : 0;
      PoolOp& d = sg.ops[q];
      d.U = (float*)h->U;
      d.V = (float*)h->V;
      d.A = (float*)h->A;
      d.st = h->st;
      d.sig = h->sig;
      d.x = o.kind == kEntry ? nullptr : pay + o.off;
      d.z1 = o.kind == kEntry ? nullptr : p->zbuf + o.off;
      d.m = h->m;
      d.n = h->n;
      d.lda = h->col_cap;
      d.i = o.i;
      d.j = o.j;
      d.delta = o.delta;
      d.tol_rel = h->tol_rel;
      d.ld = h->ld;
      d.kind = o.kind;
      d.sid = o.stream;
      d.pad = 0;
      d.seq = p->seq_next + e;
      if (o.kind == kRow) h->m += 1;
      else if (o.kind == kCol) h->n += 1;
      h->t += 1;
      if (p->rank_every > 0 && ++h->since_rank >= p->rank_every) {
        h->since_rank = 0;
        rank.push_back(PoolRankOp{h->st, h->sig, std::min<int32_t>(p->s_bucket[o.stream], p->kmax), 0});
      }
      // Due at half the cadence; checked within another half (sooner once a wave has gathered).
      if (p->orth_every > 0 && ++h->since_orth >= (p->orth_every + 1) / 2 && p->reorth_due_t[o.stream] < 0) {
        p->reorth_due_t[o.stream] = p->ticks + t;
        p->reorth_pending.push_back(o.stream);
      }
    }
    // After this tick: check the pending streams once they fill a wave of CTAs, or when the oldest
    // has waited half a cadence, so that no stream goes longer than orth_every updates unchecked.
    const int64_t now = p->ticks + t;
    const bool full = (int64_t)p->reorth_pending.size() >= p->num_sms;
    const bool overdue =
        !p->reorth_pending.empty() && now - p->reorth_due_t[p->reorth_pending.front()] >= p->orth_every / 2;
    if (full || overdue) {
      for (const int32_t sid : p->reorth_pending) {
        isvd_ctx* h = p->streams[sid];
        reorth.push_back(PoolReorthOp{(float*)h->U, (float*)h->V, h->st, h->m, h->n, h->ld, 0});
        h->since_orth = 0;
        p->reorth_due_t[sid] = -1;
      }
      p->reorth_pending.clear();
    }
  }
  reorth_start[nticks] = (int64_t)reorth.size();
  rank_start[nticks] = (int64_t)rank.size();
  if ((int64_t)rank.size() > p->rank_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->rank_dev) cudaFree(p->rank_dev);
    p->rank_dev = nullptr;
    p->rank_cap = std::max<int64_t>((int64_t)rank.size(), 2 * p->rank_cap);
    if (cudaMalloc((void**)&p->rank_dev, sizeof(PoolRankOp) * (size_t)p->rank_cap) != cudaSuccess) {
      p->rank_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool rank list");
    }
  }
  if ((int64_t)rank.size() > sg.rank_cap) {
    if (sg.rank) cudaFreeHost(sg.rank);
    sg.rank = nullptr;
    sg.rank_cap = std::max<int64_t>((int64_t)rank.size(), 2 * sg.rank_cap);
    if (cudaMallocHost((void**)&sg.rank, sizeof(PoolRankOp) * (size_t)sg.rank_cap) != cudaSuccess) {
      sg.rank_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool rank list");
    }
  }
  if ((int64_t)reorth.size() > p->reorth_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->reorth_dev) cudaFree(p->reorth_dev);
    p->reorth_dev = nullptr;
    p->reorth_cap = std::max<int64_t>((int64_t)reorth.size(), 2 * p->reorth_cap);
    if (cudaMalloc((void**)&p->reorth_dev, sizeof(PoolReorthOp) * (size_t)p->reorth_cap) != cudaSuccess) {
      p->reorth_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool monitor list");
    }
  }
  if ((int64_t)reorth.size() > sg.reorth_cap) {
    if (sg.reorth) cudaFreeHost(sg.reorth);
    sg.reorth = nullptr;
    sg.reorth_cap = std::max<int64_t>((int64_t)reorth.size(), 2 * sg.reorth_cap);
    if (cudaMallocHost((void**)&sg.reorth, sizeof(PoolReorthOp) * (size_t)sg.reorth_cap) != cudaSuccess) {
      sg.reorth_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool monitor list");
    }
  }
  auto bucket_at = [&](int64_t z) { return (int)p->s_bucket[ops[order[z]].stream]; };
  // Rotation block tables of the warp-kernel runs (one run per tick and rank bucket):
  // chunks[q] = first block of update q within its run; run_blocks[first q of a run] = total.
  std::vector<int>& run_blocks = p->v_run_blocks;
  run_blocks.assign(nops, 0);
  for (int32_t t = 0; t < nticks; ++t) {
    int64_t q = tick_start[t];
    while (q < tick_start[t + 1]) {
      if (fused[q] != 2) {
        ++q;
        continue;
      }
      int64_t b1 = q;
      int tot = 0;
      while (b1 < tick_start[t + 1] && fused[b1] == 2 && bucket_at(b1) == bucket_at(q)) {
        const PoolOp& d = sg.ops[b1];
        const int64_t nP = d.kind == kRow ? d.n : d.m, nQ = d.kind == kRow ? d.m : d.n;
        const int rr = pool_rot_rows(bucket_at(q), (p->flags & ISVD_POOL_TC_ROTATIONS) != 0);
        sg.chunks[b1] = tot;
        tot += (int)((nP + rr - 1) / rr + (nQ + rr - 1) / rr);
        ++b1;
      }
      run_blocks[q] = tot;
      q = b1;
    }
  }
  // Each run's block -> update table sits at its own offset (runs of one tick run concurrently).
  std::vector<int64_t>& run_boff = p->v_run_boff;
  run_boff.assign(nops, 0);
  int64_t total_blocks = 0;
  for (int64_t q = 0; q < nops; ++q)
    if (run_blocks[q]) {
      run_boff[q] = total_blocks;
      total_blocks += run_blocks[q];
    }
  const bool completions = (p->flags & ISVD_POOL_COMPLETIONS) != 0;
  if (completions && nops > p->comp_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->comp_dev) cudaFree(p->comp_dev);
    p->comp_dev = nullptr;
    p->comp_cap = std::max<int64_t>(nops, 2 * p->comp_cap);
    if (cudaMalloc((void**)&p->comp_dev, sizeof(PoolCompletion) * (size_t)p->comp_cap) != cudaSuccess) {
      p->comp_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool completion records");
    }
  }
  if (total_blocks > p->block_op_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->block_op) cudaFree(p->block_op);
    p->block_op = nullptr;
    p->block_op_cap = std::max<int64_t>(total_blocks, 2 * p->block_op_cap);
    if (cudaMalloc((void**)&p->block_op, sizeof(int) * (size_t)p->block_op_cap) != cudaSuccess) {
      p->block_op_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool rotation block table");
    }
  }
  const auto h3 = clk::now();
  if (cudaMemcpyAsync(p->ops_dev, sg.ops, sizeof(PoolOp) * (size_t)nops, cudaMemcpyHostToDevice, p->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(p->chunks_dev, sg.chunks, sizeof(int) * (size_t)nops, cudaMemcpyHostToDevice, p->stream) !=
          cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool descriptor copy");
  if (!reorth.empty()) {
    std::copy(reorth.begin(), reorth.end(), sg.reorth);
    if (cudaMemcpyAsync(p->reorth_dev, sg.reorth, sizeof(PoolReorthOp) * reorth.size(), cudaMemcpyHostToDevice,
                        p->stream) != cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool monitor list copy");
  }
  if (!rank.empty()) {
    std::copy(rank.begin(), rank.end(), sg.rank);
    if (cudaMemcpyAsync(p->rank_dev, sg.rank, sizeof(PoolRankOp) * rank.size(), cudaMemcpyHostToDevice,
                        p->stream) != cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool rank list copy");
  }
  cudaEventRecord(sg.copied, p->stream);
  if (cudaMemsetAsync(p->retry_n, 0, 3 * sizeof(int) * (size_t)nticks, p->stream) != cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool retry counters");
  // Each rank bucket of the warp path has its own side stream and its own regions of the rotation
  // scratch and hand-back lists, so consecutive ticks of one bucket are ordered by its stream and
  // the buckets' ticks overlap. The main stream joins them only where it must: before work on the
  // main stream (CTA-kernel and single-stream ops, the monitor, the rank rule), whose streams may
  // have warp-path updates queued, and at the end of the submit; the side streams wait for the
  // main stream again before their next work after it.
  bool need_fork = true;
  auto fork = [&]() -> isvd_status {
    if (cudaEventRecord(p->ev_fork, p->stream) != cudaSuccess) return pool_fail(p, ISVD_ECUDA, "pool fork");
    for (int i = 0; i < 3; ++i)
      if (cudaStreamWaitEvent(p->side[i], p->ev_fork, 0) != cudaSuccess) return pool_fail(p, ISVD_ECUDA, "pool fork");
    need_fork = false;
    return ISVD_OK;
  };
  bool side_busy = false;  // side streams hold work the main stream has not waited for
  // Called before any work on the main stream: afterwards the side streams must wait for it.
  auto join = [&]() -> isvd_status {
    need_fork = true;
    if (!side_busy) return ISVD_OK;
    for (int i = 0; i < 3; ++i) {
      if (cudaEventRecord(p->ev_r[i], p->side[i]) != cudaSuccess ||
          cudaStreamWaitEvent(p->stream, p->ev_r[i], 0) != cudaSuccess)
        return pool_fail(p, ISVD_ECUDA, "pool join");
    }
    side_busy = false;
    return ISVD_OK;
  };
  for (int32_t t = 0; t < nticks; ++t) {
    // Fused ops of the tick are contiguous runs; ops outside the fused kernel's limits take the
    // single-stream kernels, in the same stream order.
    int64_t q = tick_start[t];
    auto bucket_of = [&](int64_t z) { return (int)p->s_bucket[ops[order[z]].stream]; };
    while (q < tick_start[t + 1]) {
      int64_t q2 = q;
      while (q2 < tick_start[t + 1] && fused[q2] == fused[q] && (fused[q] != 1 || bucket_of(q2) == bucket_of(q))) ++q2;
      if (fused[q] == 2) {
        // Per rank bucket (contiguous runs, widest first) on the bucket's side stream: the warp
        // launch, its rotation launch (which skips the updates handed back), the hand-back launch
        // and (with completions) the records of the run's ops.
        if (need_fork && (s = fork())) return s;
        for (int64_t b0 = q; b0 < q2;) {
          int64_t b1 = b0;
          while (b1 < q2 && bucket_of(b1) == bucket_of(b0)) ++b1;
          const int cnt = (int)(b1 - b0);
          const int bi = bucket_of(b0) == 8 ? 0 : bucket_of(b0) == 16 ? 1 : 2;
          cudaStream_t cs = p->side[bi];
          int* bop = p->block_op + run_boff[b0];
          const int* ch = p->chunks_dev + b0;
          void* scr = static_cast<char*>(p->rot_scratch) + (size_t)bi * p->rot_cap * kRotScratchStride;
          int* rlist = p->retry_list + (size_t)bi * p->retry_cap;
          int* rcount = p->retry_n + 3 * t + bi;
          const PoolOp* rops = p->ops_dev + b0;
          switch (bucket_of(b0)) {
            case 8: s = pool_launch_warp<8>(p, cs, rops, cnt, scr, rlist, rcount, ch, bop, run_blocks[b0]); break;
            case 16: s = pool_launch_warp<16>(p, cs, rops, cnt, scr, rlist, rcount, ch, bop, run_blocks[b0]); break;
            default: s = pool_launch_warp<32>(p, cs, rops, cnt, scr, rlist, rcount, ch, bop, run_blocks[b0]); break;
          }
          if (s) return s;
          switch (bucket_of(b0)) {
            case 8: s = pool_launch_rotate<8>(p, cs, rops, scr, ch, bop, run_blocks[b0], cnt); break;
            case 16: s = pool_launch_rotate<16>(p, cs, rops, scr, ch, bop, run_blocks[b0], cnt); break;
            default: s = pool_launch_rotate<32>(p, cs, rops, scr, ch, bop, run_blocks[b0], cnt); break;
          }
          if (s) return s;
          if ((s = pool_launch_retry(p, cs, rops, cnt, rlist, rcount))) return s;
          if (completions) {
            const cudaError_t e = pool_complete_launch(cnt, cs, rops, p->comp_dev + b0);
            if (e != cudaSuccess)
              return pool_fail(p, ISVD_ECUDA, std::string("pool completion launch: ") + cudaGetErrorString(e));
            p->launches++;
          }
          side_busy = true;
          b0 = b1;
        }
        p->fused_ops += q2 - q;
        p->warp_ops += q2 - q;
      } else if (fused[q]) {
        if ((s = join())) return s;
        const int cnt = (int)(q2 - q);
        switch (bucket_of(q)) {
          case 8: s = pool_launch<8>(p, p->ops_dev + q, cnt); break;
          case 16: s = pool_launch<16>(p, p->ops_dev + q, cnt); break;
          case 32: s = pool_launch<32>(p, p->ops_dev + q, cnt); break;
          default: s = pool_launch<64>(p, p->ops_dev + q, cnt); break;
        }
        if (s) return s;
        p->fused_ops += cnt;
        if (completions) {
          const cudaError_t e = pool_complete_launch(cnt, p->stream, p->ops_dev + q, p->comp_dev + q);
          if (e != cudaSuccess)
            return pool_fail(p, ISVD_ECUDA, std::string("pool completion launch: ") + cudaGetErrorString(e));
          p->launches++;
        }
      } else {
        if ((s = join())) return s;
        for (int64_t z = q; z < q2; ++z) {
          const PoolOp& d = sg.ops[z];
          isvd_ctx* h = p->streams[ops[order[z]].stream];
          // Replay the shape the op saw, run the single-stream path, restore the advanced shape.
          const int64_t m_after = h->m, n_after = h->n;
          h->m = d.m;
          h->n = d.n;
          s = d.kind == kEntry ? do_entry<float>(h, d.i, d.j, d.delta) : do_append<float>(h, d.kind, d.x);
          h->m = m_after;
          h->n = n_after;
          if (s) return s;
          p->fallback_ops++;
        }
        if (completions) {
          const cudaError_t e = pool_complete_launch((int)(q2 - q), p->stream, p->ops_dev + q, p->comp_dev + q);
          if (e != cudaSuccess)
            return pool_fail(p, ISVD_ECUDA, std::string("pool completion launch: ") + cudaGetErrorString(e));
          p->launches++;
        }
      }
      q = q2;
    }
    const int64_t nre = reorth_start[t + 1] - reorth_start[t];
    const int64_t nrk = rank_start[t + 1] - rank_start[t];
    if ((nre > 0 || nrk > 0) && (s = join())) return s;  // after this tick's updates of those streams
    if (nre > 0) {
      const cudaError_t e = pool_reorth_launch((int)nre, p->stream, p->reorth_dev + reorth_start[t], p->orth_tol);
      if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool monitor launch: ") + cudaGetErrorString(e));
      p->launches++;
      p->reorth_runs += nre;
    }
    if (nrk > 0) {
      const cudaError_t e =
          pool_rank_launch((int)nrk, p->stream, p->rank_dev + rank_start[t], p->tau_evr, p->tau_shrink);
      if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool rank launch: ") + cudaGetErrorString(e));
      p->launches++;
    }
    p->ticks++;
  }
  if ((s = join())) return s;  // the submit's work is complete when the main stream reaches here
  if (completions) {
    isvd_pool_ctx::CompBatch b;
    for (size_t i = 0; i < p->comp_free.size(); ++i)
      if (p->comp_free[i].cap >= nops) {
        b = p->comp_free[i];
        p->comp_free.erase(p->comp_free.begin() + (int64_t)i);
        break;
      }
    if (!b.host) {
      b.cap = std::max<int64_t>(nops, 4096);
      if (cudaMallocHost((void**)&b.host, sizeof(PoolCompletion) * (size_t)b.cap) != cudaSuccess)
        return pool_fail(p, ISVD_ENOMEM, "pool completion batch");
      if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(b.host);
        return pool_fail(p, ISVD_ECUDA, "pool completion event");
      }
    }
    b.count = nops;
    b.taken = 0;
    if (cudaMemcpyAsync(b.host, p->comp_dev, sizeof(PoolCompletion) * (size_t)nops, cudaMemcpyDeviceToHost,
                        p->stream) != cudaSuccess ||
        cudaEventRecord(b.ev, p->stream) != cudaSuccess) {
      p->comp_free.push_back(b);
      return pool_fail(p, ISVD_ECUDA, "pool completion copy");
    }
    p->comp_q.push_back(b);
  }
  p->seq_next += nops;
  if (p->prof) {
    const auto h4 = clk::now();
    const auto us = [](clk::time_point a, clk::time_point b) {
      return std::chrono::duration<double, std::micro>(b - a).count();
    };
    p->host_us[0] += us(h0, h1);
    p->host_us[1] += us(h1, h2);
    p->host_us[2] += us(h2, h3);
    p->host_us[3] += us(h3, h4);
    p->host_submits++;
  }
  return ISVD_OK;
}

isvd_status isvd_pool_sync(isvd_pool_t p) {
  if (!p) return ISVD_EINVAL;
  // Every slot's status word in one gather and one copy; only a stream whose word is set is read
  // in full (its sticky error).
  const int64_t n = std::min<int64_t>((int64_t)p->streams.size(), p->tab_cap);
  if (n > p->status_cap) {
    cudaStreamSynchronize(p->stream);
    if (p->status_dev) cudaFree(p->status_dev);
    if (p->status_host) cudaFreeHost(p->status_host);
    p->status_dev = nullptr;
    p->status_host = nullptr;
    p->status_cap = std::max<int64_t>(n, 2 * p->status_cap);
    if (cudaMalloc((void**)&p->status_dev, sizeof(int) * (size_t)p->status_cap) != cudaSuccess ||
        cudaMallocHost((void**)&p->status_host, sizeof(int) * (size_t)p->status_cap) != cudaSuccess) {
      p->status_cap = 0;
      return pool_fail(p, ISVD_ENOMEM, "pool status words");
    }
  }
  if (cudaMemcpyAsync(p->kcheck_host, p->kcheck, 2 * sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool self-check copy");
  if (n > 0) {
    const cudaError_t e = pool_gather_status_launch(n, p->stream, p->tab_st, p->status_dev);
    if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool status gather: ") + cudaGetErrorString(e));
    p->launches++;
    if (cudaMemcpyAsync(p->status_host, p->status_dev, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, p->stream) !=
        cudaSuccess)
      return pool_fail(p, ISVD_ECUDA, "pool status copy");
  }
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return pool_fail(p, ISVD_ECUDA, "pool sync");
  if (p->kcheck_host[0] != 0)
    return pool_fail(p, ISVD_ECUDA, "pool kernel self-check failed: code " + std::to_string(p->kcheck_host[0]) +
                                        ", at " + std::to_string(p->kcheck_host[1]));
  for (int64_t i = 0; i < (int64_t)p->streams.size(); ++i) {
    isvd_ctx* h = p->streams[i];
    if (!h || (i < n && p->status_host[i] == 0)) continue;
    DevState ds;
    isvd_status s = read_state(h, &ds);
    if (s) return s;
  }
  return ISVD_OK;
}

isvd_status isvd_pool_poll(isvd_pool_t p, isvd_completion* out, int64_t cap, int64_t* nout) {
  static_assert(sizeof(isvd_completion) == sizeof(PoolCompletion), "completion record layout");
  if (!p || !nout || cap < 0 || (cap > 0 && !out)) return ISVD_EINVAL;
  *nout = 0;
  if (!(p->flags & ISVD_POOL_COMPLETIONS)) return pool_fail(p, ISVD_EINVAL, "pool created without completions");
  while (!p->comp_q.empty() && *nout < cap) {
    isvd_pool_ctx::CompBatch& b = p->comp_q.front();
    const cudaError_t q = cudaEventQuery(b.ev);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool poll: ") + cudaGetErrorString(q));
    const int64_t take = std::min(cap - *nout, b.count - b.taken);
    std::memcpy(out + *nout, b.host + b.taken, sizeof(PoolCompletion) * (size_t)take);
    b.taken += take;
    *nout += take;
    if (b.taken == b.count) {
      p->comp_free.push_back(b);
      p->comp_q.pop_front();
    }
  }
  return ISVD_OK;
}

int64_t isvd_pool_slots(isvd_pool_t p) { return p ? (int64_t)p->streams.size() : 0; }

isvd_status isvd_pool_gather_sigma(isvd_pool_t p, int32_t ld, double* out, int to_device) {
  if (!p || !out || ld < 1) return ISVD_EINVAL;
  const int64_t n = (int64_t)p->streams.size();
  if (n == 0) return ISVD_OK;
  double* dst = out;
  if (!to_device) {
    if (n * ld > p->gather_cap) {
      cudaStreamSynchronize(p->stream);
      if (p->gather_dev) cudaFree(p->gather_dev);
      p->gather_dev = nullptr;
      p->gather_cap = std::max<int64_t>(n * ld, 2 * p->gather_cap);
      if (cudaMalloc((void**)&p->gather_dev, 8 * (size_t)p->gather_cap) != cudaSuccess) {
        p->gather_cap = 0;
        return pool_fail(p, ISVD_ENOMEM, "pool sigma gather buffer");
      }
    }
    dst = p->gather_dev;
  }
  cudaError_t e = pool_gather_sigma_launch(n, p->stream, p->tab_sig, p->tab_st, ld, dst);
  if (e != cudaSuccess) return pool_fail(p, ISVD_ECUDA, std::string("pool sigma gather: ") + cudaGetErrorString(e));
  p->launches++;
  if (!to_device &&
      cudaMemcpyAsync(out, p->gather_dev, 8 * (size_t)(n * ld), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
    return pool_fail(p, ISVD_ECUDA, "pool sigma gather copy");
  return ISVD_OK;
}

const char* isvd_pool_last_error(isvd_pool_t p) { return p ? p->err.c_str() : "null pool"; }

}  // extern "C"
