/*
 * isvd.h — C ABI of libisvd, a GB300 (sm_103a) engine for the Brand-style incremental SVD
 * of arXiv 2605.24514 ("Incremental SVD for Large-Scale Dynamic Matrices").
 *
 * The engine maintains A_t ~= U_t diag(sigma_t) V_t^T for a dense matrix A_t that changes by
 * row appends, column appends and single-entry increments (Section 2.1), refreshes the
 * factorisation from the stored A_t on demand or by policy (Sections 2.4 and 3), and reports
 * the error-ratio, principal-angle and EVR metrics of Section 2.5.
 *
 * Conventions shared by every call
 *  - All matrices are ROW-MAJOR. A caller buffer for U holds m*r elements with row stride r,
 *    V holds n*r elements with row stride r; sigma is r doubles in descending order.
 *  - The element type of U, V, A and of appended rows/columns is the handle's storage type:
 *    double for ISVD_FP64, float for ISVD_FP32. sigma, rho, N_t and all metrics are double.
 *  - "on_device" / "to_device" flags say whether a pointer is CUDA device memory (on the
 *    handle's device) or host memory. Device pointers must stay valid until the call's work has
 *    finished on the handle's stream (isvd_sync); host pointers are only read during the call.
 *  - Ownership: every input is copied into the handle; the caller keeps its buffers. Outputs
 *    go into caller-allocated buffers. The handle owns all of its device memory.
 *  - Errors: every call returns an isvd_status and never aborts. Argument errors (bad shape,
 *    out-of-range index, NaN/Inf in a host input) are detected before any work is queued and
 *    leave the state unchanged. Device-side failures (core SVD not converged, non-finite data
 *    seen in a device input) are sticky: they are reported by the next call that synchronises
 *    (isvd_sync, isvd_metrics, isvd_get_*), and every later call returns the same status.
 *    isvd_last_error gives a one-line message.
 *  - Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef ISVD_H_
#define ISVD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isvd_ctx* isvd_t;

typedef enum {
  ISVD_FP64 = 0,  /* U, V, A and the core SVD in FP64 */
  ISVD_FP32 = 1   /* U, V, A in FP32; sigma, rho, N_t and the core's singular values in FP64 */
} isvd_precision;

typedef enum {
  ISVD_OK = 0,
  ISVD_EINVAL = 1,      /* bad argument (NULL handle, k < 1, unknown flag, ...) */
  ISVD_ESHAPE = 2,      /* vector length does not match the current shape */
  ISVD_EBOUNDS = 3,     /* (i, j) outside the current matrix */
  ISVD_ENOMEM = 4,      /* device allocation failed */
  ISVD_EBUDGET = 5,     /* pool admission refused: memory budget or slot count exceeded */
  ISVD_ENOTCONV = 6,    /* a core Jacobi SVD did not converge within its sweep limit */
  ISVD_ETIMEOUT = 7,    /* a bounded device-side wait gave up */
  ISVD_ECUDA = 8,       /* a CUDA runtime call failed */
  ISVD_ENONFINITE = 9   /* NaN or Inf in an input */
} isvd_status;

typedef struct {
  int32_t prec;        /* isvd_precision */
  int32_t k_max;       /* column capacity of U and V (>= k); 0 means k */
  double tol_rel;      /* rank test of Section 2.2: a new direction is kept iff
                          rho > tol_rel * ||x||; <= 0 selects 1e-10 (FP64) or 3e-6 (FP32) */
  int64_t row_cap;     /* initial row capacity of A and U (0: 2*m0) */
  int64_t col_cap;     /* initial column capacity of A and row capacity of V (0: 2*n0) */
  void* cuda_stream;   /* cudaStream_t all work is queued on; NULL = legacy default stream */
  uint64_t seed;       /* seed of the randomized refresh's test matrix */
  double orth_tol;     /* re-orthogonalisation trigger on max|U^T U - I|, max|V^T V - I|;
                          <= 0 selects 1e-5 (FP32) or 1e-12 (FP64) */
  int64_t orth_every;  /* monitor cadence in updates; 0 selects 256 (FP32) / never (FP64) */
  int32_t rsvd_oversample;   /* randomized refresh (min(m, n) > 128): extra sketch columns p,
                                sketch size l = min(k + p, 128); <= 0 selects 16 */
  int32_t rsvd_power_iters;  /* randomized refresh: power iterations q; < 0 selects 2 */
} isvd_config;

/* Policy kinds (bit set), Section 3. */
#define ISVD_POLICY_NONE 0
#define ISVD_POLICY_PERIODIC 1       /* refresh iff t mod T_refresh == 0, Eq. (periodic-refresh-rule) */
#define ISVD_POLICY_ERROR 2          /* refresh iff frob_ratio > gamma (and t - t_last >= T_min),
                                        Eq. (error-refresh-rule) */
#define ISVD_POLICY_ANGLE 4          /* refresh iff angle_to_opt > theta_max (Section 3.3) */
#define ISVD_POLICY_ADAPTIVE_RANK 8  /* k <- min(k + 1, k_max) while EVR < tau_evr at a check,
                                        Eq. (evr-rank-rule) read as a growth rule */
#define ISVD_POLICY_NOVELTY_RANK 16  /* after a row or column append with rho > eta ||x||,
                                        k <- min(k + 1, k_max) for the next update, Eq.
                                        (novelty-rank-rule); decided on the device */
#define ISVD_POLICY_RANK_SHRINK 32   /* at a check: if the leading k - 1 components explain at
                                        least tau_shrink of N_t, k <- max(k - 1, k_min) and the
                                        smallest component is dropped (the shrink side of Eq.
                                        (evr-rank-rule), Section 6); tau_shrink above tau_evr
                                        keeps the two rules from oscillating */

typedef struct {
  int32_t kind;                    /* bit set of ISVD_POLICY_* */
  int32_t k_min, k_max;            /* adaptive-rank bounds (k_max <= config k_max) */
  int32_t store_initial_subspace;  /* refresh also sets U_ref <- U_t (Section 2.4) */
  int64_t T_refresh;               /* periodic period */
  int64_t T_min;                   /* minimum spacing of error/angle refreshes */
  int64_t check_every;             /* cadence of the error/angle/EVR checks (0: never) */
  double gamma;                    /* error-ratio threshold */
  double theta_max_rad;            /* angle threshold in radians */
  double tau_evr;                  /* EVR target */
  double eta;                      /* novelty threshold in (0, 1) (ISVD_POLICY_NOVELTY_RANK) */
  double tau_shrink;               /* EVR of k - 1 components that shrinks k (ISVD_POLICY_RANK_SHRINK) */
} isvd_policy;

/* Metrics of Section 2.5 (names follow the paper). */
typedef struct {
  int64_t t, m, n;       /* updates applied, current shape */
  int32_t r, k;          /* maintained rank, working rank k_t */
  double frob_error;     /* E_inc = ||A_t - U S V^T||_F */
  double frob_opt;       /* E_opt = error of the best rank-r approximation */
  double frob_gap;       /* E_inc - E_opt */
  double frob_ratio;     /* E_inc / E_opt, NaN when E_opt is numerically zero */
  double angle;          /* theta_max(U_ref, U_t), Eq. (angle-metrics-ref) */
  double angle_to_opt;   /* theta_max(U_opt, U_t), Eq. (angle-metrics-opt) */
  double evr;            /* sum sigma^2 / N_t, Eq. (evr) */
  double rho_last;       /* residual norm of the last append, Eq. (row-residual) */
  double novelty_last;   /* rho / ||x|| of the last append (Section 3.3) */
  double orth_err_u;     /* max |U^T U - I| (measured by the last monitor run) */
  double orth_err_v;     /* max |V^T V - I| */
  double N;              /* N_t = ||A_t||_F^2 maintained incrementally (Section 2.4) */
  int64_t refreshes;     /* refreshes performed */
  int64_t reorths;       /* re-orthogonalisations performed */
  int64_t t_last;        /* time of the last refresh */
  int32_t core_sweeps;   /* last core SVD: Jacobi sweeps (-1: not converged), or 100 + i for the secular
                            core (i = 0, 1: Gram-verified after i refinements; 2: corrected weights) */
  int32_t reserved0;
  double angle_succ_u;   /* largest principal angle between span(U_{t-1}) and span(U_t) (Section 3.3,
                            subspace change per update; an appended row extends U_{t-1} by a zero
                            row); 0 for an entry update, NaN before the first update */
  double angle_succ_v;   /* the same for V */
} isvd_metrics_t;

/* Flags of isvd_metrics. */
#define ISVD_METRICS_CHEAP 0  /* t, shape, EVR, N, rho/novelty: no pass over A */
#define ISVD_METRICS_FULL 1   /* also E_inc, E_opt, ratio, gap and both angles (one pass to
                                 form E_inc and one truncated SVD of A_t) */

/* One update event for isvd_apply_events. kind: 0 row append, 1 column append, 2 entry. */
typedef struct {
  int32_t kind;
  int32_t reserved;
  int64_t i, j;    /* entry position (kind 2) */
  double delta;    /* entry increment (kind 2) */
  int64_t off;     /* payload offset in elements (kinds 0, 1) */
  int64_t len;     /* payload length: n for a row, m for a column */
} isvd_event;

/* --- single-stream engine ------------------------------------------------------------ */

/* Algorithm 1 (initialisation) and Section 2.4: (U, S, V) <- TruncatedSVD(A0, k) at rank
 * r0 = min(k, m0, n0); A <- A0; N_0 = ||A0||_F^2; U_ref <- U_0; t = 0.
 * A0 is m0 x n0 row-major with row stride lda (>= n0), host or device memory.
 * TruncatedSVD is exact (Gram matrix of the short side, Jacobi eigensolver) when
 * min(m, n) <= 128 and randomized (Halko-Martinsson-Tropp sketch with power iterations)
 * otherwise; refreshes and the metrics' optimal factorisation use the same routine. */
isvd_status isvd_create(const isvd_config* cfg, const void* A0, int64_t m0, int64_t n0,
                        int64_t lda, int k, int a0_on_device, isvd_t* out);
void isvd_destroy(isvd_t h);

/* As isvd_create, but the initial factors are supplied by the caller instead of computed:
 * U0 (m0 x r0), sigma0 (r0, descending) and V0 (n0 x r0), row-major with row stride r0, in the
 * same memory space as A0; r0 must equal min(k, m0, n0). U0 and V0 should have orthonormal
 * columns. Used to resume a stream from stored factors (and to start two engines identically). */
isvd_status isvd_create_from_factors(const isvd_config* cfg, const void* A0, int64_t m0, int64_t n0,
                                     int64_t lda, const void* U0, const double* sigma0,
                                     const void* V0, int r0, int k, int on_device, isvd_t* out);

/* Row append, Section 2.2 / Algorithm A1: A <- [A; x^T], then the projection
 * p = x^T V, residual rho = ||x^T - p V^T||, the (r+1)x(r+1) core SVD and the rotations
 * U' = blkdiag(U, 1) U_K, V' = [V z_hat] V_K, truncated to k. x has n elements. */
isvd_status isvd_append_row(isvd_t h, const void* x, int64_t n, int on_device);

/* Column append via transpose, Section 2.2 / Algorithm A2: A <- [A, y]; y has m elements. */
isvd_status isvd_append_col(isvd_t h, const void* y, int64_t m, int on_device);

/* Rank-1 entry update, Section 2.3 / Algorithm A3: A_ij <- A_ij + delta and
 * U'S'V'^T = P_U (A_hat + delta e_i e_j^T) P_V at fixed rank, Eq. (rank1-projection). */
isvd_status isvd_update_entry(isvd_t h, int64_t i, int64_t j, double delta);

/* A_ij += delta in the rank-increasing form (Section 2.3's modification A + delta e_i e_j^T in
 * Brand's general form, rather than its projection onto the current subspaces, Eq.
 * rank1-projection): with e_i = U p + alpha P and e_j = V q + beta Q (p = U[i, :], q = V[j, :],
 * alpha^2 = 1 - ||p||^2, beta^2 = 1 - ||q||^2; a residual norm <= tol_rel is dropped), the
 * (r+1) x (r+1) core diag(sigma, 0) + delta [p; alpha][q; beta]^T is factorised and U' = [U P] U_K,
 * V' = [V Q] V_K, truncated at k: the rank can grow by one. Same bookkeeping (A_ij, N_t, t) and
 * policy step as isvd_update_entry; errors as there. */
isvd_status isvd_update_entry_exact(isvd_t h, int64_t i, int64_t j, double delta);

/* Deferred rotations for the rank-1 entry updates of Section 2.3 (the fast form of the Brand
 * update that the paper builds on). enable = 1 keeps U = U0 R_U and V = V0 R_V with small
 * R_U, R_V (k x k, storage precision, owned by the handle; allocated on the first enable,
 * ENOMEM on failure): each isvd_update_entry then gathers U0[i, :] R_U and V0[j, :] R_V for its
 * core and multiplies R_U, R_V by the core's factors, O(k^3) work on k x k data, instead of
 * rotating the m x k and n x k factors. The next call that needs U or V (an append, the
 * rank-increasing entry update, refresh, metrics, re-orthogonalisation, risk, get_factors)
 * first folds U <- U0 R_U, V <- V0 R_V in one pass; enable = 0 folds and turns the mode off.
 * Results equal those of the plain form up to rounding (the product order differs). Single
 * streams only: EINVAL on a pool stream's handle or for enable outside {0, 1}. */
isvd_status isvd_set_deferred_rotations(isvd_t h, int enable);
/* 1 iff entry updates are held in R_U, R_V and not yet folded into U, V. */
int isvd_deferred_pending(isvd_t h);

/* Applies nev events in order (same semantics as the three calls above, policy included).
 * payload holds the row/column vectors, host or device memory. */
isvd_status isvd_apply_events(isvd_t h, const isvd_event* ev, int64_t nev, const void* payload,
                              int64_t payload_len, int payload_on_device);

/* Sets the policy evaluated after every update (Section 3). NULL disables it. */
isvd_status isvd_set_policy(isvd_t h, const isvd_policy* pol);

/* Refresh, Section 2.4: (U, S, V) <- TruncatedSVD(A_t, k_t); U_ref <- U_t if
 * store_initial_subspace. */
isvd_status isvd_refresh(isvd_t h, int store_initial_subspace);

/* Metrics of Section 2.5 on the current state (synchronises). */
isvd_status isvd_metrics(isvd_t h, int flags, isvd_metrics_t* out);

/* Metrics computed at the most recent policy check step (before any refresh that the check
 * triggered; t_last == t tells that one fired). Zeroed until the first check. */
isvd_status isvd_last_check_metrics(isvd_t h, isvd_metrics_t* out);

/* Copies U (m x r), sigma (r) and V (n x r) into caller buffers (any may be NULL). */
isvd_status isvd_get_factors(isvd_t h, void* U, double* sigma, void* V, int to_device);

/* Copies the stored dense A_t (m x n, row stride n) into a caller buffer. */
isvd_status isvd_get_matrix(isvd_t h, void* A, int to_device);

/* Current shape and ranks (synchronises, so r is the device's value). */
isvd_status isvd_get_shape(isvd_t h, int64_t* m, int64_t* n, int32_t* r, int32_t* k);

/* Runs the loss-of-orthogonality monitor now and, if max|Q^T Q - I| exceeds the configured
 * tolerance for U or V, re-orthonormalises both by two Cholesky-QR passes (sigma unchanged). */
isvd_status isvd_reorthogonalize(isvd_t h, int force, double* err_u, double* err_v);

/* Waits for all queued work; reports sticky device-side errors. */
isvd_status isvd_sync(isvd_t h);

/* Number of kernels this handle has launched so far. */
int64_t isvd_kernel_launches(isvd_t h);

/* Kernel classes for isvd_profile_read. */
#define ISVD_KCLASS_PROJ 0     /* projection and residual passes (Eq. row-residual) */
#define ISVD_KCLASS_CORE 1     /* core SVD (assembly, Jacobi, sort, truncation) */
#define ISVD_KCLASS_ROTATE 2   /* rotations of U and V */
#define ISVD_KCLASS_CHECK 3    /* policy checks: metrics incl. the truncated SVD of A */
#define ISVD_KCLASS_REFRESH 4  /* refreshes */
#define ISVD_KCLASS_REORTH 5   /* orthogonality monitor and re-orthogonalisation */
#define ISVD_NUM_KCLASS 6

/* Enables (1) or disables (0) device-time profiling and clears its counters. While enabled,
 * CUDA events are recorded around every launch of the classes above and at the end of every
 * update, on the handle's stream. */
isvd_status isvd_profile(isvd_t h, int enable);

/* Totals since isvd_profile: device milliseconds, algorithmic bytes (the bytes the method must
 * move, e.g. U and V read and written once for a rotation) and launches of one class. */
isvd_status isvd_profile_read(isvd_t h, int cls, double* total_ms, double* bytes, int64_t* launches);

/* Device time of each update since isvd_profile (microseconds between consecutive update ends
 * on the stream), up to cap values; *count receives the total number. */
isvd_status isvd_latencies(isvd_t h, double* us, int64_t cap, int64_t* count);

const char* isvd_last_error(isvd_t h);
const char* isvd_status_string(isvd_status s);

/* --- batched pool of independent streams ---------------------------------------------------
 * Many streams (each the single-stream engine above, FP32 bulk) share one CUDA stream. A submit
 * takes an ordered list of ops; ops of the same stream are applied in list order, ops of different
 * streams are grouped into "ticks" (at most one op per stream). Per tick, the appends of rank
 * buckets 8, 16 and 32 run as one launch per bucket of a warp-per-update kernel (projection with
 * CGS2, core SVD, dense-A and N_t bookkeeping) followed by one launch of a rotation kernel per
 * bucket (FP32 pipes; tensor cores for buckets 16 and 32 with ISVD_POOL_TC_ROTATIONS); each bucket
 * has its own internal CUDA stream, so ticks of different buckets overlap, and the pool's CUDA
 * stream waits for them before its own work and at the end of every submit. Entry updates,
 * bucket 64 and the updates the warp kernel hands back take a CTA-per-update kernel.
 * The launch count per tick does not depend on the number of streams. Streams are admitted under an
 * HBM budget; a staggered loss-of-orthogonality monitor re-orthonormalises streams as needed. The
 * pool path runs no refresh policy; isvd_pool_stream gives the stream's handle for refresh, metrics
 * and reads. */
typedef struct isvd_pool_ctx* isvd_pool_t;

typedef struct {
  int32_t k_max;             /* largest admitted rank, 1..128 (streams above 64 take the
                                single-stream kernels, in order) */
  int32_t flags;             /* bit set of ISVD_POOL_* below (0: defaults) */
  int64_t max_streams;       /* slot limit (0: unlimited) */
  int64_t hbm_budget_bytes;  /* admission budget for the streams' device memory (0: unlimited) */
  void* cuda_stream;         /* CUDA stream of all pool work (NULL: legacy default stream) */
  double tol_rel;            /* rank test (<= 0: 3e-6) */
  int64_t orth_every;        /* loss-of-orthogonality monitor: every stream is checked after this many
                                of its updates (0: 256; < 0: never); streams are staggered so that
                                about 1/orth_every of them are checked per tick */
  double orth_tol;           /* re-orthogonalise U or V when max|Q^T Q - I| exceeds it (<= 0: 1e-5) */
  int64_t rank_every;        /* adaptive rank (Section 3, Eq. evr-rank-rule read as a growth rule):
                                after every rank_every-th update of a stream (t mod rank_every == 0),
                                k <- min(k + 1, capacity) if sum sigma^2 / N_t < tau_evr; the new
                                component arrives with the stream's next append that keeps its
                                residual. 0: off. The capacity is the stream's rank bucket (8, 16,
                                32, 64 or 128, the smallest holding the admitted k) capped by k_max. */
  double tau_evr;            /* EVR target of the adaptive rank rule */
  double eta_novelty;        /* novelty rank rule for every stream (Eq. novelty-rank-rule): after an
                                append with rho > eta_novelty ||x||, k <- min(k + 1, capacity) for
                                the stream's next update; 0: off, else in (0, 1) */
  double tau_shrink;         /* with rank_every: at the same checks, k <- k - 1 (at least 1) and the
                                smallest component dropped when the leading k - 1 components
                                explain at least tau_shrink of N_t; 0: off, else in (tau_evr, 1] */
} isvd_pool_config;

/* isvd_pool_config.flags */
#define ISVD_POOL_TC_ROTATIONS 1    /* rotate rank buckets 16 and 32 on the tensor cores (exact
                                       BF16 digit products; same accuracy class, measured slower at
                                       these ranks). Default: FP32 pipes in every bucket */
#define ISVD_POOL_COMPLETIONS 2     /* every op of a submit leaves a completion record for
                                       isvd_pool_poll */
#define ISVD_POOL_DEVICE_CHECKS 4   /* a host payload is not scanned on the host: non-finite values
                                       are caught by the kernels, as for a device payload (a sticky
                                       ISVD_ENONFINITE of that stream at the next isvd_pool_sync,
                                       and status ISVD_ENONFINITE in the op's completion record);
                                       submit then costs no pass over the payload on the host */

/* Completion record of one pool op (ISVD_POOL_COMPLETIONS). */
typedef struct {
  int64_t seq;        /* pool-wide sequence number: the ops of all submits are numbered from 0 in the
                         order they were given (submit by submit, op by op) */
  int32_t stream;     /* stream id */
  int32_t kind;       /* 0 row append, 1 column append, 2 entry update */
  int32_t status;     /* ISVD_OK, or the stream's sticky device status after the op */
  int32_t r;          /* maintained rank after the op */
  double rho;         /* residual norm of an append, Eq. (row-residual); 0 for an entry update */
  double sigma_max;   /* largest singular value after the op */
  uint64_t done_ns;   /* device clock (%globaltimer, ns) when the record was written, right after the
                         op's tick */
} isvd_completion;

/* One op of a pool submit: kind 0 row append, 1 column append, 2 entry update (as isvd_event). */
typedef struct {
  int32_t stream;
  int32_t kind;
  int64_t i, j;
  double delta;
  int64_t off, len;  /* FP32 payload slice for appends */
} isvd_op;

isvd_status isvd_pool_create(const isvd_pool_config* cfg, isvd_pool_t* out);
void isvd_pool_destroy(isvd_pool_t p);

/* Admits a stream started from A0 (FP32, m0 x n0, row stride lda) at rank k <= k_max, with
 * initial capacities row_cap/col_cap, optionally from given factors (U0 m0 x r0, sigma0 r0, V0
 * n0 x r0, row-major, with r0 = min(k, m0, n0) as in isvd_create_from_factors; the library reads
 * exactly that many values) or NULL to compute TruncatedSVD(A0, k). Returns ISVD_EBUDGET (nothing
 * admitted) when the stream's device footprint would exceed the budget or the slots are full. */
isvd_status isvd_pool_admit(isvd_pool_t p, const void* A0, int64_t m0, int64_t n0, int64_t lda, int k,
                            int64_t row_cap, int64_t col_cap, const void* U0, const double* sigma0,
                            const void* V0, int on_device, int32_t* stream_id);

/* Releases a stream and its memory (synchronises). */
isvd_status isvd_pool_release(isvd_pool_t p, int32_t stream_id);

/* Queues ops (see above). All ops are validated (stream, kind, shape, bounds, finite deltas)
 * before any work is queued; on error nothing is queued. payload is FP32, host or device memory
 * (payload_on_device). A host payload is also scanned for NaN/Inf first (ISVD_ENONFINITE, nothing
 * queued; the scan reads the whole payload once), unless the pool has ISVD_POOL_DEVICE_CHECKS.
 * A host payload is copied on the pool's CUDA stream: from pageable memory before the call
 * returns, from page-locked memory when the stream reaches the copy (keep such a buffer unchanged
 * until then, e.g. until isvd_pool_sync or the ops' completion records). A device payload is not
 * read by the host: a non-finite value there is seen by the kernels and reported as a sticky
 * ISVD_ENONFINITE of that stream by the next isvd_pool_sync, as for device inputs of a single
 * stream. */
isvd_status isvd_pool_submit(isvd_pool_t p, const isvd_op* ops, int64_t nops, const void* payload,
                             int64_t payload_len, int payload_on_device);

/* Waits for the pool's work; reports sticky device errors of any stream. */
isvd_status isvd_pool_sync(isvd_pool_t p);

/* Completion records (pool created with ISVD_POOL_COMPLETIONS): copies up to cap records of ops
 * whose work has finished on the device and that no earlier poll returned into out, and their
 * number into *nout. Never waits. Records come submit by submit; within a submit, tick by tick
 * (a stream's ops in its order), and within a tick in the pool's launch order (seq identifies the
 * op). Records are kept (in pinned host memory) until polled. ISVD_EINVAL if the pool was created
 * without ISVD_POOL_COMPLETIONS; ISVD_ECUDA if a CUDA call failed. */
isvd_status isvd_pool_poll(isvd_pool_t p, isvd_completion* out, int64_t cap, int64_t* nout);

/* Number of stream slots (one past the largest stream id ever admitted). */
int64_t isvd_pool_slots(isvd_pool_t p);

/* Singular values of every slot in one array: out[s * ld + c] = sigma_c of stream s for
 * c < min(r_s, ld), zero elsewhere (released slots are all zero); out holds isvd_pool_slots(p) * ld
 * doubles, device memory (to_device = 1) or host memory. The gather is queued on the pool's CUDA
 * stream after all submitted work: a device or pinned host buffer is filled asynchronously (ready
 * when the stream reaches it, e.g. after isvd_pool_sync); a pageable host buffer is filled before
 * the call returns. ld >= 1. */
isvd_status isvd_pool_gather_sigma(isvd_pool_t p, int32_t ld, double* out, int to_device);

/* The single-stream handle of a pool stream (owned by the pool; do not destroy), or NULL. */
isvd_t isvd_pool_stream(isvd_pool_t p, int32_t stream_id);

int64_t isvd_pool_bytes_used(isvd_pool_t p);
int64_t isvd_pool_kernel_launches(isvd_pool_t p);
const char* isvd_pool_last_error(isvd_pool_t p);

/* Launch classes of the pool's kernels, for isvd_pool_profile_read: the warp-per-update
 * projection + core kernels and the row-parallel rotation kernels of rank buckets 8/16/32, the
 * hand-back CTA kernel, and the CTA kernel (entry updates, rank bucket 64). */
#define ISVD_POOL_KCLASS_WARP8 0
#define ISVD_POOL_KCLASS_WARP16 1
#define ISVD_POOL_KCLASS_WARP32 2
#define ISVD_POOL_KCLASS_ROT8 3
#define ISVD_POOL_KCLASS_ROT16 4
#define ISVD_POOL_KCLASS_ROT32 5
#define ISVD_POOL_KCLASS_RETRY 6
#define ISVD_POOL_KCLASS_CTA 7
#define ISVD_POOL_NUM_KCLASS 8

/* enable != 0 clears and starts per-class timing of the pool's launches (CUDA events recorded on
 * each launch's own stream); 0 stops it. Host cost: two event records per launch. */
isvd_status isvd_pool_profile(isvd_pool_t p, int enable);
/* Synchronizes the pool and writes, per launch class, the summed device time in ms (ms_out) and
 * the number of launches (launches_out), each an array of n <= ISVD_POOL_NUM_KCLASS entries. */
isvd_status isvd_pool_profile_read(isvd_pool_t p, double* ms_out, int64_t* launches_out, int n);
/* Host wall time (microseconds) that isvd_pool_submit spent since profiling was enabled, by phase:
 * [0] validating the ops, [1] ordering them into ticks and rank buckets, [2] staging descriptors
 * (including any wait for the copy of two submits ago), [3] enqueueing copies and launches;
 * n <= 4 entries. *submits (may be NULL) receives the number of submits counted. */
isvd_status isvd_pool_host_profile(isvd_pool_t p, double* us_out, int n, int64_t* submits);

/* --- finance layer (Section 5) --------------------------------------------------------------
 * Causal centering of return rows before they are appended (Section 5.1), and the low-rank
 * covariance and portfolio risk implied by a handle's factors (Section 5.3). */

#define ISVD_CENTER_CAUSAL 1  /* expanding mean, Option A: mu_t = mu_{t-1} + (r_t - mu_{t-1}) / t */
#define ISVD_CENTER_EW 2      /* exponentially weighted mean, Option B: mu_t = (1 - a) mu_{t-1} + a r_t */

typedef struct isvd_center_ctx* isvd_center_t;

/* Centering state for n assets (mu = 0, no rows yet), arithmetic in FP64, rows of the storage type of
 * prec (double for ISVD_FP64, float for ISVD_FP32), work queued on cuda_stream. alpha is Option B's
 * forgetting factor in (0, 1) (ignored for ISVD_CENTER_CAUSAL). ISVD_EINVAL for a bad mode, alpha, n or
 * prec; ISVD_ENOMEM if the state cannot be allocated. */
isvd_status isvd_center_create(int32_t mode, double alpha, int64_t n, int32_t prec, void* cuda_stream,
                               isvd_center_t* out);
void isvd_center_destroy(isvd_center_t c);

/* Centers `rows` raw return rows in time order (row stride ld_raw >= n) into out (row stride
 * ld_out >= n): out_t = r_t - mu_t with mu_t updated by row t first, so each row is centered with
 * the returns up to and including its own. Both buffers are device memory (on_device = 1) or host
 * memory (copied through the state's staging buffer; the call returns when out is written). The
 * state advances by `rows`. */
isvd_status isvd_center_rows(isvd_center_t c, const void* raw, int64_t rows, int64_t ld_raw, void* out,
                             int64_t ld_out, int on_device);

/* New assets (columns appended to the returns matrix): their current means (count host doubles). */
isvd_status isvd_center_add_assets(isvd_center_t c, const double* mu_new, int64_t count);

/* Copies the n current means into host memory (mu may be NULL) and the number of rows centered. */
isvd_status isvd_center_state(isvd_center_t c, double* mu, int64_t* count);

/* Low-rank covariance and portfolio risk of a handle, Section 5.3: with t = m rows of the centered
 * returns matrix, S_inc = V diag(sigma^2) V^T / (t - 1) (Eq. low-rank-covariances) and the portfolio
 * volatility vol = sqrt(w^T S_inc w) (Eq. portfolio-vol) for weights w (n values of the storage type,
 * host or device memory; NULL selects the equal-weight portfolio 1/n). With ISVD_RISK_FULL also the
 * same quantities for the optimal rank-r factorisation of A_t (the truncated SVD of the metrics),
 * the risk error |vol - vol_opt| / vol_opt (Eq. risk-error) and the covariance error
 * ||S_inc - S_opt||_F / ||S_opt||_F (Eq. cov-error), computed from r x r Gram matrices of the factors
 * without forming an n x n matrix. Synchronises. */
#define ISVD_RISK_CHEAP 0
#define ISVD_RISK_FULL 1
typedef struct {
  int64_t t;          /* rows of the centered returns matrix */
  int32_t r;          /* rank of the factors */
  int32_t reserved;
  double vol;         /* sqrt(w^T S_inc w) */
  double vol_opt;     /* sqrt(w^T S_opt w) (ISVD_RISK_FULL), NaN otherwise */
  double risk_error;  /* |vol - vol_opt| / vol_opt (ISVD_RISK_FULL), NaN otherwise */
  double cov_error;   /* ||S_inc - S_opt||_F / ||S_opt||_F (ISVD_RISK_FULL), NaN otherwise */
  double cov_norm;    /* ||S_inc||_F */
} isvd_risk_t;
isvd_status isvd_risk(isvd_t h, const void* w, int w_on_device, int flags, isvd_risk_t* out);

/* --- allocation-free orthogonality measurement ----------------------------------------------
 * The paper has no counterpart: this is a library service for callers that cannot allocate
 * device memory, e.g. code running under a memory pool that forbids new allocations, code that
 * must not trigger the device synchronisation cudaMalloc/cudaFree can cause, or a process whose
 * device allocator belongs to another framework.
 *
 * Computes max|Q^T Q - I| (the quantity isvd_reorthogonalize reports as err_u / err_v) for a
 * device matrix Q (rows x r, row-major, row stride ld >= r, element type double for ISVD_FP64 or
 * float for ISVD_FP32) and writes it to *err_out, a caller-provided DEVICE pointer, on
 * cuda_stream (NULL = legacy default stream); the value is ready when that stream reaches it.
 * Allocates nothing: the r x r FP64 scratch lives in a fixed 128 KiB device array inside the
 * library, which every GPU that loads the library holds until the process exits.
 *  - r may be at most ISVD_NOALLOC_MAX_R (128); larger r returns ISVD_ESHAPE and does nothing.
 *  - rows < 0, r < 1, ld < r, NULL pointers or an unknown precision return ISVD_EINVAL.
 *  - The first call on each device looks up the scratch array's device address (once per
 *    device, with that device current); make that first call before any stream capture.
 *  - Every call shares the one scratch array (each call clears what it needs first), so calls
 *    whose work overlaps on the GPU race with each other; serialise them (same stream, or
 *    events). Returns ISVD_ECUDA if a CUDA call fails. */
#define ISVD_NOALLOC_MAX_R 128
isvd_status isvd_orth_error_noalloc(const void* Q, int64_t rows, int32_t r, int64_t ld, int32_t prec,
                                    double* err_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ISVD_H_ */
