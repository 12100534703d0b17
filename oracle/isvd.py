"""CPU oracle for the Brand-style incremental SVD engine (TEST INFRASTRUCTURE ONLY).

Plain, slow, FP64 NumPy/LAPACK restatement of the method of arXiv 2605.24514
("Incremental SVD for Large-Scale Dynamic Matrices"), written from the paper and
shared with nothing on the CUDA path. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it; the product never does.

Every routine follows the paper's steps in its own order and notation:

* engine control flow ........................ Algorithm 1 (Section 2.1)
* row append ................................. Section 2.2, Eq. (row-residual), Algorithm A1
* column append via transpose ................ Section 2.2 ("Column Append via Transpose"), Algorithm A2
* rank-1 entry update (projection rule) ...... Section 2.3, Eq. (rank1-projection), Algorithm A3
* rank-1 entry update, rank-increasing form ... Section 2.3's modification in Brand's general form
* refresh / truncated SVD .................... Section 2.4 ("Refresh Operation")
* principal angles ........................... Section 2.4, Eqs. (theta-max), (angle-metrics-ref/opt)
* Frobenius errors, ratio, EVR, N_t .......... Section 2.5, Eqs. (frob-errors), (frob-ratio), (evr)
* refresh and rank policies .................. Section 3, Eqs. (periodic-refresh-rule),
                                               (error-refresh-rule), angle rule, (evr-rank-rule)
                                               with its shrink side, (novelty-rank-rule)
* successive-subspace angles ................. Section 3.3 ("subspace-change per update")

Readings taken where the paper is silent or ambiguous are stated inline (marked
"Reading:"); the same list appears in the design notes of the repository.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Event kinds (Section 2.1 lists exactly these three update types).
ROW, COL, ENTRY = 0, 1, 2

# Policy flags (Section 3: periodic, error-based, angle-based, adaptive rank).
POLICY_NONE = 0
POLICY_PERIODIC = 1
POLICY_ERROR = 2
POLICY_ANGLE = 4
POLICY_ADAPTIVE_RANK = 8
POLICY_NOVELTY_RANK = 16
POLICY_RANK_SHRINK = 32


# ---------------------------------------------------------------------------
# Dense linear-algebra steps (library primitives serve as single steps)
# ---------------------------------------------------------------------------

def truncated_svd(A: np.ndarray, k: int):
    """TruncatedSVD(A, k) of Algorithm 1 / the refresh of Section 2.4: full SVD of A,
    keep the leading ``min(k, m, n)`` triplets. Returns (U, sigma, V) with V = Z[:r].T."""
    W, s, Zt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    r = min(k, s.size)
    return W[:, :r].copy(), s[:r].copy(), Zt[:r].T.copy()


def row_append_update(U, s, V, x, tol_rel):
    """Row append of Section 2.2 (Algorithm A1), before truncation.

    The appended matrix factors exactly through a small core: split x into its part in span(V),
    with coordinates p = V^T x, and the residual z = x - V p of norm rho (Eq. row-residual).
    Then [U S V^T; x^T] = blkdiag(U, 1) K [V, z/rho]^T with K the (r+1) x (r+1) lower arrow
    matrix holding S on its diagonal, p^T as its last row and rho in the corner; an SVD of K,
    K = W S' Z^T, gives the new factors blkdiag(U, 1) W and [V, z/rho] Z.

    Reading (rank test): the residual is kept as a new direction only when rho exceeds
    tol_rel * ||x||, a threshold relative to the row. Reading (residual dropped): the row then
    lies in span(V) to rounding, z/rho is not a unit vector, and the factorisation is taken
    with the (r+1) x r core [S; p^T] and right factor V Z (rank unchanged), which is the same
    as keeping rho = 0 and discarding the zero singular value it produces.

    Returns (U', s', V', rho, p, rank_grew).
    """
    x = np.asarray(x, dtype=np.float64)
    r = s.size
    m = U.shape[0]
    p = V.T @ x
    z = x - V @ p
    rho = float(np.linalg.norm(z))
    left = np.zeros((m + 1, r + 1))          # blkdiag(U, 1)
    left[:m, :r] = U
    left[m, r] = 1.0
    grew = rho > tol_rel * float(np.linalg.norm(x))
    if grew:
        K = np.zeros((r + 1, r + 1))
        K[:r, :r] = np.diag(s)
        K[r, :r] = p
        K[r, r] = rho
        right = np.hstack([V, (z / rho)[:, None]])
        W, s_new, Zt = np.linalg.svd(K)
    else:
        K = np.vstack([np.diag(s), p[None, :]])
        right = V
        W, s_new, Zt = np.linalg.svd(K, full_matrices=False)
    return left @ W, s_new, right @ Zt.T, rho, p, grew


def col_append_update(U, s, V, y, tol_rel):
    """ColAppendUpdateViaTranspose, Algorithm A2: row append on A^T with
    U~ = V, V~ = U, then transpose back (U' = V~', V' = U~')."""
    Ut, sK, Vt, rho, p, grew = row_append_update(V, s, U, y, tol_rel)
    return Vt, sK, Ut, rho, p, grew


def rank_one_update(U, s, V, i, j, delta):
    """RankOneUpdate, Algorithm A3 / Section 2.3.

    s_u = U[i, :], s_v = row j of V (Reading: the text's "j-th column of V" is read as
    Algorithm A3's (V^T)[:, j], i.e. the coordinates of e_j in span(V)).
    K = Sigma + delta s_u s_v^T (r x r), SVD K = U_K S' V_K^T, U' = U U_K, V' = V V_K.
    """
    su = U[i, :].copy()
    sv = V[j, :].copy()
    K = np.diag(s) + delta * np.outer(su, sv)
    UK, sK, VKt = np.linalg.svd(K)
    return U @ UK, sK, V @ VKt.T


def residual_direction(Q, e, tol_rel):
    """Coordinates c = Q^T e of a unit vector e in span(Q) and its residual direction: e = Q c +
    alpha d with d orthogonal to span(Q), alpha = ||e - Q c|| (two Gram-Schmidt passes, as for the
    appends' residual); alpha <= tol_rel counts as zero (d = 0)."""
    c = Q.T @ e
    z = e - Q @ c
    c2 = Q.T @ z
    z = z - Q @ c2
    c = c + c2
    alpha = float(np.linalg.norm(z))
    if alpha <= tol_rel:
        return c, 0.0, np.zeros_like(e)
    return c, alpha, z / alpha


def rank_one_update_exact(U, s, V, i, j, delta, tol_rel):
    """The rank-increasing form of the entry update (Brand's rank-one modification, the general
    form of Section 2.3's A + delta e_i e_j^T that the projection rule, Eq. (rank1-projection),
    approximates): with e_i = U p + alpha P and e_j = V q + beta Q,

        U S V^T + delta e_i e_j^T = [U P] K [V Q]^T,  K = diag(S, 0) + delta [p; alpha] [q; beta]^T,

    an (r+1) x (r+1) core; its SVD K = W S' Z^T gives U' = [U P] W and V' = [V Q] Z, exactly the
    SVD of the updated low-rank matrix before truncation."""
    m, n = U.shape[0], V.shape[0]
    ei = np.zeros(m)
    ei[i] = 1.0
    ej = np.zeros(n)
    ej[j] = 1.0
    p, alpha, P = residual_direction(U, ei, tol_rel)
    q, beta, Q = residual_direction(V, ej, tol_rel)
    r = s.size
    K = np.zeros((r + 1, r + 1))
    K[:r, :r] = np.diag(s)
    K += delta * np.outer(np.append(p, alpha), np.append(q, beta))
    W, sK, Zt = np.linalg.svd(K)
    return np.hstack([U, P[:, None]]) @ W, sK, np.hstack([V, Q[:, None]]) @ Zt.T


def truncate(U, s, V, k):
    """Truncate: keep the top-k singular values (already descending from LAPACK,
    stable order on ties) and the matching columns (Algorithm 1, "Truncate")."""
    r = min(k, s.size)
    return U[:, :r].copy(), s[:r].copy(), V[:, :r].copy()


def theta_max(Q1: np.ndarray, Q2: np.ndarray) -> float:
    """Largest principal angle, Eq. (theta-max): arccos(sigma_min(Q1^T Q2)).

    Reading: when Q1 has fewer rows than Q2 (rows were appended after Q1 was stored),
    Q1 is embedded with zero rows, i.e. the stored subspace seen inside the larger
    space. The cosine is clipped to [0, 1] (principal angles lie in [0, pi/2])."""
    Q1 = np.asarray(Q1, dtype=np.float64)
    Q2 = np.asarray(Q2, dtype=np.float64)
    m = max(Q1.shape[0], Q2.shape[0])
    if Q1.shape[0] < m:
        Q1 = np.vstack([Q1, np.zeros((m - Q1.shape[0], Q1.shape[1]))])
    if Q2.shape[0] < m:
        Q2 = np.vstack([Q2, np.zeros((m - Q2.shape[0], Q2.shape[1]))])
    if Q1.shape[1] == 0 or Q2.shape[1] == 0:
        return float("nan")
    mu = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    return float(np.arccos(np.clip(mu.min(), 0.0, 1.0)))


# ---------------------------------------------------------------------------
# Policies and metrics containers
# ---------------------------------------------------------------------------

@dataclass
class Policy:
    """Refresh / rank policy (Section 3). ``kind`` is a bit set of POLICY_* flags.

    Reading (evaluation time): the policy runs after every update (t counts all
    three update kinds, Section 3.1); error, angle and EVR signals are recomputed
    only on check steps (t % check_every == 0), the steps at which Section 4 takes a full
    SVD of A_t.
    """

    kind: int = POLICY_NONE
    T_refresh: int = 0
    T_min: int = 0
    check_every: int = 0
    gamma: float = 1.1
    theta_max: float = np.pi / 2
    tau_evr: float = 0.9
    tau_shrink: float = 0.99
    k_min: int = 1
    k_max: int = 0
    store_initial_subspace: bool = False
    eta: float = 0.5


@dataclass
class Metrics:
    t: int = 0
    m: int = 0
    n: int = 0
    r: int = 0
    frob_error: float = float("nan")
    frob_opt: float = float("nan")
    frob_gap: float = float("nan")
    frob_ratio: float = float("nan")
    angle: float = float("nan")
    angle_to_opt: float = float("nan")
    evr: float = float("nan")
    angle_succ_u: float = float("nan")
    angle_succ_v: float = float("nan")
    refreshed: bool = False


# ---------------------------------------------------------------------------
# The engine (Algorithm 1)
# ---------------------------------------------------------------------------

class _Dense:
    """Growable dense store of A_t (the engine keeps A for refresh and A_ij)."""

    def __init__(self, A0):
        A0 = np.asarray(A0, dtype=np.float64)
        self.m, self.n = A0.shape
        self.buf = np.zeros((max(4, 2 * self.m), max(4, 2 * self.n)))
        self.buf[:self.m, :self.n] = A0

    def view(self):
        return self.buf[:self.m, :self.n]

    def _grow(self, rows, cols):
        R, C = self.buf.shape
        if rows <= R and cols <= C:
            return
        nb = np.zeros((max(R, 2 * rows), max(C, 2 * cols)))
        nb[:self.m, :self.n] = self.view()
        self.buf = nb

    def append_row(self, x):
        self._grow(self.m + 1, self.n)
        self.buf[self.m, :self.n] = x
        self.m += 1

    def append_col(self, y):
        self._grow(self.m, self.n + 1)
        self.buf[:self.m, self.n] = y
        self.n += 1


class OracleISVD:
    """State (U, sigma, V, A, N_t, t, U_ref) and the three update rules.

    ``create`` follows the initialisation of Algorithm 1 and Section 2.4: (U, S, V) from the
    truncated SVD of A0 at rank r0 = min(k, m0, n0) (Reading: the paper's rank-k
    truncated SVD when A0 has fewer than k rows or columns), N_0 = ||A0||_F^2,
    U_ref = U_0.
    """

    def __init__(self, A0, k, tol_rel=1e-10, policy: Policy | None = None, factors=None):
        self.A = _Dense(A0)
        self.k = int(k)          # current working rank k_t
        self.tol_rel = float(tol_rel)
        self.policy = policy or Policy()
        if factors is None:
            self.U, self.s, self.V = truncated_svd(self.A.view(), self.k)
        else:                    # resume from given factors (U0, sigma0, V0)
            self.U, self.s, self.V = (np.array(f, dtype=np.float64, copy=True) for f in factors)
        self.N = float(np.sum(self.A.view() ** 2))   # N_0 = ||A_0||_F^2
        self.U_ref = self.U.copy()
        self.t = 0
        self.t_last = 0
        self.refreshes = 0
        self.rho_last = float("nan")
        self.novelty_last = float("nan")
        self.angle_succ_u = float("nan")   # largest principal angle between span(U_{t-1}) and span(U_t)
        self.angle_succ_v = float("nan")
        self.log: list[Metrics] = []

    # -- shape helpers ------------------------------------------------------
    @property
    def r(self):
        return int(self.s.size)

    @property
    def m(self):
        return self.A.m

    @property
    def n(self):
        return self.A.n

    def A_view(self):
        return self.A.view()

    def reconstruction(self):
        return (self.U * self.s) @ self.V.T

    # -- update primitives (Algorithm 1 loop body) --------------------------
    def append_row(self, x):
        x = np.asarray(x, dtype=np.float64)
        assert x.size == self.n
        self.A.append_row(x)                              # append x^T to A
        self.N += float(x @ x)                            # N_{t+1} = N_t + ||x||^2
        U, s, V, rho, p, _ = row_append_update(self.U, self.s, self.V, x, self.tol_rel)
        U0, V0 = self.U, self.V
        self.U, self.s, self.V = truncate(U, s, V, self.k)
        self._successive_angles(U0, V0)
        self.rho_last = rho
        nx = float(np.linalg.norm(x))
        self.novelty_last = rho / nx if nx > 0 else 0.0   # ||z|| / ||x|| (Section 3.3)
        self._novelty_rule(rho, nx)
        self._after_update()

    def append_col(self, y):
        y = np.asarray(y, dtype=np.float64)
        assert y.size == self.m
        self.A.append_col(y)                              # append y as right-most column
        self.N += float(y @ y)                            # N_{t+1} = N_t + ||y||^2
        U, s, V, rho, p, _ = col_append_update(self.U, self.s, self.V, y, self.tol_rel)
        U0, V0 = self.U, self.V
        self.U, self.s, self.V = truncate(U, s, V, self.k)
        self._successive_angles(U0, V0)
        self.rho_last = rho
        ny = float(np.linalg.norm(y))
        self.novelty_last = rho / ny if ny > 0 else 0.0
        self._novelty_rule(rho, ny)
        self._after_update()

    def update_entry(self, i, j, delta):
        i, j, delta = int(i), int(j), float(delta)
        assert 0 <= i < self.m and 0 <= j < self.n
        Av = self.A.view()
        a_ij = float(Av[i, j])
        self.N += 2.0 * delta * a_ij + delta * delta      # N_{t+1} = N_t + 2 delta A_ij + delta^2
        Av[i, j] = a_ij + delta                           # A_ij <- A_ij + delta
        U, s, V = rank_one_update(self.U, self.s, self.V, i, j, delta)
        U0, V0 = self.U, self.V
        self.U, self.s, self.V = truncate(U, s, V, self.k)
        self._successive_angles(U0, V0)
        self._after_update()

    def update_entry_exact(self, i, j, delta):
        """A_ij <- A_ij + delta through the rank-increasing core (rank_one_update_exact), then
        truncation at k_t; the same bookkeeping and policy step as update_entry."""
        i, j, delta = int(i), int(j), float(delta)
        assert 0 <= i < self.m and 0 <= j < self.n
        Av = self.A.view()
        a_ij = float(Av[i, j])
        self.N += 2.0 * delta * a_ij + delta * delta
        Av[i, j] = a_ij + delta
        U, s, V = rank_one_update_exact(self.U, self.s, self.V, i, j, delta, self.tol_rel)
        U0, V0 = self.U, self.V
        self.U, self.s, self.V = truncate(U, s, V, self.k)
        self._successive_angles(U0, V0)
        self._after_update()

    def apply(self, kind, vec=None, i=0, j=0, delta=0.0):
        if kind == ROW:
            self.append_row(vec)
        elif kind == COL:
            self.append_col(vec)
        elif kind == ENTRY:
            self.update_entry(i, j, delta)
        else:
            raise ValueError(kind)

    def run(self, events, start=0, stop=None):
        """Apply events[start:stop] of a ``streams.EventStream``-like object."""
        stop = len(events) if stop is None else stop
        for e in range(start, stop):
            kd = int(events.kind[e])
            if kd == ENTRY:
                self.update_entry(events.i[e], events.j[e], events.delta[e])
            else:
                self.apply(kd, events.vector(e))

    # -- refresh and metrics ------------------------------------------------
    def refresh(self, store_initial_subspace=None):
        """Refresh (Section 2.4): truncated SVD of the current A_t at the current
        working rank k_t; optionally U_ref <- U_t."""
        self.U, self.s, self.V = truncated_svd(self.A.view(), self.k)
        self.t_last = self.t
        self.refreshes += 1
        sis = self.policy.store_initial_subspace if store_initial_subspace is None else store_initial_subspace
        if sis:
            self.U_ref = self.U.copy()

    def metrics(self) -> Metrics:
        """Section 2.5 metrics on the current state.

        E_inc = ||A_t - U S V^T||_F (formed explicitly); E_opt from the full SVD of
        A_t as the tail sqrt(sum_{i>r} s_i^2) at the maintained rank r = r_t
        (Reading: the best approximation of the same rank as the maintained one, so
        that Eckart-Young gives ratio >= 1); ratio NaN when E_opt is numerically zero
        (Reading: E_opt <= 1e-12 sqrt(N_t)); EVR = sum sigma^2 / N_t (Eq. evr);
        angle = theta_max(U_ref, U_t), angle_to_opt = theta_max(U_opt, U_t).
        """
        A = self.A.view()
        E_inc = float(np.linalg.norm(A - self.reconstruction()))
        W, s_full, _ = np.linalg.svd(A, full_matrices=False)
        r = self.r
        E_opt = float(np.sqrt(np.sum(s_full[r:] ** 2)))
        if E_opt <= 1e-12 * np.sqrt(max(self.N, 0.0)):
            ratio = float("nan")
        else:
            ratio = E_inc / E_opt
        U_opt = W[:, :r]
        mt = Metrics(t=self.t, m=self.m, n=self.n, r=r, frob_error=E_inc, frob_opt=E_opt,
                     frob_gap=E_inc - E_opt, frob_ratio=ratio,
                     angle=theta_max(self.U_ref, self.U),
                     angle_to_opt=theta_max(U_opt, self.U),
                     evr=float(np.sum(self.s ** 2) / self.N) if self.N > 0 else float("nan"),
                     angle_succ_u=self.angle_succ_u, angle_succ_v=self.angle_succ_v)
        return mt

    def _successive_angles(self, U0, V0):
        """Section 3.3, "subspace-change per update": the largest principal angle between the
        subspaces before and after the update, Eq. (theta-max) applied to (U_{t-1}, U_t) and to
        (V_{t-1}, V_t). Reading: an appended row (column) extends the previous basis by a zero
        row, as for the angle to the stored basis; with bases of different ranks the angle is
        taken over the min(r_{t-1}, r_t) principal angles (zero when one span contains the other)."""
        self.angle_succ_u = theta_max(U0, self.U)
        self.angle_succ_v = theta_max(V0, self.V)

    def _novelty_rule(self, rho, xnorm):
        """Eq. (novelty-rank-rule): ||z_t|| > eta ||x_t||  =>  k_{t+1} <- min(k_t + 1, k_max).
        Reading: the rule acts after the append (the append itself is truncated at k_t), for row
        and column appends alike, and the grown rank takes effect at the next update."""
        pol = self.policy
        if pol.kind & POLICY_NOVELTY_RANK and rho > pol.eta * xnorm:
            self.k = min(self.k + 1, pol.k_max if pol.k_max > 0 else self.k + 1)

    def _after_update(self):
        """t <- t + 1, then the refresh rule pi(t, metrics) (Algorithm 1)."""
        self.t += 1
        pol = self.policy
        fire = False
        mt = None
        if pol.kind & POLICY_PERIODIC and pol.T_refresh > 0 and self.t % pol.T_refresh == 0:
            fire = True                                   # Eq. (periodic-refresh-rule)
        if pol.check_every > 0 and self.t % pol.check_every == 0:
            mt = self.metrics()
            spaced = (self.t - self.t_last) >= pol.T_min
            if pol.kind & POLICY_ERROR and spaced and np.isfinite(mt.frob_ratio) \
                    and mt.frob_ratio > pol.gamma:
                fire = True                               # Eq. (error-refresh-rule)
            if pol.kind & POLICY_ANGLE and spaced and np.isfinite(mt.angle_to_opt) \
                    and mt.angle_to_opt > pol.theta_max:
                fire = True                               # angle-based rule, Section 3.3
            if pol.kind & POLICY_ADAPTIVE_RANK and np.isfinite(mt.evr) and mt.evr < pol.tau_evr:
                # Reading of Eq. (evr-rank-rule) as "grow k while EVR < tau", one step
                # per check, bounded by k_max.
                self.k = min(self.k + 1, pol.k_max if pol.k_max > 0 else self.k + 1)
            elif pol.kind & POLICY_RANK_SHRINK and self.k > max(pol.k_min, 1) and self.N > 0:
                # The shrink side (Section 6's remark, and Eq. (evr-rank-rule)'s smallest k): when
                # the leading k - 1 components alone explain at least tau_shrink of N_t (a target
                # above tau, the hysteresis against oscillation), k <- k - 1 and the smallest
                # maintained component is dropped, one step per check, bounded by k_min.
                evr_km1 = float(np.sum(self.s[:self.k - 1] ** 2) / self.N)
                if evr_km1 >= pol.tau_shrink:
                    self.k -= 1
                    self.U, self.s, self.V = truncate(self.U, self.s, self.V, self.k)
        if fire:
            self.refresh()
        if mt is not None:
            mt.refreshed = fire
            self.log.append(mt)

