"""Pins of the oracle's local angular signals (Section 3.3) and novelty rank rule (Eq.
novelty-rank-rule) against closed forms that use a different route than the oracle's own.

The oracle measures the successive-subspace angle by definition (Eq. theta-max on the bases before
and after the update). The closed forms used here come from the block structure of the update:
after a row append U_t = blkdiag(U_{t-1}, 1) W_k, so [U_{t-1}; 0]^T U_t is W_k without its last row,
whose smallest singular value is sqrt(1 - ||c||^2) with c the last row of W_k, which is the new
row of U_t. Hence sin(angle_u) = ||U_t[-1, :]|| whenever the rank did not grow (k_t <= r_{t-1}).
Likewise V_t = [V_{t-1}, z_hat] Z_k gives sin(angle_v) = ||V_t^T z_hat||.
"""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(11)


def _stream(m=40, n=18, k=5, **pol):
    A0 = rng.standard_normal((m, 6)) @ rng.standard_normal((6, n)) + 1e-3 * rng.standard_normal((m, n))
    return oracle.OracleISVD(A0, k, tol_rel=1e-10, policy=oracle.Policy(**pol) if pol else None)


def test_successive_angle_row_append_closed_forms():
    o = _stream()
    for _ in range(6):
        V0 = o.V.copy()
        x = rng.standard_normal(o.n)
        z = x - V0 @ (V0.T @ x)
        zhat = z / np.linalg.norm(z)
        r0 = o.r
        o.append_row(x)
        assert o.r == r0                                   # truncated back to k: the rank did not grow
        np.testing.assert_allclose(o.angle_succ_u, np.arcsin(np.linalg.norm(o.U[-1])), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(o.angle_succ_v, np.arcsin(np.linalg.norm(o.V.T @ zhat)), rtol=1e-9, atol=1e-12)
        assert 0.0 < o.angle_succ_u < np.pi / 2


def test_successive_angle_col_append_is_the_transposed_row_append():
    o = _stream()
    U0 = o.U.copy()
    y = rng.standard_normal(o.m)
    z = y - U0 @ (U0.T @ y)
    o.append_col(y)
    np.testing.assert_allclose(o.angle_succ_v, np.arcsin(np.linalg.norm(o.V[-1])), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(o.angle_succ_u, np.arcsin(np.linalg.norm(o.U.T @ (z / np.linalg.norm(z)))),
                               rtol=1e-9, atol=1e-12)


def test_successive_angle_special_cases():
    o = _stream()
    # an entry update (Eq. rank1-projection) rotates within the current subspaces: no change of span
    o.update_entry(3, 4, 0.7)
    assert o.angle_succ_u < 1e-7 and o.angle_succ_v < 1e-7
    # a row inside span(V) keeps span(V); span(U) still tilts towards the new row
    x = o.V @ rng.standard_normal(o.r)
    o.append_row(x)
    assert o.angle_succ_v < 1e-7
    assert o.angle_succ_u > 1e-3
    # growing rank (k above r): the old span is contained in the new one
    o.k = o.r + 1
    o.append_row(rng.standard_normal(o.n))
    assert o.r == o.k
    assert o.angle_succ_u < 1e-7 and o.angle_succ_v < 1e-7


def test_novelty_rule_grows_k_on_novel_rows_only():
    o = _stream(kind=oracle.POLICY_NOVELTY_RANK, eta=0.3, k_max=7)
    k0 = o.k
    # a row inside span(V): novelty ~ 0, k unchanged
    o.append_row(o.V @ rng.standard_normal(o.r))
    assert o.novelty_last < 1e-8 and o.k == k0
    # a row orthogonal to span(V): novelty 1 > eta, k grows by one for the next update
    x = rng.standard_normal(o.n)
    x -= o.V @ (o.V.T @ x)
    r_before = o.r
    o.append_row(x)
    assert o.novelty_last == pytest.approx(1.0, abs=1e-12) and o.k == k0 + 1
    assert o.r == r_before                                 # this append itself was truncated at k_t
    # the next novel append keeps its new direction (rank k0 + 1), and the cap holds at k_max
    for _ in range(4):
        x = rng.standard_normal(o.n)
        x -= o.V @ (o.V.T @ x)
        o.append_row(x)
    assert o.k == 7 and o.r == 7


def test_novelty_rule_threshold_is_strict_and_reads_rho_over_norm():
    o = _stream(kind=oracle.POLICY_NOVELTY_RANK, eta=0.6, k_max=9)
    k0 = o.k
    # novelty 0.5 < eta: no growth; a column append with novelty 0.8 > eta: growth
    u = rng.standard_normal(o.n)
    u -= o.V @ (o.V.T @ u)
    u /= np.linalg.norm(u)
    w = o.V[:, 0]
    o.append_row(0.5 * u + np.sqrt(0.75) * w)
    assert o.novelty_last == pytest.approx(0.5, rel=1e-9) and o.k == k0
    y = rng.standard_normal(o.m)
    y -= o.U @ (o.U.T @ y)
    y /= np.linalg.norm(y)
    o.append_col(0.8 * y + 0.6 * o.U[:, 0])
    assert o.novelty_last == pytest.approx(0.8, rel=1e-9) and o.k == k0 + 1


def test_planted_reversed_novelty_comparison_fails_the_pin():
    """A copy of the rule with the comparison reversed grows k on an in-span row."""
    class Reversed(oracle.OracleISVD):
        def _novelty_rule(self, rho, xnorm):
            if self.policy.kind & oracle.POLICY_NOVELTY_RANK and rho < self.policy.eta * xnorm:
                self.k += 1
    A0 = rng.standard_normal((30, 12))
    o = Reversed(A0, 4, policy=oracle.Policy(kind=oracle.POLICY_NOVELTY_RANK, eta=0.3, k_max=8))
    o.append_row(o.V @ rng.standard_normal(o.r))
    assert o.k != 4


def _three_factor_stream(k, **pol):
    """A panel with three orthogonal components of energies 100, 25 and 4 (sigma 10, 5, 2) and
    negligible noise: EVR(1) = 100 / 129, EVR(2) = 125 / 129, EVR(3) ~ 1."""
    m, n = 50, 20
    Q1, _ = np.linalg.qr(rng.standard_normal((m, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, 3)))
    A0 = (Q1 * np.array([10.0, 5.0, 2.0])) @ Q2.T + 1e-6 * rng.standard_normal((m, n))
    return oracle.OracleISVD(A0, k, tol_rel=1e-10, policy=oracle.Policy(**pol))


def test_rank_shrink_stops_at_the_smallest_k_whose_k_minus_1_components_fall_short():
    # shrink while EVR(k - 1) >= 0.99: from k = 6 down to 3, where EVR(2) = 125 / 129 < 0.99
    o = _three_factor_stream(6, kind=oracle.POLICY_ADAPTIVE_RANK | oracle.POLICY_RANK_SHRINK,
                             check_every=1, tau_evr=0.9, tau_shrink=0.99, k_min=1, k_max=8)
    for t in range(6):
        o.update_entry(t, t, 0.0)                      # a no-op update: one check per step
    assert o.k == 3 and o.r == 3
    np.testing.assert_allclose(o.s, [10.0, 5.0, 2.0], rtol=1e-6)
    # with tau_shrink = 0.96, EVR(2) = 0.969 also qualifies: one more step down to 2
    o2 = _three_factor_stream(6, kind=oracle.POLICY_ADAPTIVE_RANK | oracle.POLICY_RANK_SHRINK,
                              check_every=1, tau_evr=0.5, tau_shrink=0.96, k_min=1, k_max=8)
    for t in range(6):
        o2.update_entry(t, t, 0.0)
    assert o2.k == 2 and o2.r == 2


def test_rank_shrink_respects_k_min_and_needs_the_flag():
    o = _three_factor_stream(6, kind=oracle.POLICY_ADAPTIVE_RANK | oracle.POLICY_RANK_SHRINK,
                             check_every=1, tau_evr=0.9, tau_shrink=0.99, k_min=5, k_max=8)
    for t in range(4):
        o.update_entry(t, t, 0.0)
    assert o.k == 5
    o = _three_factor_stream(6, kind=oracle.POLICY_ADAPTIVE_RANK, check_every=1, tau_evr=0.9)
    for t in range(4):
        o.update_entry(t, t, 0.0)
    assert o.k == 6                                    # growth-only rule: EVR ~ 1 >= tau, no change


def test_planted_shrink_on_evr_of_k_fails_the_pin():
    """Comparing EVR(k) instead of EVR(k - 1) shrinks one step too far (to k = 2)."""
    class Wrong(oracle.OracleISVD):
        def _after_update(self):
            self.t += 1
            evr_k = float(np.sum(self.s[:self.k] ** 2) / self.N)
            if self.k > 1 and evr_k >= self.policy.tau_shrink:
                self.k -= 1
                self.U, self.s, self.V = oracle.truncate(self.U, self.s, self.V, self.k)
    m, n = 50, 20
    Q1, _ = np.linalg.qr(rng.standard_normal((m, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, 3)))
    A0 = (Q1 * np.array([10.0, 5.0, 2.0])) @ Q2.T + 1e-6 * rng.standard_normal((m, n))
    o = Wrong(A0, 6, policy=oracle.Policy(kind=oracle.POLICY_RANK_SHRINK, tau_shrink=0.99))
    for t in range(6):
        o.update_entry(t, t, 0.0)
    assert o.k != 3
