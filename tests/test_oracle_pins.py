"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms,
brute-force LAPACK on explicitly formed matrices, a LAPACK-free one-sided Jacobi on the
same matrices, identities stated in the paper, and special cases that reduce to a plain full SVD.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import (OracleISVD, Policy, col_append_update, rank_one_update,
                    row_append_update, theta_max, truncate, truncated_svd)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def orth_err(Q):
    return float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()) if Q.shape[1] else 0.0


def lowrank(g, m, n, r, noise=0.0):
    A = g.standard_normal((m, r)) @ g.standard_normal((r, n))
    return A + noise * g.standard_normal((m, n))


# --- golden closed forms ---------------------------------------------------

def test_golden_rank1_diag2x2():
    d = json.load(open(os.path.join(GOLD, "rank1_diag2x2.json")))
    s = np.asarray(d["s"])
    U, V = np.eye(2), np.eye(2)
    U2, s2, V2 = rank_one_update(U, s, V, d["i"], d["j"], d["delta"])
    np.testing.assert_allclose(s2, d["sigma_expected"], rtol=1e-14)
    expect = np.diag(s)
    expect[d["i"], d["j"]] += d["delta"]
    np.testing.assert_allclose((U2 * s2) @ V2.T, expect, atol=1e-14)


def test_golden_row_append_diag2x2():
    d = json.load(open(os.path.join(GOLD, "row_append_diag2x2.json")))
    o = OracleISVD(np.asarray(d["A0"]), 2)
    o.append_row(np.asarray(d["x"]))
    np.testing.assert_allclose(o.s, d["sigma_expected"], rtol=1e-14)
    assert abs(o.rho_last - d["rho_expected"]) < 1e-14
    assert o.r == 2


# --- untruncated updates reproduce the full SVD -----------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_untruncated_rows_reproduce_full_svd(seed):
    g = rng(seed)
    A0 = lowrank(g, 7, 5, 3)                   # exact rank 3 < k = 5 = n
    o = OracleISVD(A0, 5)
    for _ in range(6):
        o.append_row(g.standard_normal(5))
        A = o.A_view()
        s_true = np.linalg.svd(A, compute_uv=False)
        np.testing.assert_allclose(o.s, s_true[:o.r], rtol=1e-11, atol=1e-12 * s_true[0])
        assert np.linalg.norm(A - o.reconstruction()) <= 1e-11 * np.linalg.norm(A)
    assert o.r == 5


@pytest.mark.parametrize("seed", [3, 4])
def test_untruncated_cols_reproduce_full_svd(seed):
    g = rng(seed)
    A0 = lowrank(g, 5, 7, 2)                   # exact rank 2 < k = 5 = m
    o = OracleISVD(A0, 5)
    for _ in range(6):
        o.append_col(g.standard_normal(5))
        A = o.A_view()
        s_true = np.linalg.svd(A, compute_uv=False)
        np.testing.assert_allclose(o.s, s_true[:o.r], rtol=1e-11, atol=1e-12 * s_true[0])
        assert np.linalg.norm(A - o.reconstruction()) <= 1e-11 * np.linalg.norm(A)


@pytest.mark.parametrize("seed", [5, 6])
def test_rank_one_full_rank_square_is_exact(seed):
    # k = m = n: P_U = P_V = I, so the projection rule is the exact rank-1 update.
    g = rng(seed)
    A0 = g.standard_normal((6, 6))
    o = OracleISVD(A0, 6)
    for _ in range(10):
        i, j, d = int(g.integers(6)), int(g.integers(6)), float(g.standard_normal())
        o.update_entry(i, j, d)
        A = o.A_view()
        np.testing.assert_allclose(o.s, np.linalg.svd(A, compute_uv=False), rtol=1e-11)
        assert np.linalg.norm(A - o.reconstruction()) <= 1e-12 * np.linalg.norm(A)


# --- per-step optimality (Eckart-Young on the core) ------------------------

@pytest.mark.parametrize("seed", range(4))
def test_row_append_is_best_rank_k_of_stacked(seed):
    g = rng(10 + seed)
    m, n, k = 9, 7, 3
    U, s, V = truncated_svd(g.standard_normal((m, n)), k)
    Ahat = (U * s) @ V.T
    x = g.standard_normal(n)
    U2, s2, V2, rho, p, grew = row_append_update(U, s, V, x, 1e-12)
    U2, s2, V2 = truncate(U2, s2, V2, k)
    Ub, sb, Vb = truncated_svd(np.vstack([Ahat, x[None, :]]), k)   # brute force
    np.testing.assert_allclose(s2, sb, rtol=1e-12)
    np.testing.assert_allclose((U2 * s2) @ V2.T, (Ub * sb) @ Vb.T, atol=1e-12)
    assert grew and rho > 0


@pytest.mark.parametrize("seed", range(4))
def test_col_append_is_best_rank_k_of_stacked(seed):
    g = rng(20 + seed)
    m, n, k = 7, 9, 4
    U, s, V = truncated_svd(g.standard_normal((m, n)), k)
    Ahat = (U * s) @ V.T
    y = g.standard_normal(m)
    U2, s2, V2, *_ = col_append_update(U, s, V, y, 1e-12)
    U2, s2, V2 = truncate(U2, s2, V2, k)
    Ub, sb, Vb = truncated_svd(np.hstack([Ahat, y[:, None]]), k)
    np.testing.assert_allclose(s2, sb, rtol=1e-12)
    np.testing.assert_allclose((U2 * s2) @ V2.T, (Ub * sb) @ Vb.T, atol=1e-12)
    assert U2.shape == (m, k) and V2.shape == (n + 1, k)


@pytest.mark.parametrize("seed", range(4))
def test_rank_one_projection_rule(seed):
    # Eq. (rank1-projection): U'S'V'^T = P_U (Ahat + delta e_i e_j^T) P_V, with the
    # projectors formed explicitly (no core SVD involved on the right-hand side).
    g = rng(30 + seed)
    m, n, k = 8, 6, 3
    U, s, V = truncated_svd(g.standard_normal((m, n)), k)
    Ahat = (U * s) @ V.T
    i, j, d = int(g.integers(m)), int(g.integers(n)), float(g.standard_normal())
    U2, s2, V2 = rank_one_update(U, s, V, i, j, d)
    E = np.zeros((m, n))
    E[i, j] = d
    expect = (U @ U.T) @ (Ahat + E) @ (V @ V.T)
    np.testing.assert_allclose((U2 * s2) @ V2.T, expect, atol=1e-12)
    assert orth_err(U2) < 1e-13 and orth_err(V2) < 1e-13
    assert np.all(np.diff(s2) <= 0)


def test_in_span_row_is_exact_and_rank_preserving():
    g = rng(40)
    U, s, V = truncated_svd(g.standard_normal((8, 6)), 3)
    Ahat = (U * s) @ V.T
    x = V @ g.standard_normal(3)                 # x in span(V)
    U2, s2, V2, rho, p, grew = row_append_update(U, s, V, x, 1e-10)
    assert rho <= 1e-14 * np.linalg.norm(x)
    assert not grew and s2.size == 3
    np.testing.assert_allclose((U2 * s2) @ V2.T, np.vstack([Ahat, x[None, :]]), atol=1e-13)
    assert orth_err(V2) < 1e-13 and orth_err(U2) < 1e-13


def test_zero_row_keeps_rank():
    g = rng(41)
    o = OracleISVD(g.standard_normal((6, 5)), 3)
    s0 = o.s.copy()
    o.append_row(np.zeros(5))
    assert o.r == 3
    np.testing.assert_allclose(o.s, s0, rtol=1e-13)


# --- invariants over a long mixed stream -----------------------------------

def _mixed_oracle(seed, steps=300, k=5, policy=None):
    g = rng(seed)
    A0 = lowrank(g, 30, 20, 6, noise=0.05)
    o = OracleISVD(A0, k, policy=policy)
    for _ in range(steps):
        u = g.random()
        if u < 0.5:
            o.append_row(g.standard_normal(6) @ g.standard_normal((6, o.n)) * 0.3 + 0.05 * g.standard_normal(o.n))
        elif u < 0.6:
            o.append_col(g.standard_normal(o.m))
        else:
            o.update_entry(int(g.integers(o.m)), int(g.integers(o.n)), 0.1 * g.standard_normal())
    return o


def test_invariants_long_mixed_stream():
    o = _mixed_oracle(50)
    A = o.A_view()
    assert orth_err(o.U) < 1e-12 and orth_err(o.V) < 1e-12
    # N_t maintained incrementally equals ||A_t||_F^2 (Section 2.5)
    assert abs(o.N - float(np.sum(A * A))) <= 1e-12 * o.N
    # ||Ahat||_F^2 = sum sigma^2 (orthonormal factors)
    assert abs(np.sum(o.reconstruction() ** 2) - np.sum(o.s ** 2)) <= 1e-12 * np.sum(o.s ** 2)
    mt = o.metrics()
    assert mt.frob_ratio >= 1 - 1e-12                       # Eckart-Young
    assert 0 <= mt.angle <= math.pi / 2 and 0 <= mt.angle_to_opt <= math.pi / 2
    # E_opt is the error of the best rank-r approximation (brute force)
    Ub, sb, Vb = truncated_svd(A, o.r)
    assert abs(mt.frob_opt - np.linalg.norm(A - (Ub * sb) @ Vb.T)) <= 1e-10 * mt.frob_opt
    assert np.all(np.diff(o.s) <= 0)


def test_refresh_resets_ratio_angle_and_evr_identity():
    o = _mixed_oracle(51, steps=120)
    before = o.metrics()
    assert before.frob_ratio > 1 + 1e-6                      # drift exists
    o.refresh()
    mt = o.metrics()
    assert abs(mt.frob_ratio - 1.0) < 1e-10
    assert mt.angle_to_opt < 1e-6
    # right after a refresh Ahat = A_opt, so EVR = 1 - E_opt^2 / N
    assert abs(mt.evr - (1 - mt.frob_opt ** 2 / o.N)) < 1e-12


def test_ratio_nan_when_opt_error_zero():
    g = rng(52)
    o = OracleISVD(lowrank(g, 10, 8, 2), 3)                  # rank 2 < k: E_opt = 0
    assert math.isnan(o.metrics().frob_ratio)


# --- principal angles -------------------------------------------------------

@pytest.mark.parametrize("theta", [0.0, 1e-3, 0.3, 1.0, math.pi / 2])
def test_theta_max_closed_form(theta):
    e = np.eye(4)
    Q1 = e[:, [0, 1]]
    Q2 = np.stack([e[:, 0], math.cos(theta) * e[:, 1] + math.sin(theta) * e[:, 2]], axis=1)
    assert abs(theta_max(Q1, Q2) - theta) < 1e-7


def test_theta_max_matches_sine_form():
    g = rng(60)
    for _ in range(5):
        Q1 = np.linalg.qr(g.standard_normal((12, 3)))[0]
        Q2 = np.linalg.qr(Q1 + 0.3 * g.standard_normal((12, 3)))[0]
        sin_form = np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2)
        assert abs(math.sin(theta_max(Q1, Q2)) - sin_form) < 1e-10


def test_theta_max_embeds_shorter_basis():
    e = np.eye(5)
    Q1 = e[:3, [0]]                       # stored 3-row basis
    Q2 = (e[:, [0]] + e[:, [4]]) / math.sqrt(2)
    assert abs(theta_max(Q1, Q2) - math.pi / 4) < 1e-12


# --- policies ---------------------------------------------------------------

def test_periodic_policy_counts():
    pol = Policy(kind=oracle.POLICY_PERIODIC, T_refresh=25)
    o = _mixed_oracle(70, steps=110, policy=pol)
    assert o.refreshes == 110 // 25 and o.t_last == 100


def test_error_policy_fires_and_respects_tmin():
    pol = Policy(kind=oracle.POLICY_ERROR, check_every=10, gamma=0.5, T_min=30)
    o = _mixed_oracle(71, steps=100, policy=pol)
    fired = [m.t for m in o.log if m.refreshed]
    assert fired == [30, 60, 90]
    pol2 = Policy(kind=oracle.POLICY_ERROR, check_every=10, gamma=1e9)
    assert _mixed_oracle(71, steps=50, policy=pol2).refreshes == 0


def test_angle_policy_fires():
    pol = Policy(kind=oracle.POLICY_ANGLE, check_every=20, theta_max=-1.0)
    o = _mixed_oracle(72, steps=60, policy=pol)
    assert o.refreshes == 3
    assert all(m.refreshed for m in o.log)


def test_adaptive_rank_grows_to_kmax():
    pol = Policy(kind=oracle.POLICY_ADAPTIVE_RANK, check_every=5, tau_evr=1.5, k_max=7)
    o = _mixed_oracle(73, steps=60, k=4, policy=pol)
    assert o.k == 7 and o.r == 7


def test_store_initial_subspace():
    g = rng(80)
    pol = Policy(store_initial_subspace=True)
    o = OracleISVD(lowrank(g, 20, 10, 4, 0.1), 3, policy=pol)
    for _ in range(10):
        o.append_row(g.standard_normal(10))
    assert o.metrics().angle > 1e-3
    o.refresh()
    assert o.metrics().angle < 1e-7


# --- core singular values against a LAPACK-free Jacobi ------------------------

def jacobi_singular_values(M, sweeps=80):
    """Plain one-sided (Hestenes) Jacobi written out in Python, independent of LAPACK: rotate
    column pairs of W = M until all pairs are orthogonal; the singular values are then the
    column norms, sorted descending."""
    W = np.array(M, dtype=np.float64, copy=True)
    n = W.shape[1]
    for _ in range(sweeps):
        worst = 0.0
        for a in range(n - 1):
            for b in range(a + 1, n):
                alpha = float(W[:, a] @ W[:, a])
                beta = float(W[:, b] @ W[:, b])
                gamma = float(W[:, a] @ W[:, b])
                if gamma == 0.0 or abs(gamma) <= 1e-16 * math.sqrt(alpha * beta):
                    continue
                worst = max(worst, abs(gamma) / math.sqrt(alpha * beta))
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                wa, wb = W[:, a].copy(), W[:, b].copy()
                W[:, a] = c * wa - s * wb
                W[:, b] = s * wa + c * wb
        if worst < 1e-15:
            break
    return np.sort(np.sqrt(np.sum(W * W, axis=0)))[::-1]


def test_jacobi_reference_on_closed_form():
    # diag(3, 1) rotated by orthogonal factors: singular values 3 and 1 whatever the rotations.
    th, ph = 0.3, 1.1
    Rl = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Rr = np.array([[math.cos(ph), math.sin(ph)], [-math.sin(ph), math.cos(ph)]])
    np.testing.assert_allclose(jacobi_singular_values(Rl @ np.diag([3.0, 1.0]) @ Rr), [3.0, 1.0], atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_update_spectra_match_lapack_free_jacobi(seed):
    # Sections 2.2-2.3: the untruncated core's singular values are those of the explicitly formed
    # updated matrix (stacked row, stacked column, or projected rank-one change), computed here by
    # the Jacobi above rather than by LAPACK.
    g = rng(70 + seed)
    m, n, k = 7, 5, 3
    U, s, V = truncated_svd(g.standard_normal((m, n)), k)
    Ahat = (U * s) @ V.T
    x = g.standard_normal(n)
    _, sK, _, _, _, grew = row_append_update(U, s, V, x, 1e-10)
    assert grew
    ref = jacobi_singular_values(np.vstack([Ahat, x[None, :]]))[:k + 1]
    np.testing.assert_allclose(sK, ref, rtol=0, atol=1e-12 * ref[0])
    y = g.standard_normal(m)
    sK2 = col_append_update(U, s, V, y, 1e-10)[1]
    ref2 = jacobi_singular_values(np.hstack([Ahat, y[:, None]]))[:k + 1]
    np.testing.assert_allclose(sK2, ref2, rtol=0, atol=1e-12 * ref2[0])
    i, j, d = int(g.integers(m)), int(g.integers(n)), float(g.standard_normal())
    s3 = rank_one_update(U, s, V, i, j, d)[1]
    E = np.zeros((m, n))
    E[i, j] = d
    ref3 = jacobi_singular_values((U @ U.T) @ (Ahat + E) @ (V @ V.T))[:k]
    np.testing.assert_allclose(s3, ref3, rtol=0, atol=1e-12 * ref3[0])
