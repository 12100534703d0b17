"""Pins of the oracle's rank-increasing entry update (Section 2.3's modification A + delta e_i e_j^T
in Brand's general form) against independent computations: the SVD of the explicitly formed
updated low-rank matrix (brute force), Eckart-Young after truncation, and the projection rule (Eq.
rank1-projection) when e_i and e_j lie in the current subspaces."""
import numpy as np

import oracle

rng = np.random.default_rng(23)


def _lowrank(m, n, r):
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s = np.sort(rng.uniform(0.5, 3.0, r))[::-1]
    return U, s, V


def test_exact_update_is_the_svd_of_the_updated_low_rank_matrix():
    U, s, V = _lowrank(30, 12, 4)
    for (i, j, d) in [(3, 5, 0.7), (0, 0, -1.3), (29, 11, 2.0)]:
        U2, s2, V2 = oracle.rank_one_update_exact(U, s, V, i, j, d, 1e-12)
        B = (U * s) @ V.T
        B[i, j] += d
        sv = np.linalg.svd(B, compute_uv=False)
        np.testing.assert_allclose(s2, sv[:5], rtol=1e-12, atol=1e-12)      # rank grows by one
        np.testing.assert_allclose((U2 * s2) @ V2.T, B, rtol=0, atol=1e-12)
        np.testing.assert_allclose(U2.T @ U2, np.eye(5), atol=1e-12)
        np.testing.assert_allclose(V2.T @ V2, np.eye(5), atol=1e-12)


def test_exact_update_truncated_is_eckart_young():
    U, s, V = _lowrank(25, 10, 3)
    U2, s2, V2 = oracle.truncate(*oracle.rank_one_update_exact(U, s, V, 7, 2, 0.9, 1e-12), 3)
    B = (U * s) @ V.T
    B[7, 2] += 0.9
    W, sv, Zt = np.linalg.svd(B)
    np.testing.assert_allclose(s2, sv[:3], rtol=1e-12)
    best = (W[:, :3] * sv[:3]) @ Zt[:3]
    np.testing.assert_allclose((U2 * s2) @ V2.T, best, atol=1e-11)


def test_exact_update_reduces_to_the_projection_rule_inside_the_spans():
    # U and V with e_i and e_j inside their spans: alpha = beta = 0, so the extra component is zero
    m, n, r = 12, 9, 4
    U = np.zeros((m, r))
    U[:r, :] = np.linalg.qr(rng.standard_normal((r, r)))[0]
    V = np.zeros((n, r))
    V[:r, :] = np.linalg.qr(rng.standard_normal((r, r)))[0]
    s = np.array([3.0, 2.0, 1.0, 0.5])
    Ue, se, Ve = oracle.rank_one_update_exact(U, s, V, 1, 2, 0.4, 1e-12)
    Up, sp, Vp = oracle.rank_one_update(U, s, V, 1, 2, 0.4)
    np.testing.assert_allclose(se[:r], sp, rtol=1e-12)
    assert abs(se[r]) < 1e-12
    np.testing.assert_allclose((Ue[:, :r] * se[:r]) @ Ve[:, :r].T, (Up * sp) @ Vp.T, atol=1e-12)


def test_engine_bookkeeping_of_the_exact_update():
    A0 = rng.standard_normal((20, 8)) @ rng.standard_normal((8, 15))
    o = oracle.OracleISVD(A0, 8, tol_rel=1e-12)
    N0 = o.N
    a = o.A_view()[4, 6]
    o.update_entry_exact(4, 6, 0.25)
    assert o.t == 1 and abs(o.N - (N0 + 2 * 0.25 * a + 0.0625)) < 1e-12
    # A had rank 8 = k, so the exact update of the rank-8 factorisation reproduces A + delta e e^T
    # up to the one dropped component
    sv = np.linalg.svd(o.A_view(), compute_uv=False)
    np.testing.assert_allclose(o.s, sv[:8], rtol=1e-10)


def test_planted_missing_residual_term_fails_the_pin():
    """Dropping alpha (the projection rule on both sides) misses the update's out-of-span part."""
    U, s, V = _lowrank(30, 12, 4)
    Up, sp, Vp = oracle.rank_one_update(U, s, V, 3, 5, 0.7)
    B = (U * s) @ V.T
    B[3, 5] += 0.7
    assert np.linalg.norm((Up * sp) @ Vp.T - B) > 1e-3
