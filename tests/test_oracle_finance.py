"""Pins of the finance-layer oracle (Section 5) against closed forms and independent computations.

Each pin fixes something a plausible slip would break: the centering divisor (t vs t - 1), the
EW weights (a and 1 - a swapped), the covariance normalisation 1 / (t - 1), sigma vs sigma^2, and
the sign freedom of singular vectors.
"""
import numpy as np
import pytest

from oracle import finance as F

rng = np.random.default_rng(5)


def test_causal_centering_closed_forms():
    # a constant series centers to zero; a ramp r_t = c t (t = 1, 2, ...) to c (t - 1) / 2
    const = np.tile(np.array([[0.3, -1.2, 5.0]]), (7, 1))
    out, mu, cnt = F.center_rows(const, F.CAUSAL)
    assert np.abs(out).max() == 0.0 and cnt == 7
    t = np.arange(1, 9, dtype=np.float64)[:, None]
    c = np.array([[2.0, -0.5]])
    out, mu, _ = F.center_rows(t * c, F.CAUSAL)
    np.testing.assert_allclose(out, c * (t - 1) / 2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(mu, c[0] * 4.5, rtol=1e-15)


def test_causal_centering_is_expanding_mean():
    raw = rng.standard_normal((40, 6))
    out, _, _ = F.center_rows(raw, F.CAUSAL)
    expanding = np.cumsum(raw, axis=0) / np.arange(1, 41)[:, None]
    np.testing.assert_allclose(out, raw - expanding, rtol=0, atol=1e-13)


def test_ew_centering_closed_form():
    a, c = 0.1, 3.0
    out, mu, _ = F.center_rows(np.full((12, 2), c), F.EW, alpha=a)
    t = np.arange(1, 13)[:, None]
    # mu_t = c (1 - (1 - a)^t) from mu_0 = 0, so r_t - mu_t = c (1 - a)^t
    np.testing.assert_allclose(out, c * (1 - a) ** t * np.ones((1, 2)), rtol=1e-13)


def test_centering_in_batches_equals_one_pass():
    raw = rng.standard_normal((30, 5))
    for mode, a in ((F.CAUSAL, 0.0), (F.EW, 0.2)):
        whole, mu, cnt = F.center_rows(raw, mode, alpha=a)
        o1, m1, c1 = F.center_rows(raw[:11], mode, alpha=a)
        o2, m2, c2 = F.center_rows(raw[11:], mode, alpha=a, mu=m1, count=c1)
        np.testing.assert_array_equal(np.vstack([o1, o2]), whole)
        assert c2 == cnt


def test_covariance_from_svd_identity():
    # Eq. (cov-from-svd): with every component, V diag(s^2) V^T / (t - 1) is the sample covariance
    R = rng.standard_normal((25, 7))
    _, s, Vt = np.linalg.svd(R, full_matrices=False)
    np.testing.assert_allclose(F.lowrank_covariance(Vt.T, s, 25), F.sample_covariance(R), rtol=1e-12, atol=1e-14)
    # the sample covariance of centered columns is numpy's (ddof = 1) covariance
    Rc = R - R.mean(axis=0)
    np.testing.assert_allclose(F.sample_covariance(Rc), np.cov(Rc, rowvar=False), rtol=1e-12, atol=1e-15)


def test_portfolio_vol_is_the_std_of_the_reconstructed_portfolio_returns():
    R = rng.standard_normal((30, 9))
    U, s, Vt = np.linalg.svd(R, full_matrices=False)
    k = 4
    Ak = (U[:, :k] * s[:k]) @ Vt[:k]
    for w in (np.full(9, 1 / 9), rng.dirichlet(np.ones(9)), np.eye(9)[3]):
        series = Ak @ w                       # the rank-k factor model's portfolio return series
        np.testing.assert_allclose(F.portfolio_vol(Vt[:k].T, s[:k], 30, w), np.sqrt(series @ series / 29),
                                   rtol=1e-12)


def test_covariance_and_risk_errors_closed_forms():
    V, _ = np.linalg.qr(rng.standard_normal((8, 3)))
    s = np.array([3.0, 2.0, 0.5])
    assert F.covariance_error(V, s, V, s, 10) == 0.0
    eps = 1e-3
    # sigma scaled by (1 + eps): the covariance scales by (1 + eps)^2, the volatility by (1 + eps)
    np.testing.assert_allclose(F.covariance_error(V, s * (1 + eps), V, s, 10), (1 + eps) ** 2 - 1, rtol=1e-10)
    w = rng.dirichlet(np.ones(8))
    np.testing.assert_allclose(F.risk_error(V, s * (1 + eps), V, s, 10, w), eps, rtol=1e-10)
    # sign-free: flipping columns of V changes nothing
    Vf = V * np.array([1.0, -1.0, -1.0])
    assert F.covariance_error(Vf, s, V, s, 10) < 1e-15
    assert F.risk_error(Vf, s, V, s, 10, w) < 1e-15


@pytest.mark.parametrize("bad", ["divisor", "sigma", "ew", "count"])
def test_planted_mistakes_fail_a_pin(bad):
    """Each plausible slip, written out, violates the closed form that the pins above check."""
    if bad == "divisor":      # covariance normalised by t instead of t - 1
        R = rng.standard_normal((25, 7))
        _, s, Vt = np.linalg.svd(R, full_matrices=False)
        assert not np.allclose((Vt.T * s ** 2) @ Vt / 25, F.sample_covariance(R), rtol=1e-6)
    elif bad == "sigma":      # sigma instead of sigma^2 in the low-rank covariance
        V, _ = np.linalg.qr(rng.standard_normal((8, 3)))
        s = np.array([3.0, 2.0, 0.5])
        wrong = np.linalg.norm((V * (s * 1.001)) @ V.T - (V * s) @ V.T) / np.linalg.norm((V * s) @ V.T)
        assert abs(wrong - (1.001 ** 2 - 1)) > 1e-4
    elif bad == "ew":         # EW weights swapped
        a, c, mu = 0.1, 3.0, 0.0
        for _ in range(12):
            mu = a * mu + (1 - a) * c
        assert abs((c - mu) - c * (1 - a) ** 12) > 1e-3
    else:                     # expanding mean divided by t - 1 (off by one)
        t = np.arange(1, 9, dtype=np.float64)
        mu, out = 0.0, []
        for i, r in enumerate(2.0 * t):
            mu = mu + (r - mu) / max(i, 1)
            out.append(r - mu)
        assert not np.allclose(out, 2.0 * (t - 1) / 2)
