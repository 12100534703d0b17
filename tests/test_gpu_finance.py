"""The finance layer (Section 5) on the GPU against the oracle, through the C ABI: causal and EW
centering of return rows (Section 5.1), and the low-rank covariance, portfolio volatility, risk
error and covariance error of an incremental factor model of centered returns (Section 5.3),
on a factor-model return panel shaped like the paper's ETF study (60 assets, an initial window
of 250 days, k = 5, one appended row per day, periodic refresh every 100 days)."""
import numpy as np
import pytest

import oracle
from oracle import finance as F
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mode", [F.CAUSAL, F.EW])
def test_centering_matches_oracle(isvd, prec, mode):
    dt = np.float64 if prec == 0 else np.float32
    raw, fm = streams.make_panel(90, 17, 4, seed=3)
    raw = (raw + 0.001).astype(dt)                         # returns with a drift
    alpha = 0.05 if mode == F.EW else 0.0
    c = isvd.Centering(17, mode=mode, alpha=alpha, prec=prec)
    got = np.vstack([c.rows(raw[:40]), c.rows(raw[40:41]), c.rows(raw[41:])])   # state carried across calls
    exp, mu, cnt = F.center_rows(raw.astype(np.float64), mode, alpha=alpha)
    np.testing.assert_array_equal(got, exp.astype(dt))     # the same FP64 arithmetic, one rounding to dt
    mu_g, cnt_g = c.state()
    np.testing.assert_array_equal(mu_g, mu)
    assert cnt_g == cnt == 90
    # a new asset joins with its own mean; its column is centered from then on
    c.add_assets([0.25])
    row = np.append(raw[-1], dt(0.5)).astype(dt)[None, :]
    exp2, _, _ = F.center_rows(row.astype(np.float64), mode, alpha=alpha, mu=np.append(mu, 0.25), count=cnt)
    np.testing.assert_array_equal(c.rows(row), exp2.astype(dt))
    c.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_risk_and_covariance_errors_match_oracle(isvd, prec):
    dt = np.float64 if prec == 0 else np.float32
    tol_rel = 1e-10 if prec == 0 else 1e-5
    tol_abs = 1e-9 if prec == 0 else 5e-5
    # The covariance error is evaluated through r x r Grams (||C1 - C2||^2 = ||C1||^2 + ||C2||^2 -
    # 2 <C1, C2>), which cancels to about sqrt(eps) relative when the two covariances coincide (right
    # after a refresh): that is the FP64 floor of this quantity, not of the factors.
    tol_cov = 1e-7 if prec == 0 else 5e-5
    raw, fm = streams.make_panel(450, 60, 8, seed=17)
    raw = raw.astype(dt)
    R, _, _ = F.center_rows(raw.astype(np.float64), F.CAUSAL)
    R = R.astype(dt)                                        # the centered panel, in the storage type
    T0, k = 250, 5
    A0 = R[:T0]
    pol = oracle.Policy(kind=oracle.POLICY_PERIODIC, T_refresh=100)
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=1e-10 if prec == 0 else 3e-6, policy=pol)
    g = isvd.ISVD(A0, k, prec=prec)
    g.set_policy(kind=isvd.POLICY_PERIODIC, T_refresh=100)
    w_rand = np.random.default_rng(4).dirichlet(np.ones(60))
    for day in range(T0, 450):
        g.append_row(R[day])
        o.append_row(R[day].astype(np.float64))
        if (day + 1 - T0) % 50 == 0:
            t = o.m
            Wo, so, Zt = np.linalg.svd(o.A_view(), full_matrices=False)
            Vopt, sopt = Zt[:o.r].T, so[:o.r]
            for w in (None, w_rand.astype(dt)):
                ww = np.full(60, 1 / 60) if w is None else w.astype(np.float64)
                got = g.risk(w=w, full=True)
                assert got["t"] == t and got["r"] == o.r
                vol = F.portfolio_vol(o.V, o.s, t, ww)
                vol_opt = F.portfolio_vol(Vopt, sopt, t, ww)
                assert abs(got["vol"] - vol) <= tol_rel * vol, day
                assert abs(got["vol_opt"] - vol_opt) <= tol_rel * vol_opt, day
                assert abs(got["risk_error"] - F.risk_error(o.V, o.s, Vopt, sopt, t, ww)) <= tol_abs, day
                assert abs(got["cov_error"] - F.covariance_error(o.V, o.s, Vopt, sopt, t)) <= tol_cov, day
                cov_norm = np.linalg.norm(F.lowrank_covariance(o.V, o.s, t))
                assert abs(got["cov_norm"] - cov_norm) <= tol_rel * cov_norm, day
    cheap = g.risk(full=False)
    assert np.isnan(cheap["vol_opt"]) and np.isnan(cheap["cov_error"]) and cheap["vol"] > 0
