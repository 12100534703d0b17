"""Refresh and rank policies (Section 3) on the GPU against the oracle, through the C ABI.

Each test runs the library and the oracle on the same seeded factor-model stream (70% row appends,
10% column appends, 20% entry updates, the mix of the 2,000 x 1,000 k = 64 workload reduced to a
200 x 80 panel so that the oracle finishes in seconds) with the same policy, and compares at
every check step: the signal the rule reads (error ratio, Eq. frob-ratio; largest principal angle
to the optimal subspace, Section 3.3; EVR, Eq. evr), whether a refresh fired (t_last), the working
rank k_t after the check, and at the end sigma and U S V^T.

The inputs were chosen so that every decision has a margin larger than the comparison tolerance
(the tests assert this margin from the oracle's own log, so a change of the inputs that makes a
decision borderline fails loudly instead of comparing coin flips).
"""
import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu

RECON_TOL = {0: 1e-10, 1: 1e-5}
RATIO_TOL = {0: 1e-9, 1: 1e-4}      # relative
ANGLE_TOL = {0: 1e-7, 1: 5e-4}      # radians (angles of a few degrees)
EVR_TOL = {0: 1e-10, 1: 1e-4}       # relative
# Randomized truncated SVD (min(m, n) > 128): power iterations and the relative accuracy of its
# E_opt against the exact optimum on the factor panel below, and the error threshold tested there.
RSVD_Q = 4
RSVD_ACC = 1e-3
RSVD_GAMMA = 1.006


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


def _stream(seed, k, n_events, m0=200, n0=80, f=10):
    A0, fm = streams.make_panel(m0, n0, f, seed)
    ev = streams.make_events(fm, m0, n_events, mix=(0.7, 0.1, 0.2), seed=seed + 1000)
    # min(m, n) stays <= 128, so refreshes and metrics take the exact truncated SVD
    assert ev.n_after.max() <= 128
    return A0, ev, k


def _run_lockstep(pkg, prec, A0, ev, k, pol_kw, k_max=0):
    """GPU and oracle side by side; returns the per-check records of both and the engines."""
    dt = np.float32 if prec == 1 else np.float64
    Ao = A0.astype(dt).astype(np.float64)
    pol = oracle.Policy(**pol_kw)
    o = oracle.OracleISVD(Ao, k, tol_rel=1e-10 if prec == 0 else 3e-6, policy=pol)
    g = pkg.ISVD(A0, k, prec=prec, k_max=k_max)
    kw = dict(pol_kw)
    kw["theta_max"] = kw.pop("theta_max", np.pi / 2)
    g.set_policy(**kw)
    ce = pol_kw["check_every"]
    recs = []
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            g.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            v = ev.vector(e).astype(dt)
            (g.append_row if kd == streams.ROW else g.append_col)(v)
            (o.append_row if kd == streams.ROW else o.append_col)(v.astype(np.float64))
        if (e + 1) % ce == 0:
            gm = g.last_check_metrics()
            om = o.log[-1]
            recs.append((gm, om, g.shape()[3], o.k))
    return g, o, recs


def _check_end(g, o, prec):
    U, s, V = g.factors()
    assert s.size == o.r
    np.testing.assert_allclose(s, o.s, rtol=0, atol=RECON_TOL[prec] * o.s[0])
    Ro = o.reconstruction()
    R = (U.astype(np.float64) * s) @ V.astype(np.float64).T
    assert np.linalg.norm(R - Ro) <= RECON_TOL[prec] * np.linalg.norm(Ro)


@pytest.mark.parametrize("prec", [0, 1])
def test_error_threshold_policy_matches_oracle(isvd, prec):
    """Eq. error-refresh-rule: refresh iff E_inc / E_opt > gamma, at least T_min after the last."""
    gamma, t_min = 1.006, 50
    A0, ev, k = _stream(7, 16, 400)
    pol = dict(kind=oracle.POLICY_ERROR, check_every=25, gamma=gamma, T_min=t_min)
    g, o, recs = _run_lockstep(isvd, prec, A0, ev, k, pol)
    t_last, fired = 0, 0
    for gm, om, kg, ko in recs:
        assert gm["t"] == om.t
        if om.t - t_last >= t_min:   # the decision is read only where the spacing allows it
            assert abs(om.frob_ratio - gamma) > 4 * RATIO_TOL[prec] * gamma, "borderline input"
        assert abs(gm["frob_ratio"] - om.frob_ratio) <= RATIO_TOL[prec] * om.frob_ratio, om.t
        assert (gm["t_last"] == gm["t"]) == om.refreshed, om.t
        if om.refreshed:
            t_last = om.t
            fired += 1
    assert fired == o.refreshes >= 3
    assert g.metrics(full=False)["refreshes"] == o.refreshes
    _check_end(g, o, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_angle_threshold_policy_matches_oracle(isvd, prec):
    """Section 3.3: refresh iff the largest principal angle to the optimal subspace exceeds
    theta_max (here 3 degrees, k = 3 so that the subspace is the factors' and well defined)."""
    theta, t_min = np.deg2rad(3.0), 50
    A0, ev, k = _stream(7, 3, 400)
    pol = dict(kind=oracle.POLICY_ANGLE, check_every=25, theta_max=theta, T_min=t_min)
    g, o, recs = _run_lockstep(isvd, prec, A0, ev, k, pol)
    t_last = 0
    for gm, om, kg, ko in recs:
        if om.t - t_last >= t_min:
            assert abs(om.angle_to_opt - theta) > 4 * ANGLE_TOL[prec], "borderline input"
        assert abs(gm["angle_to_opt"] - om.angle_to_opt) <= ANGLE_TOL[prec], om.t
        assert abs(gm["angle"] - om.angle) <= ANGLE_TOL[prec], om.t
        assert (gm["t_last"] == gm["t"]) == om.refreshed, om.t
        if om.refreshed:
            t_last = om.t
    assert o.refreshes >= 3
    assert g.metrics(full=False)["refreshes"] == o.refreshes
    _check_end(g, o, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_rank_policy_matches_oracle(isvd, prec):
    """Eq. evr-rank-rule read as a growth rule: k <- min(k + 1, k_max) at a check while
    EVR < tau; the new component arrives with the next append that keeps its residual."""
    A0, ev, k = _stream(4, 3, 300)
    pol = dict(kind=oracle.POLICY_ADAPTIVE_RANK, check_every=25, tau_evr=0.9, k_max=10)
    g, o, recs = _run_lockstep(isvd, prec, A0, ev, k, pol, k_max=12)
    ks = []
    for gm, om, kg, ko in recs:
        assert abs(om.evr - 0.9) > 0.05, "borderline input"
        assert abs(gm["evr"] - om.evr) <= EVR_TOL[prec] * om.evr, om.t
        assert gm["r"] == om.r, om.t
        assert kg == ko, om.t
        ks.append(ko)
    assert ks[0] == 4 and ks[-1] == 10 and o.r == 10     # grew one step per check, then capped
    _check_end(g, o, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_combined_error_and_angle_policy_matches_oracle(isvd, prec):
    """The 2,000 x 1,000 workload's rules (ratio > 1.05 or angle > 5 degrees, k = 16 with 20
    factors) on the reduced panel: with k in the noise bulk the angle to the optimal subspace is
    large, so a refresh fires at every check the spacing allows."""
    t_min = 50
    A0, ev, k = _stream(5, 16, 300, f=20)
    pol = dict(kind=oracle.POLICY_ERROR | oracle.POLICY_ANGLE, check_every=25, gamma=1.05,
               theta_max=np.deg2rad(5.0), T_min=t_min)
    g, o, recs = _run_lockstep(isvd, prec, A0, ev, k, pol)
    t_last = 0
    for gm, om, kg, ko in recs:
        if om.t - t_last >= t_min:
            assert om.angle_to_opt > np.deg2rad(10.0) or om.angle_to_opt < np.deg2rad(2.5), "borderline input"
            assert gm["angle_to_opt"] > np.deg2rad(5.0)
        assert abs(gm["frob_ratio"] - om.frob_ratio) <= RATIO_TOL[prec] * om.frob_ratio, om.t
        assert (gm["t_last"] == gm["t"]) == om.refreshed, om.t
        if om.refreshed:
            t_last = om.t
    assert o.refreshes >= 4
    assert g.metrics(full=False)["refreshes"] == o.refreshes
    _check_end(g, o, prec)


def test_reorthogonalisation_fires_and_keeps_parity(isvd):
    """Loss-of-orthogonality monitor: with a tolerance below the FP32 level it fires at every
    cadence step; U and V come back orthonormal to FP32 accuracy, sigma is unchanged, and the
    stream still matches the oracle (which keeps exactly orthonormal factors)."""
    A0, ev, k = _stream(9, 12, 200)
    Ao = A0.astype(np.float32).astype(np.float64)
    factors = oracle.truncated_svd(Ao, k)
    g = isvd.ISVD(A0, k, prec=1, orth_tol=1e-9, orth_every=20, factors=factors)
    o = oracle.OracleISVD(Ao, k, tol_rel=3e-6, factors=factors)
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            g.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            v = ev.vector(e).astype(np.float32)
            (g.append_row if kd == streams.ROW else g.append_col)(v)
            (o.append_row if kd == streams.ROW else o.append_col)(v.astype(np.float64))
    mt = g.metrics(full=False)
    assert mt["reorths"] == len(ev) // 20
    s_before = g.sigma()
    eu, ev_ = g.reorthogonalize(force=True)
    assert eu < 1e-5 and ev_ < 1e-5
    U, s, V = g.factors()
    np.testing.assert_array_equal(s, s_before)
    for Q in (U, V):
        Q = Q.astype(np.float64)
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-6
    _check_end(g, o, 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_randomized_path_error_ratio_bounds_and_decisions(isvd, prec):
    """min(m, n) > 128 takes the randomized truncated SVD (oversampling 16, power iterations q).
    E_opt there is the residual of the computed rank-r factorisation, an upper bound of the
    optimum: at every check it lies between the oracle's exact E_opt and (1 + ACC) times it (the
    dense matrix, hence E_opt, is the same on both sides whatever the refreshes did). Refresh
    decisions agree with the oracle's up to the first refresh (after it the GPU continues from
    a randomized factorisation, the oracle from the exact one) wherever the oracle's ratio is
    farther than ACC from gamma."""
    A0, fm = streams.make_panel(400, 160, 10, seed=13)
    ev = streams.make_events(fm, 400, 300, mix=(0.7, 0.1, 0.2), seed=14)
    k, gamma = 16, RSVD_GAMMA
    dt = np.float32 if prec == 1 else np.float64
    Ao = A0.astype(dt).astype(np.float64)
    factors = oracle.truncated_svd(Ao, k)
    pol = oracle.Policy(kind=oracle.POLICY_ERROR, check_every=50, gamma=gamma)
    o = oracle.OracleISVD(Ao, k, tol_rel=1e-10 if prec == 0 else 3e-6, policy=pol, factors=factors)
    g = isvd.ISVD(A0, k, prec=prec, factors=factors, rsvd_power_iters=RSVD_Q)
    g.set_policy(kind=isvd.POLICY_ERROR, check_every=50, gamma=gamma)
    decided, same_path = 0, True
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            g.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            v = ev.vector(e).astype(dt)
            (g.append_row if kd == streams.ROW else g.append_col)(v)
            (o.append_row if kd == streams.ROW else o.append_col)(v.astype(np.float64))
        if (e + 1) % 50 == 0:
            gm, om = g.last_check_metrics(), o.log[-1]
            assert gm["frob_opt"] >= om.frob_opt * (1 - 1e-5), om.t
            assert gm["frob_opt"] <= om.frob_opt * (1 + RSVD_ACC), (om.t, gm["frob_opt"] / om.frob_opt - 1)
            if same_path:
                assert abs(gm["frob_error"] - om.frob_error) <= 1e-4 * om.frob_error, om.t
                if abs(om.frob_ratio - gamma) > 2 * RSVD_ACC * gamma:
                    assert (gm["t_last"] == gm["t"]) == om.refreshed, om.t
                    decided += 1
                same_path = not (om.refreshed or gm["t_last"] == gm["t"])
    assert decided >= 2 and o.refreshes >= 1
