"""GPU (libisvd) vs CPU oracle parity on identical seeded inputs, through the C ABI.

FP64 path: singular values and reconstruction within relative 1e-10 of the oracle; the stored
matrix and N_t match to rounding. FP32-bulk path: within relative 1e-5 (sigma relative to
sigma_1, reconstruction relative to ||A_hat||_F). Comparisons are sign-free (sigma and
U S V^T), so the sign and order freedom of singular vectors does not matter.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def recon(U, s, V):
    return (U.astype(np.float64) * s) @ V.astype(np.float64).T


def compare(g, o, prec, ctx=""):
    U, s, V = g.factors()
    tol = TOL[prec]
    assert s.size == o.r, f"{ctx}: rank {s.size} vs {o.r}"
    np.testing.assert_allclose(s, o.s, rtol=0, atol=tol * max(o.s[0], 1e-300), err_msg=ctx)
    Ro = o.reconstruction()
    err = np.linalg.norm(recon(U, s, V) - Ro) / max(np.linalg.norm(Ro), 1e-300)
    assert err <= tol, f"{ctx}: reconstruction rel err {err:.3e}"
    oe = 10 * tol if prec == 0 else 1e-4
    assert np.abs(U.T.astype(np.float64) @ U - np.eye(U.shape[1])).max() < oe, ctx
    assert np.abs(V.T.astype(np.float64) @ V - np.eye(V.shape[1])).max() < oe, ctx


def run_pair(pkg, A0, ev, k, prec, policy=None, shared_start=None, **kw):
    """GPU engine and oracle on the same A0. For min(m, n) > 128 (where the GPU's own initial
    truncated SVD is the randomized one) both start from the oracle's exact factors."""
    tol_rel = 1e-10 if prec == 0 else 3e-6
    Ao = A0.astype(np.float32).astype(np.float64) if prec == 1 else A0
    if shared_start is None:
        shared_start = min(A0.shape) > 128
    factors = oracle.truncated_svd(Ao, k) if shared_start else None
    g = pkg.ISVD(A0, k, prec=prec, factors=factors, **kw)
    o = oracle.OracleISVD(Ao, k, tol_rel=tol_rel, policy=policy, factors=factors)
    return g, o


def feed(g, o, ev, e, prec):
    kd = int(ev.kind[e])
    if kd == streams.ENTRY:
        g.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
    else:
        v = ev.vector(e)
        if prec == 1:
            v = v.astype(np.float32)
        (g.append_row if kd == streams.ROW else g.append_col)(v)
        (o.append_row if kd == streams.ROW else o.append_col)(v.astype(np.float64))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_mixed_stream_every_step(isvd, prec, seed):
    A0, ev, k, _ = streams.workload("tiny", seed=seed, n_events=60)
    g, o = run_pair(isvd, A0, ev, k, prec)
    compare(g, o, prec, "create")
    for e in range(len(ev)):
        feed(g, o, ev, e, prec)
        compare(g, o, prec, f"event {e} kind {ev.kind[e]}")
    A = g.matrix().astype(np.float64)
    np.testing.assert_allclose(A, o.A_view(), rtol=0, atol=1e-12 if prec == 0 else 1e-6)
    mt = g.metrics(full=False)
    assert abs(mt["N"] - o.N) <= (1e-12 if prec == 0 else 1e-6) * o.N


def test_fp64_panel_200x50_k10_periodic_with_metrics(isvd):
    """The 200x50, k=10 FP64 workload: 1,000 row appends then 200 entry updates, periodic refresh
    every 250, metrics every 50, compared at every check."""
    A0, ev, k, _ = streams.workload("panel-200x50-k10", seed=0)
    pol = oracle.Policy(kind=oracle.POLICY_PERIODIC, T_refresh=250, check_every=50)
    g = isvd.ISVD(A0, k, prec=0)
    g.set_policy(kind=isvd.POLICY_PERIODIC, T_refresh=250, check_every=50)
    o = oracle.OracleISVD(A0, k, tol_rel=1e-10, policy=pol)
    logs = []
    for e in range(len(ev)):
        feed(g, o, ev, e, 0)
        if (e + 1) % 50 == 0:
            gm = g.last_check_metrics()
            om = o.log[-1]
            assert gm["t"] == om.t == e + 1
            for key in ["frob_error", "frob_opt", "evr"]:
                assert abs(gm[key] - getattr(om, key)) <= 1e-9 * abs(getattr(om, key)), (e, key)
            assert abs(gm["frob_ratio"] - om.frob_ratio) <= 1e-9 * om.frob_ratio
            assert abs(gm["angle_to_opt"] - om.angle_to_opt) <= 1e-6
            assert abs(gm["angle"] - om.angle) <= 1e-6
            logs.append(gm["frob_ratio"])
        if (e + 1) % 100 == 0:
            compare(g, o, 0, f"event {e}")
    compare(g, o, 0, "end")
    assert g.metrics(full=False)["refreshes"] == o.refreshes == 4
    assert min(logs) >= 1 - 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_medium_multi_tile(isvd, prec):
    """n and m span several projection blocks and rotation tiles, with ragged tails."""
    A0, fm = streams.make_panel(333, 150, 8, seed=7)
    ev = streams.make_events(fm, 333, 120, mix=(0.5, 0.2, 0.3), seed=8)
    g, o = run_pair(isvd, A0, ev, 24, prec)
    for e in range(len(ev)):
        feed(g, o, ev, e, prec)
        if e % 20 == 19:
            compare(g, o, prec, f"event {e}")
    compare(g, o, prec, "end")


@pytest.mark.parametrize("prec", [0, 1])
def test_rank_deficient_start_grows_rank(isvd, prec):
    g0 = rng(3)
    A0 = g0.standard_normal((20, 2)) @ g0.standard_normal((2, 9))      # exact rank 2, k = 6
    g, o = run_pair(isvd, A0, None, 6, prec)
    for step in range(8):
        x = g0.standard_normal(9)
        if prec == 1:
            x = x.astype(np.float32)
        g.append_row(x)
        o.append_row(x.astype(np.float64))
        U, s, V = g.factors()
        assert s.size == o.r
        Ro = o.reconstruction()
        assert np.linalg.norm(recon(U, s, V) - Ro) <= TOL[prec] * 10 * np.linalg.norm(Ro)
    assert o.r == 6


@pytest.mark.parametrize("prec", [0, 1])
def test_in_span_and_zero_rows_keep_rank(isvd, prec):
    A0, fm = streams.make_panel(40, 12, 3, seed=11)
    g, o = run_pair(isvd, A0, None, 4, prec)
    U, s, V = g.factors()
    r0 = s.size
    for x in [V.astype(np.float64) @ np.array([1.0, -2.0, 0.5, 0.25]), np.zeros(12)]:
        if prec == 1:
            x = x.astype(np.float32)
        g.append_row(x)
        o.append_row(x.astype(np.float64))
        mt = g.metrics(full=False)
        assert mt["r"] == r0
        assert mt["rho_last"] <= (1e-12 if prec == 0 else 1e-5) * max(np.linalg.norm(x), 1.0)
        compare(g, o, prec, "in-span")


def test_untruncated_square_entry_updates_equal_full_svd(isvd):
    g0 = rng(5)
    A0 = g0.standard_normal((7, 7))
    g = isvd.ISVD(A0, 7, prec=0)
    A = A0.copy()
    for _ in range(12):
        i, j, d = int(g0.integers(7)), int(g0.integers(7)), float(g0.standard_normal())
        g.update_entry(i, j, d)
        A[i, j] += d
        U, s, V = g.factors()
        np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-11)
        assert np.linalg.norm(recon(U, s, V) - A) <= 1e-11 * np.linalg.norm(A)


@pytest.mark.parametrize("prec", [0, 1])
def test_refresh_equals_truncated_svd(isvd, prec):
    A0, fm = streams.make_panel(90, 60, 6, seed=21)
    ev = streams.make_events(fm, 90, 40, mix=(0.6, 0.2, 0.2), seed=22)
    g, o = run_pair(isvd, A0, ev, 8, prec)
    for e in range(len(ev)):
        feed(g, o, ev, e, prec)
    g.refresh()
    o.refresh()
    compare(g, o, prec, "refresh")
    mt = g.metrics(full=True)
    assert abs(mt["frob_ratio"] - 1.0) < (1e-9 if prec == 0 else 1e-4)
    assert mt["angle_to_opt"] < (1e-6 if prec == 0 else 2e-3)


@pytest.mark.parametrize("prec", [0, 1])
def test_wide_matrix_refresh_path(isvd, prec):
    g0 = rng(31)
    A0 = g0.standard_normal((30, 200))
    g = isvd.ISVD(A0, 5, prec=prec)
    o = oracle.OracleISVD(A0.astype(np.float32).astype(np.float64) if prec else A0, 5)
    compare(g, o, prec, "wide create")


def test_metrics_match_oracle_fp32(isvd):
    A0, fm = streams.make_panel(120, 40, 4, seed=41)
    ev = streams.make_events(fm, 120, 80, mix=(0.7, 0.1, 0.2), seed=42)
    g, o = run_pair(isvd, A0, ev, 6, 1)
    for e in range(len(ev)):
        feed(g, o, ev, e, 1)
    gm, om = g.metrics(full=True), o.metrics()
    assert abs(gm["frob_ratio"] - om.frob_ratio) <= 1e-4 * om.frob_ratio
    assert abs(gm["frob_error"] - om.frob_error) <= 1e-4 * om.frob_error
    assert abs(gm["evr"] - om.evr) <= 1e-5 * om.evr
    assert abs(gm["angle_to_opt"] - om.angle_to_opt) <= 1e-3
    assert abs(gm["angle"] - om.angle) <= 1e-3


def test_errors_leave_state_unchanged(isvd):
    A0, fm = streams.make_panel(30, 10, 3, seed=51)
    g = isvd.ISVD(A0, 4, prec=0)
    U0, s0, V0 = g.factors()
    with pytest.raises(isvd.IsvdError) as e:
        g.append_row(np.ones(11))
    assert e.value.name == "ESHAPE"
    with pytest.raises(isvd.IsvdError) as e:
        g.update_entry(30, 0, 1.0)
    assert e.value.name == "EBOUNDS"
    with pytest.raises(isvd.IsvdError) as e:
        g.append_row(np.array([np.nan] + [0.0] * 9))
    assert e.value.name == "ENONFINITE"
    U1, s1, V1 = g.factors()
    assert np.array_equal(s0, s1) and np.array_equal(U0, U1) and g.shape()[:2] == (30, 10)


def test_device_inputs_match_host_inputs(isvd):
    torch = pytest.importorskip("torch")
    A0, fm = streams.make_panel(64, 20, 3, seed=61)
    ev = streams.make_events(fm, 64, 30, mix=(0.6, 0.2, 0.2), seed=62)
    g1 = isvd.ISVD(A0, 5, prec=0)
    g2 = isvd.ISVD(torch.tensor(A0, device="cuda"), 5, prec=0)
    g1.apply_events(ev)
    g2.apply_events(ev, payload=torch.tensor(ev.payload, device="cuda"))
    U1, s1, V1 = g1.factors()
    U2, s2, V2 = g2.factors()
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(U1, U2)


def test_apply_events_matches_single_calls(isvd):
    A0, ev, k, _ = streams.workload("tiny", seed=3, n_events=30)
    g1 = isvd.ISVD(A0, k, prec=1)
    g2 = isvd.ISVD(A0, k, prec=1)
    g1.apply_events(ev)
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            g2.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            (g2.append_row if kd == streams.ROW else g2.append_col)(ev.vector(e))
    U1, s1, V1 = g1.factors()
    U2, s2, V2 = g2.factors()
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(V1, V2)


@pytest.mark.parametrize("prec", [0, 1])
def test_randomized_refresh_matches_exact_with_spectral_gap(isvd, prec):
    """min(m, n) > 128 takes the randomized refresh; with a clear gap after k its factors
    agree with the exact truncated SVD."""
    g0 = rng(71)
    m, n, k = 400, 260, 8
    A0 = (g0.standard_normal((m, k)) * np.linspace(10, 3, k)) @ np.linalg.qr(g0.standard_normal((n, k)))[0].T
    A0 = A0 + 1e-6 * g0.standard_normal((m, n))
    g = isvd.ISVD(A0, k, prec=prec)
    Ao = A0.astype(np.float32).astype(np.float64) if prec else A0
    Ue, se, Ve = oracle.truncated_svd(Ao, k)
    U, s, V = g.factors()
    tol = 1e-9 if prec == 0 else 2e-5
    np.testing.assert_allclose(s, se, rtol=tol)
    assert np.linalg.norm(recon(U, s, V) - (Ue * se) @ Ve.T) <= tol * np.linalg.norm(se)


@pytest.mark.parametrize("prec", [0, 1])
def test_randomized_metrics_on_factor_panel(isvd, prec):
    """Noise-bulk spectrum (factor model): the randomized E_opt is within 1% of the exact one."""
    A0, fm = streams.make_panel(600, 300, 10, seed=81)
    ev = streams.make_events(fm, 600, 60, mix=(0.7, 0.1, 0.2), seed=82)
    g, o = run_pair(isvd, A0, ev, 16, prec)
    for e in range(len(ev)):
        feed(g, o, ev, e, prec)
    gm, om = g.metrics(full=True), o.metrics()
    assert abs(gm["frob_opt"] - om.frob_opt) <= 1e-2 * om.frob_opt
    assert abs(gm["frob_error"] - om.frob_error) <= 1e-4 * om.frob_error
    assert abs(gm["frob_ratio"] - om.frob_ratio) <= 1e-2 * om.frob_ratio


def _spectrum_model(M, N, rank, seed):
    """A M x N matrix of exact rank ``rank`` with singular values 10 * 0.96^i (relative gaps of
    4%, so truncation picks the same directions on both sides), plus noise of 1e-7."""
    g = rng(seed)
    L, _ = np.linalg.qr(g.standard_normal((M, rank)))
    R, _ = np.linalg.qr(g.standard_normal((N, rank)))
    s = 10.0 * 0.96 ** np.arange(rank)
    return (L * s) @ R.T + 1e-7 * g.standard_normal((M, N))


@pytest.mark.parametrize("prec,k,k_max", [(1, 100, 128), (0, 90, 96)])
def test_largest_rank_buckets(isvd, prec, k, k_max):
    """Ranks above 64: the 128 bucket (FP32) and the FP64 ceiling of 96, with rows, columns and
    entries cut from one fixed matrix so that the stream stays consistent."""
    Af = _spectrum_model(260, 200, 120, seed=11)
    m, n = 150, 130
    A0 = Af[:m, :n].copy()
    g, o = run_pair(isvd, A0, None, k, prec, k_max=k_max, row_cap=260, col_cap=200)
    ev_rng = rng(12)
    for e in range(40):
        u = ev_rng.random()
        if u < 0.5:
            v = Af[m, :n]
            v = v.astype(np.float32) if prec == 1 else v
            g.append_row(v)
            o.append_row(v.astype(np.float64))
            m += 1
        elif u < 0.75:
            v = Af[:m, n]
            v = v.astype(np.float32) if prec == 1 else v
            g.append_col(v)
            o.append_col(v.astype(np.float64))
            n += 1
        else:
            i, j = int(ev_rng.integers(m)), int(ev_rng.integers(n))
            d = float(ev_rng.normal(0, 0.005))
            g.update_entry(i, j, d)
            o.update_entry(i, j, d)
        if e % 10 == 9:
            compare(g, o, prec, f"k={k} event {e}")
    assert g.shape()[:2] == (m, n)


def test_handles_with_different_k_max_share_kernels(isvd):
    """Handles whose k_max fall in one rank bucket (8 and 16) run the same kernel instantiation;
    creating the smaller one after the larger must not break the larger one's launches."""
    A0, fm = streams.make_panel(40, 30, 6, seed=21)
    ev = streams.make_events(fm, 40, 30, mix=(0.6, 0.2, 0.2), seed=22)
    ga, oa = run_pair(isvd, A0, ev, 12, 1, k_max=16)
    gb, ob = run_pair(isvd, A0, ev, 4, 1, k_max=8)
    for e in range(len(ev)):
        feed(ga, oa, ev, e, 1)
        feed(gb, ob, ev, e, 1)
    compare(ga, oa, 1, "k_max 16")
    compare(gb, ob, 1, "k_max 8")
