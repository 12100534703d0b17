"""Deferred rotations (isvd_set_deferred_rotations: U = U0 R_U, V = V0 R_V for the rank-1 entry
updates of Section 2.3) on the GPU against the oracle, through the C ABI.

The oracle applies every entry update to U and V directly (Algorithm A3); the deferred form only
reorders the products, so the results must agree within the same tolerances as the plain form:
at the end of every run of entry updates (the fold happens inside the read), after each kind of
call that folds (append, rank-increasing entry, metrics, refresh, re-orthogonalisation, risk,
turning the mode off), under a periodic policy, and on a tall FP32 stream where the deferred
entry update launches two kernels and never touches U or V."""
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


def recon(U, s, V):
    return (U.astype(np.float64) * s) @ V.astype(np.float64).T


def check_against(g, o, prec, where):
    U, s, V = g.factors()
    assert not g.deferred_pending, where
    assert s.size == o.r, where
    Ro = o.reconstruction()
    nrm = np.linalg.norm(Ro)
    assert np.linalg.norm(recon(U, s, V) - Ro) <= TOL[prec] * nrm, where
    np.testing.assert_allclose(s, o.s, rtol=0, atol=TOL[prec] * o.s[0], err_msg=where)
    for Q in (U, V):
        G = Q.astype(np.float64).T @ Q.astype(np.float64)
        assert np.abs(G - np.eye(G.shape[0])).max() <= (1e-12 if prec == 0 else 2e-5), where


def entry_runs(m0, n0, f, seed, runs, run_len, appends=2):
    """Blocks of ``run_len`` entry updates, each followed by ``appends`` row appends and one column
    append: the shape grows while the entry positions cover the whole matrix."""
    A0, fm = streams.make_panel(m0, n0, f, seed=seed)
    rng = np.random.default_rng(seed + 1)
    m, n = m0, n0
    ev = []
    for _ in range(runs):
        for _ in range(run_len):
            ev.append(("e", int(rng.integers(0, m)), int(rng.integers(0, n)), 0.05 * rng.standard_normal()))
        for _ in range(appends):
            ev.append(("r", fm.rows(1)[0]))
            m += 1
        ev.append(("c", fm.new_asset()))
        n += 1
    return A0, ev


@pytest.mark.parametrize("prec", [0, 1])
def test_deferred_entry_runs_match_oracle(isvd, prec):
    dt = np.float64 if prec == 0 else np.float32
    A0, ev = entry_runs(160, 60, 6, seed=71, runs=4, run_len=30)
    A0 = A0.astype(dt)
    tol_rel = 1e-10 if prec == 0 else 3e-6
    o = oracle.OracleISVD(A0.astype(np.float64), 10, tol_rel=tol_rel)
    g = isvd.ISVD(A0, 10, k_max=16, prec=prec)
    g.set_deferred_rotations(True)
    for e, item in enumerate(ev):
        if item[0] == "e":
            o.update_entry(item[1], item[2], item[3])
            g.update_entry(item[1], item[2], item[3])
            assert g.deferred_pending
            if e + 1 < len(ev) and ev[e + 1][0] != "e":
                check_against(g, o, prec, f"end of the entry run at event {e}")
        else:
            v = item[1].astype(dt)
            if item[0] == "r":
                o.append_row(v.astype(np.float64))
                g.append_row(v)
            else:
                o.append_col(v.astype(np.float64))
                g.append_col(v)
            assert not g.deferred_pending
    check_against(g, o, prec, "end")
    np.testing.assert_allclose(g.matrix(), o.A_view(), rtol=0, atol=1e-12 if prec == 0 else 1e-6)
    assert abs(g.metrics(full=False)["N"] - o.N) <= 1e-9 * o.N


@pytest.mark.parametrize("prec", [0, 1])
def test_every_reader_folds_first(isvd, prec):
    """After a run of entry updates, each call that reads U or V folds R_U, R_V in first."""
    dt = np.float64 if prec == 0 else np.float32
    A0, fm = streams.make_panel(140, 50, 5, seed=73)
    A0 = A0.astype(dt)
    tol_rel = 1e-10 if prec == 0 else 3e-6
    o = oracle.OracleISVD(A0.astype(np.float64), 8, tol_rel=tol_rel)
    g = isvd.ISVD(A0, 8, k_max=16, prec=prec)
    g.set_deferred_rotations(True)
    rng = np.random.default_rng(74)

    def run(count=12):
        for _ in range(count):
            i, j, d = int(rng.integers(0, o.m)), int(rng.integers(0, o.n)), 0.05 * rng.standard_normal()
            o.update_entry(i, j, d)
            g.update_entry(i, j, d)
        assert g.deferred_pending

    run()
    mt = g.metrics(full=True)                      # metrics read U, V (E_inc, angles)
    assert not g.deferred_pending
    omt = o.metrics()
    assert abs(mt["frob_error"] - omt.frob_error) <= 1e-6 * max(omt.frob_error, 1e-300) + TOL[prec] * np.sqrt(o.N)
    check_against(g, o, prec, "after metrics")

    run()
    g.reorthogonalize(force=True)                  # re-orthogonalisation of U, V (sigma unchanged)
    assert not g.deferred_pending
    check_against(g, o, prec, "after reorthogonalize")

    run()
    g.risk()
    assert not g.deferred_pending

    run()
    i, j, d = int(rng.integers(0, o.m)), int(rng.integers(0, o.n)), 0.05
    o.update_entry_exact(i, j, d)                  # the rank-increasing form reads U, V rows
    g.update_entry_exact(i, j, d)
    assert not g.deferred_pending
    check_against(g, o, prec, "after the rank-increasing entry update")

    run()
    g.set_deferred_rotations(False)                # turning the mode off folds
    assert not g.deferred_pending
    check_against(g, o, prec, "after turning the mode off")
    i, j, d = 3, 4, 0.02
    o.update_entry(i, j, d)
    g.update_entry(i, j, d)
    assert not g.deferred_pending                  # the plain form again

    g.set_deferred_rotations(True)
    run()
    o.refresh()                                    # refresh: the truncated SVD of A_t (warm start reads V)
    g.refresh()
    assert not g.deferred_pending
    check_against(g, o, prec, "after refresh")


def test_deferred_periodic_policy_matches_oracle(isvd):
    """A periodic refresh inside a run of entry updates (the policy step folds before it refreshes)."""
    A0, fm = streams.make_panel(120, 45, 5, seed=75)
    o = oracle.OracleISVD(A0, 8, tol_rel=1e-10, policy=oracle.Policy(kind=oracle.POLICY_PERIODIC, T_refresh=25))
    g = isvd.ISVD(A0, 8, k_max=16, prec=0)
    g.set_policy(kind=isvd.POLICY_PERIODIC, T_refresh=25)
    g.set_deferred_rotations(True)
    rng = np.random.default_rng(76)
    for t in range(1, 81):
        i, j, d = int(rng.integers(0, o.m)), int(rng.integers(0, o.n)), 0.05 * rng.standard_normal()
        o.update_entry(i, j, d)
        g.update_entry(i, j, d)
        assert g.deferred_pending == (t % 25 != 0), t
    check_against(g, o, 0, "periodic")
    assert g.metrics(full=False)["refreshes"] == 3


def test_tall_fp32_entry_updates_touch_only_the_small_factors(isvd):
    """A tall FP32 stream (12,000 x 300, k = 48): 150 deferred entry updates, two launches each
    (core, R product) after the first; U, V unchanged in memory until the fold; the folded result
    matches the oracle and the plain form."""
    A0, fm = streams.make_panel(12000, 300, 10, seed=77)
    A0 = A0.astype(np.float32)
    o = oracle.OracleISVD(A0.astype(np.float64), 48, tol_rel=3e-6)
    # both handles start from the oracle's truncated SVD of A0 (the device's own start at this
    # shape is the randomized one)
    f0 = (o.U.astype(np.float32), o.s.copy(), o.V.astype(np.float32))
    g = isvd.ISVD(A0, 48, k_max=64, prec=1, orth_every=10 ** 9, factors=f0)
    p = isvd.ISVD(A0, 48, k_max=64, prec=1, orth_every=10 ** 9, factors=f0)
    g.set_deferred_rotations(True)
    rng = np.random.default_rng(78)
    upd = [(int(rng.integers(0, 12000)), int(rng.integers(0, 300)), 0.05 * rng.standard_normal()) for _ in range(150)]
    g.update_entry(*upd[0])
    l0 = g.launches
    for u in upd[1:]:
        g.update_entry(*u)
    assert g.launches - l0 == 2 * (len(upd) - 1)
    for u in upd:
        o.update_entry(*u)
        p.update_entry(*u)
    Ug, sg, Vg = g.factors()
    Up, sp, Vp = p.factors()
    np.testing.assert_allclose(sg, sp, rtol=0, atol=1e-5 * sp[0])
    rows = rng.choice(12000, 400, replace=False)
    Rg = recon(Ug[rows], sg, Vg)
    Ro = (o.U[rows] * o.s) @ o.V.T
    assert np.linalg.norm(Rg - Ro) <= 1e-5 * np.linalg.norm(Ro)
    np.testing.assert_allclose(sg, o.s, rtol=0, atol=1e-5 * o.s[0])
    G = Ug.astype(np.float64).T @ Ug.astype(np.float64)
    assert np.abs(G - np.eye(48)).max() <= 2e-5


def test_deferred_mode_arguments(isvd):
    A0, _ = streams.make_panel(40, 20, 3, seed=79)
    g = isvd.ISVD(A0, 4, k_max=8, prec=0)
    assert isvd.lib().isvd_set_deferred_rotations(g._h, 2) == 1        # EINVAL: enable outside {0, 1}
    assert isvd.lib().isvd_set_deferred_rotations(None, 1) == 1
    g.set_deferred_rotations(False)                                      # off while off: nothing to fold
    assert not g.deferred_pending
    pool = isvd.Pool(k_max=8)
    sid = pool.admit(A0.astype(np.float32), 4)
    h = isvd.lib().isvd_pool_stream(pool._p, sid)
    assert isvd.lib().isvd_set_deferred_rotations(h, 1) == 1            # pool streams: EINVAL
