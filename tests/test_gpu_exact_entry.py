"""The rank-increasing entry update (isvd_update_entry_exact: Section 2.3's A + delta e_i e_j^T in
Brand's general form) on the GPU against the oracle, through the C ABI: every step of a mixed
stream (row appends and exact entry updates) in both precisions, from a start below the working
rank so that the entry updates also grow the rank, and the successive-subspace angles."""
import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}
ANG_TOL = {0: 5e-7, 1: 2e-4}


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


def recon(U, s, V):
    return (U.astype(np.float64) * s) @ V.astype(np.float64).T


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_entry_updates_match_oracle(isvd, prec):
    dt = np.float64 if prec == 0 else np.float32
    A0, fm = streams.make_panel(120, 40, 6, seed=41)
    ev = streams.make_events(fm, 120, 60, mix=(0.5, 0.0, 0.5), seed=42, delta_sd=0.05)
    A0 = A0.astype(dt)
    # start at rank 4; the adaptive rule with an unreachable EVR target raises k by one per update
    # up to 8, so the updates (exact entries included) can grow the rank
    tol_rel = 1e-10 if prec == 0 else 3e-6
    pol = oracle.Policy(kind=oracle.POLICY_ADAPTIVE_RANK, check_every=1, tau_evr=1.01, k_max=8)
    o = oracle.OracleISVD(A0.astype(np.float64), 4, tol_rel=tol_rel, policy=pol)
    g = isvd.ISVD(A0, 4, k_max=16, prec=prec)
    g.set_policy(kind=isvd.POLICY_ADAPTIVE_RANK, check_every=1, tau_evr=1.01, k_max=8)
    ranks = []
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            o.update_entry_exact(ev.i[e], ev.j[e], ev.delta[e])
            g.update_entry_exact(int(ev.i[e]), int(ev.j[e]), float(ev.delta[e]))
        else:
            v = ev.vector(e).astype(dt)
            o.apply(kd, v.astype(np.float64))
            g.append_row(v)
        mt = g.metrics(full=False)
        assert mt["r"] == o.r, e
        U, s, V = g.factors()
        Ro = o.reconstruction()
        nrm = np.linalg.norm(Ro)
        assert np.linalg.norm(recon(U, s, V) - Ro) <= TOL[prec] * nrm, e
        np.testing.assert_allclose(s, o.s, rtol=0, atol=TOL[prec] * o.s[0])
        assert abs(mt["angle_succ_u"] - o.angle_succ_u) <= ANG_TOL[prec], e
        assert abs(mt["angle_succ_v"] - o.angle_succ_v) <= ANG_TOL[prec], e
        ranks.append(o.r)
    assert ranks[:4] == [4, 5, 6, 7] and max(ranks) == 8  # events 3 and 4 (exact entries) each grow the rank
    A = g.matrix()
    np.testing.assert_allclose(A, o.A_view(), rtol=0, atol=1e-12 if prec == 0 else 1e-6)
    assert abs(g.metrics(full=False)["N"] - o.N) <= 1e-9 * o.N
