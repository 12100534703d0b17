"""The 2,000 x 1,000 panel workload (20 factors, k = 64, FP32 bulk, 70% row appends / 10% column
appends / 20% entry updates, delta sd 0.005) at its full size against the oracle, through the C
ABI, in the plain form and with deferred rotations.

Both engines start from the oracle's truncated SVD of A0 (at this shape the device's own start is
the randomized one, whose noise-subspace columns differ from the exact ones), then take the same
600 events. The refresh policies are left out here: at this shape the device refreshes through
the randomized SVD, so a refresh would end the lockstep; their decisions are compared against the
oracle's on the reduced panel (tests/test_gpu_policies.py)."""
import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


@pytest.mark.parametrize("deferred", [False, True])
def test_panel_2000x1000_k64_against_oracle(isvd, deferred):
    A0, ev, k, _ = streams.workload("panel-2000x1000-k64", seed=3, n_events=600)
    A0 = A0.astype(np.float32)
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6)
    g = isvd.ISVD(A0, k, prec=isvd.FP32, k_max=k, factors=(o.U.astype(np.float32), o.s.copy(),
                                                          o.V.astype(np.float32)))
    if deferred:
        g.set_deferred_rotations(True)
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            g.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            v = ev.vector(e).astype(np.float32)
            (g.append_row if kd == streams.ROW else g.append_col)(v)
            (o.append_row if kd == streams.ROW else o.append_col)(v.astype(np.float64))
    m, n, r, _ = g.shape()
    assert (m, n, r) == (o.m, o.n, o.r) == (int(ev.m_after[-1]), int(ev.n_after[-1]), k)
    U, s, V = g.factors()
    np.testing.assert_allclose(s, o.s, rtol=0, atol=1e-5 * o.s[0])
    Ro = o.reconstruction()
    assert np.linalg.norm((U.astype(np.float64) * s) @ V.astype(np.float64).T - Ro) <= 1e-5 * np.linalg.norm(Ro)
    for Q in (U, V):
        G = Q.astype(np.float64).T @ Q.astype(np.float64)
        assert np.abs(G - np.eye(k)).max() <= 5e-5
    np.testing.assert_allclose(g.matrix(), o.A_view(), rtol=0, atol=1e-6)
    assert abs(g.metrics(full=False)["N"] - o.N) <= 1e-9 * o.N
