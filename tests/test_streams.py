"""The seeded stream generator (no GPU)."""
import numpy as np

from paper_2605_24514_gb300 import streams


def test_slices_rebase_payload_offsets():
    A0, ev, k, _ = streams.workload("tiny", seed=2, n_events=50)
    for a in range(0, 50, 7):
        sl = ev.slice(a, min(a + 9, 50))
        for e in range(len(sl)):
            if sl.kind[e] != streams.ENTRY:
                np.testing.assert_array_equal(sl.vector(e), ev.vector(a + e))
            assert 0 <= sl.off[e] <= sl.payload.size


def test_shapes_track_events():
    A0, ev, k, _ = streams.workload("tiny", seed=3, n_events=40)
    m, n = A0.shape
    for e in range(len(ev)):
        if ev.kind[e] == streams.ROW:
            assert ev.length[e] == n
            m += 1
        elif ev.kind[e] == streams.COL:
            assert ev.length[e] == m
            n += 1
        else:
            assert 0 <= ev.i[e] < m and 0 <= ev.j[e] < n
        assert (ev.m_after[e], ev.n_after[e]) == (m, n)


def test_seeded_reproducible():
    a = streams.workload("tiny", seed=5)[1]
    b = streams.workload("tiny", seed=5)[1]
    np.testing.assert_array_equal(a.payload, b.payload)
    np.testing.assert_array_equal(a.kind, b.kind)


def test_factor_model_follows_the_stated_recipe():
    """Generator recipe: factor j has volatility 0.02 * 0.7**j, loadings are N(0, 1/f), the
    idiosyncratic term is 0.01 times a unit-scale Student-t with 4 degrees of freedom (pinned by its
    median absolute value, the t4 distribution's 0.75 quantile, 0.74070), and entry deltas have
    standard deviation 0.005."""
    f = 5
    fm = streams.FactorModel(n=2000, f=f, seed=1)
    X = fm.rows(4000)
    F = fm.F[:4000]
    vol = F.std(axis=0) / (0.02 * 0.7 ** np.arange(f))
    assert np.all(np.abs(vol - 1.0) < 0.05), vol
    assert abs(fm.B.var() * f - 1.0) < 0.03
    E = X - F @ fm.B.T
    assert abs(np.median(np.abs(E)) / 0.01 - 0.740697) < 0.005
    fm2 = streams.FactorModel(n=50, f=f, seed=2)
    ev = streams.make_events(fm2, 100, 20000, mix=(0.0, 0.0, 1.0), seed=3)
    d = ev.delta[ev.kind == streams.ENTRY]
    assert d.size == 20000 and abs(d.std() / 0.005 - 1.0) < 0.03
