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
