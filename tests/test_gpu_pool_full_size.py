"""The batched workload at its full size, in the launch configuration the bench times: 4,096
independent factor-model streams (n ~ U[50, 500] assets, m0 = 2n rows, 5 factors, k drawn from
{8, 16, 32}) in one pool, one row append per stream per tick. A sample of streams (every rank
bucket, the narrowest and the widest panel) is checked one by one against the oracle started from
the same factors; the rest are admitted with the pool's own truncated SVD, as in the bench."""
import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu

S = 4096
TICKS = 3
KS = (8, 16, 32)


def _panel(job):
    """Stream sidx's initial panel (FP32) and its next TICKS rows, seeded per stream."""
    sidx, n = job
    A0, fm = streams.make_panel(2 * n, n, 5, seed=7_000_003 + sidx)
    return A0.astype(np.float32), fm.rows(TICKS).astype(np.float32)


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


def test_pool_full_size_sampled_against_oracle(isvd):
    rng = np.random.Generator(np.random.PCG64(11))
    ns = rng.integers(50, 501, size=S)
    ks = rng.choice(np.asarray(KS), size=S)
    sample = set()
    for kb in KS:
        sample |= set(np.flatnonzero(ks == kb)[:4].tolist())
    sample |= {int(np.argmin(ns)), int(np.argmax(ns))}
    pool = isvd.Pool(k_max=max(KS))
    ids, rows, start = [], [], {}
    for sidx in range(S):
        n = int(ns[sidx])
        A0, x = _panel((sidx, n))
        f = None
        if sidx in sample:
            f = oracle.truncated_svd(A0.astype(np.float64), int(ks[sidx]))
            start[sidx] = (A0, f)
        ids.append(pool.admit(A0, int(ks[sidx]), row_cap=2 * n + TICKS + 8, col_cap=n + 2, factors=f))
        rows.append(x)
    offs = np.concatenate([[0], np.cumsum(ns)[:-1]])
    l0 = pool.launches
    for t in range(TICKS):
        ops = [(ids[s], streams.ROW, 0, 0, 0.0, int(offs[s]), int(ns[s])) for s in range(S)]
        pool.submit(ops, np.concatenate([rows[s][t] for s in range(S)]))
    pool.sync()
    # per tick and rank bucket a warp, a rotation and a hand-back launch (and the monitor), plus
    # the sync's status gather, whatever the number of streams
    assert pool.launches - l0 <= TICKS * (3 * 3 + 1) + 1
    for sidx in sorted(sample):
        A0, f = start[sidx]
        k = int(ks[sidx])
        o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
        for t in range(TICKS):
            o.apply(streams.ROW, rows[sidx][t].astype(np.float64))
        U, s, V = pool.stream(ids[sidx]).factors()
        assert s.size == o.r, sidx
        Ro = o.reconstruction()
        R = (U.astype(np.float64) * s) @ V.astype(np.float64).T
        assert np.linalg.norm(R - Ro) <= 1e-5 * np.linalg.norm(Ro), sidx
        np.testing.assert_allclose(s, o.s, rtol=0, atol=1e-5 * o.s[0])
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(s.size)).max() < 1e-4, sidx
        assert np.abs(V.T.astype(np.float64) @ V - np.eye(s.size)).max() < 1e-4, sidx
        np.testing.assert_allclose(pool.stream(ids[sidx]).matrix(), o.A_view(), rtol=0, atol=1e-6)
    pool.close()
