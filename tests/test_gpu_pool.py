"""Batched pool (fused per-tick launches) vs the oracle and vs the same stream run alone."""
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


def recon(U, s, V):
    return (U.astype(np.float64) * s) @ V.astype(np.float64).T


def make_streams(n_streams, seed, n_events=12, mix=(0.6, 0.2, 0.2), ks=(4, 8, 16, 32), nrange=(24, 160)):
    rng = np.random.default_rng(seed)
    out = []
    for sidx in range(n_streams):
        n = int(rng.integers(*nrange))
        k = int(rng.choice(ks))
        A0, fm = streams.make_panel(2 * n, n, 5, seed=seed * 1000 + sidx)
        ev = streams.make_events(fm, 2 * n, n_events, mix=mix, seed=seed * 1000 + sidx + 500)
        out.append((A0.astype(np.float32), ev, k))
    return out


def interleave(pool_ids, data):
    """One op list: per-stream order kept, streams interleaved (several ops per stream)."""
    ops, chunks, pos = [], [], 0
    cursors = [0] * len(data)
    remaining = sum(len(d[1]) for d in data)
    rng = np.random.default_rng(5)
    while remaining:
        s = int(rng.integers(len(data)))
        ev = data[s][1]
        e = cursors[s]
        if e >= len(ev):
            continue
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            ops.append((pool_ids[s], kd, int(ev.i[e]), int(ev.j[e]), float(ev.delta[e]), 0, 0))
        else:
            v = ev.vector(e).astype(np.float32)
            ops.append((pool_ids[s], kd, 0, 0, 0.0, pos, v.size))
            chunks.append(v)
            pos += v.size
        cursors[s] += 1
        remaining -= 1
    payload = np.concatenate(chunks) if chunks else np.zeros(1, np.float32)
    return ops, payload


def test_pool_matches_oracle_and_alone(isvd):
    data = make_streams(24, seed=3)
    pool = isvd.Pool(k_max=32)
    factors = [oracle.truncated_svd(A0.astype(np.float64), k) for A0, _, k in data]
    ids = [pool.admit(A0, k, factors=f) for (A0, _, k), f in zip(data, factors)]
    ops, payload = interleave(ids, data)
    pool.submit(ops, payload)
    pool.sync()
    for sidx, ((A0, ev, k), f) in enumerate(zip(data, factors)):
        # oracle
        o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
        for e in range(len(ev)):
            kd = int(ev.kind[e])
            if kd == streams.ENTRY:
                o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            else:
                o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
        # the same stream alone through the single-stream engine
        g = isvd.ISVD(A0, k, prec=isvd.FP32, k_max=32, factors=f)
        g.apply_events(ev)
        U, s, V = pool.stream(ids[sidx]).factors()
        Ua, sa, Va = g.factors()
        assert s.size == o.r == sa.size
        Ro = o.reconstruction()
        nrm = np.linalg.norm(Ro)
        assert np.linalg.norm(recon(U, s, V) - Ro) <= 1e-5 * nrm, sidx
        assert np.linalg.norm(recon(U, s, V) - recon(Ua, sa, Va)) <= 1e-5 * nrm, sidx
        np.testing.assert_allclose(s, o.s, rtol=0, atol=1e-5 * o.s[0])
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(s.size)).max() < 1e-4
        A = pool.stream(ids[sidx]).matrix()
        np.testing.assert_allclose(A, o.A_view(), rtol=0, atol=1e-6)
        g.close()
    assert pool.launches <= max(len(d[1]) for d in data) * 3
    pool.close()


def test_pool_admission_budget(isvd):
    pool = isvd.Pool(k_max=16, hbm_budget_bytes=30 * 2**20)
    A0, _ = streams.make_panel(200, 100, 4, seed=1)
    ids = []
    with pytest.raises(isvd.IsvdError) as e:
        for _ in range(100):
            ids.append(pool.admit(A0, 8))
    assert e.value.name == "EBUDGET"
    used = pool.bytes_used
    assert 0 < used <= 30 * 2**20 and len(ids) >= 1
    pool.release(ids[0])
    assert pool.bytes_used < used
    ids[0] = pool.admit(A0, 8)          # memory freed -> admitted again
    pool.close()


def test_pool_rejects_bad_ops_without_side_effects(isvd):
    pool = isvd.Pool(k_max=16)
    A0, _ = streams.make_panel(40, 20, 3, seed=2)
    sid = pool.admit(A0, 6)
    U0, s0, V0 = pool.stream(sid).factors()
    with pytest.raises(isvd.IsvdError) as e:
        pool.submit([(sid, 2, 0, 0, 0.1, 0, 0), (sid, 0, 0, 0, 0.0, 0, 21)], np.zeros(21, np.float32))
    assert e.value.name == "ESHAPE"
    U1, s1, V1 = pool.stream(sid).factors()
    assert np.array_equal(s0, s1)
    pool.close()
