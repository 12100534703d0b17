"""Serving-style use of the batched pool, through the C ABI: requests of many streams arriving in
an arbitrary interleaving over many submits (continuous batching: each submit admits what has
arrived, a stream's requests keep their order), the 60/10/30 row/column/entry mix of the serving
workload with ranks 8..64 (every batched kernel: warp-per-update appends, CTA-per-update entries
and rank bucket 64), the adaptive-rank rule inside the pool, and rank bucket 128 (single-stream
kernels). Each stream's result must be the oracle's and the same as when it runs alone.
"""
import numpy as np
import pytest

import oracle
from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu

MIX = (0.6, 0.1, 0.3)


@pytest.fixture(scope="module")
def isvd():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg


def recon(U, s, V):
    return (U.astype(np.float64) * s) @ V.astype(np.float64).T


def oracle_run(A0, ev, k, f, policy=None):
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f, policy=policy)
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
    return o


def op_list(sid, ev, e, pos):
    kd = int(ev.kind[e])
    if kd == streams.ENTRY:
        return (sid, kd, int(ev.i[e]), int(ev.j[e]), float(ev.delta[e]), 0, 0), None
    v = ev.vector(e).astype(np.float32)
    return (sid, kd, 0, 0, 0.0, pos, v.size), v


def submit_chunks(pool, items, rng, max_chunk=9):
    """items: (sid, ev, e) in arrival order; submitted in chunks of random size, each chunk's
    payload packed from 0."""
    q = 0
    while q < len(items):
        c = int(rng.integers(1, max_chunk + 1))
        ops, chunks, pos = [], [], 0
        for sid, ev, e in items[q:q + c]:
            o, v = op_list(sid, ev, e, pos)
            ops.append(o)
            if v is not None:
                chunks.append(v)
                pos += v.size
        pool.submit(ops, np.concatenate(chunks) if chunks else np.zeros(1, np.float32))
        q += c


def check(U, s, V, o, tol=1e-5, what=""):
    assert s.size == o.r, what
    Ro = o.reconstruction()
    assert np.linalg.norm(recon(U, s, V) - Ro) <= tol * np.linalg.norm(Ro), what
    np.testing.assert_allclose(s, o.s, rtol=0, atol=tol * o.s[0], err_msg=what)


def test_serving_mix_alone_and_in_the_mix(isvd):
    """12 streams, n in [60, 300], k uniform in [8, 64], 16 requests each at the 60/10/30 mix,
    arriving interleaved at random over many small submits."""
    rng = np.random.default_rng(41)
    data = []
    for sidx in range(12):
        n = int(rng.integers(60, 301))
        k = int(rng.integers(8, 65))
        A0, fm = streams.make_panel(2 * n, n, 6, seed=900 + sidx)
        ev = streams.make_events(fm, 2 * n, 16, mix=MIX, seed=950 + sidx)
        A0 = A0.astype(np.float32)
        data.append((A0, ev, k, oracle.truncated_svd(A0.astype(np.float64), k)))
    pool = isvd.Pool(k_max=64, flags=isvd.POOL_COMPLETIONS)
    ids = [pool.admit(A0, k, factors=f) for A0, ev, k, f in data]
    # arrival order: a random interleaving that keeps each stream's order
    cursors = [0] * len(data)
    items = []
    while len(items) < sum(len(d[1]) for d in data):
        s_ = int(rng.integers(len(data)))
        if cursors[s_] < len(data[s_][1]):
            items.append((ids[s_], data[s_][1], cursors[s_]))
            cursors[s_] += 1
    submit_chunks(pool, items, rng)
    pool.sync()
    recs = []
    while True:
        r = pool.poll()
        if not r.size:
            break
        recs.append(r)
    recs = np.concatenate(recs)
    assert recs.size == len(items) and np.all(recs["status"] == 0)
    for sidx, (A0, ev, k, f) in enumerate(data):
        o = oracle_run(A0, ev, k, f)
        U, s, V = pool.stream(ids[sidx]).factors()
        check(U, s, V, o, what=f"mix stream {sidx} k={k}")
        # the same stream alone in a pool of its own, one request per submit
        alone = isvd.Pool(k_max=64)
        a = alone.admit(A0, k, factors=f)
        submit_chunks(alone, [(a, ev, e) for e in range(len(ev))], rng, max_chunk=1)
        alone.sync()
        Ua, sa, Va = alone.stream(a).factors()
        nrm = np.linalg.norm(o.reconstruction())
        assert np.linalg.norm(recon(U, s, V) - recon(Ua, sa, Va)) <= 1e-5 * nrm, sidx
        alone.close()
    pool.close()


def test_pool_adaptive_rank_matches_oracle(isvd):
    """Eq. evr-rank-rule in the pool: after every 25th update of a stream, k <- min(k + 1, cap)
    while sum sigma^2 / N_t < 0.9; cap = the stream's rank bucket."""
    data = []
    for sidx, (k0, cap) in enumerate([(3, 8), (10, 16), (25, 32)]):
        A0, fm = streams.make_panel(240, 90, 6, seed=970 + sidx)
        ev = streams.make_events(fm, 240, 240, mix=(0.7, 0.1, 0.2), seed=980 + sidx)
        A0 = A0.astype(np.float32)
        data.append((A0, ev, k0, cap, oracle.truncated_svd(A0.astype(np.float64), k0)))
    pool = isvd.Pool(k_max=32, rank_every=25, tau_evr=0.9)
    ids = [pool.admit(A0, k0, factors=f) for A0, ev, k0, cap, f in data]
    items = [(sid, d[1], e) for e in range(240) for sid, d in zip(ids, data)]
    submit_chunks(pool, items, np.random.default_rng(3), max_chunk=6)
    pool.sync()
    for sid, (A0, ev, k0, cap, f) in zip(ids, data):
        pol = oracle.Policy(kind=oracle.POLICY_ADAPTIVE_RANK, check_every=25, tau_evr=0.9, k_max=cap)
        o = oracle_run(A0, ev, k0, f, policy=pol)
        assert all(abs(m.evr - 0.9) > 0.05 for m in o.log), "borderline input"
        h = pool.stream(sid)
        assert h.shape()[3] == o.k == cap       # grew one step per check up to the bucket
        U, s, V = h.factors()
        check(U, s, V, o, what=f"adaptive k0={k0}")


def test_pool_rank_bucket_128(isvd):
    """k above 64: the pool runs those streams' requests through the single-stream kernels, in
    order, inside the same submits (appends and entry updates)."""
    g = np.random.default_rng(12)
    M, N, R = 260, 200, 120
    L, _ = np.linalg.qr(g.standard_normal((M, R)))
    Rt, _ = np.linalg.qr(g.standard_normal((N, R)))
    Af = (L * (10.0 * 0.96 ** np.arange(R))) @ Rt.T + 1e-7 * g.standard_normal((M, N))
    m, n, k = 150, 130, 100
    A0 = Af[:m, :n].astype(np.float32)
    f = oracle.truncated_svd(A0.astype(np.float64), k)
    pool = isvd.Pool(k_max=128)
    sid = pool.admit(A0, k, row_cap=260, col_cap=200, factors=f)
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
    for e in range(24):
        u = g.random()
        if u < 0.5:
            v = Af[m, :n].astype(np.float32)
            pool.submit([(sid, streams.ROW, 0, 0, 0.0, 0, v.size)], v)
            o.append_row(v.astype(np.float64))
            m += 1
        elif u < 0.7:
            v = Af[:m, n].astype(np.float32)
            pool.submit([(sid, streams.COL, 0, 0, 0.0, 0, v.size)], v)
            o.append_col(v.astype(np.float64))
            n += 1
        else:
            i, j, d = int(g.integers(m)), int(g.integers(n)), float(g.normal(0, 0.005))
            pool.submit([(sid, streams.ENTRY, i, j, d, 0, 0)], np.zeros(1, np.float32))
            o.update_entry(i, j, d)
    pool.sync()
    U, s, V = pool.stream(sid).factors()
    check(U, s, V, o, what="bucket 128")
    pool.close()
