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
    # per tick, independent of the number of streams: per warp-path rank bucket (8, 16, 32) a warp,
    # a rotation and a hand-back launch, one CTA launch per rank bucket with entry updates (8, 16,
    # 32, 64), the monitor and the rank rule
    assert pool.launches <= max(len(d[1]) for d in data) * (3 * 3 + 4 + 2)
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


def _check_stream(pool, sid, o, tol=1e-5):
    U, s, V = pool.stream(sid).factors()
    Ro = o.reconstruction()
    nrm = np.linalg.norm(Ro)
    assert s.size == o.r
    assert np.linalg.norm(recon(U, s, V) - Ro) <= tol * nrm
    np.testing.assert_allclose(s, o.s, rtol=0, atol=tol * o.s[0])


def test_pool_k64_bucket(isvd):
    """k_max = 64 selects the widest fused-kernel bucket."""
    data = make_streams(6, seed=11, n_events=10, ks=(40, 64), nrange=(90, 200))
    pool = isvd.Pool(k_max=64)
    factors = [oracle.truncated_svd(A0.astype(np.float64), k) for A0, _, k in data]
    ids = [pool.admit(A0, k, factors=f) for (A0, _, k), f in zip(data, factors)]
    ops, payload = interleave(ids, data)
    pool.submit(ops, payload)
    pool.sync()
    for sidx, ((A0, ev, k), f) in enumerate(zip(data, factors)):
        o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
        for e in range(len(ev)):
            kd = int(ev.kind[e])
            if kd == streams.ENTRY:
                o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            else:
                o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
        _check_stream(pool, ids[sidx], o)
    pool.close()


def _oracle_for(A0, ev, k, f, stop=None):
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
    for e in range(len(ev) if stop is None else stop):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
    return o


@pytest.mark.parametrize("k,k_max", [(6, 16), (40, 64)])
def test_pool_long_side(isvd, k, k_max):
    """Column appends on a 4,200-row panel. Rank capacity <= 32: the warp-per-update kernel (no
    row buffer). Capacity 64: the CTA kernel's row buffer (4,096) is too short, so those appends
    run through the single-stream kernels, in order, inside the same submit."""
    A0, fm = streams.make_panel(4200, 48, 3, seed=13)
    A0 = A0.astype(np.float32)
    f = oracle.truncated_svd(A0.astype(np.float64), k)
    pool = isvd.Pool(k_max=k_max)
    sid = pool.admit(A0, k, factors=f)
    ev = streams.make_events(fm, 4200, 8, mix=(0.3, 0.5, 0.2), seed=14)
    ops, chunks, pos = [], [], 0
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            ops.append((sid, kd, int(ev.i[e]), int(ev.j[e]), float(ev.delta[e]), 0, 0))
        else:
            v = ev.vector(e).astype(np.float32)
            ops.append((sid, kd, 0, 0, 0.0, pos, v.size))
            chunks.append(v)
            pos += v.size
    pool.submit(ops, np.concatenate(chunks))
    pool.sync()
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
    for e in range(len(ev)):
        kd = int(ev.kind[e])
        if kd == streams.ENTRY:
            o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
        else:
            o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
    assert int(np.sum(ev.kind == streams.COL)) > 0
    _check_stream(pool, sid, o)
    pool.close()


def _spectrum_panel(m, n, s, seed):
    g = np.random.default_rng(seed)
    L, _ = np.linalg.qr(g.standard_normal((m, len(s))))
    R, _ = np.linalg.qr(g.standard_normal((n, len(s))))
    return (L * np.asarray(s)) @ R.T, R


def test_pool_warp_hand_back_paths(isvd):
    """Updates the warp kernel hands to the CTA kernel (tied singular values, a zero row, an
    empty factorisation) and ones it keeps (an in-span row, rank growth from a rank-deficient
    start), all in one submit, each stream against the oracle."""
    cases = []
    # tied singular values: the core's poles coincide
    A, R = _spectrum_panel(60, 30, [5.0, 3.0, 3.0, 3.0, 1.0, 0.5], seed=1)
    g = np.random.default_rng(2)
    rows = [R @ g.standard_normal(6) for _ in range(3)]
    rows.insert(1, rows[0].copy())  # the same row twice: the next core has deflated weights
    cases.append((A, 4, rows))
    # zero row, then an in-span row (a combination of rows already in A)
    A, R = _spectrum_panel(50, 20, [4.0, 2.0, 1.0], seed=3)
    cases.append((A, 3, [np.zeros(20), 0.5 * A[3] - 2.0 * A[7], R @ np.array([1.0, -1.0, 0.5]) + 0.1]))
    # rank-deficient start (exact rank 2, k = 8, both sides take their own initial SVD): the
    # rank grows with each new direction
    A, R = _spectrum_panel(40, 25, [3.0, 1.0], seed=4)
    g = np.random.default_rng(5)
    cases.append((A, 8, [g.standard_normal(25) for _ in range(5)]))
    pool = isvd.Pool(k_max=16)
    ids, fs = [], []
    for ci, (A, k, _) in enumerate(cases):
        f = oracle.truncated_svd(A, k) if ci < 2 else None
        fs.append(f)
        ids.append(pool.admit(A.astype(np.float32), k, factors=f))
    ops, chunks, pos = [], [], 0
    for t in range(max(len(c[2]) for c in cases)):
        for sid, (_, _, rows) in zip(ids, cases):
            if t < len(rows):
                v = np.asarray(rows[t], np.float32)
                ops.append((sid, streams.ROW, 0, 0, 0.0, pos, v.size))
                chunks.append(v)
                pos += v.size
    pool.submit(ops, np.concatenate(chunks))
    pool.sync()
    for sid, (A, k, rows), f in zip(ids, cases, fs):
        o = oracle.OracleISVD(A.astype(np.float32).astype(np.float64), k, tol_rel=3e-6, factors=f)
        for v in rows:
            o.append_row(np.asarray(v, np.float32).astype(np.float64))
        _check_stream(pool, sid, o)
        U, s, V = pool.stream(sid).factors()
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(s.size)).max() < 1e-4
        assert np.abs(V.T.astype(np.float64) @ V - np.eye(s.size)).max() < 1e-4
    pool.close()


@pytest.mark.parametrize("k", [3, 8, 13, 16, 27, 32])
def test_pool_warp_ranks_and_sides(isvd, k):
    """Warp kernel at every row-load shape (rank not a multiple of 4, full buckets), rows and
    columns interleaved, checked after every tick."""
    A0, fm = streams.make_panel(90, 70, 40, seed=20 + k)
    A0 = A0.astype(np.float32)
    f = oracle.truncated_svd(A0.astype(np.float64), k)
    ev = streams.make_events(fm, 90, 12, mix=(0.5, 0.5, 0.0), seed=40 + k)
    pool = isvd.Pool(k_max=32)
    sid = pool.admit(A0, k, factors=f)
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
    for e in range(len(ev)):
        v = ev.vector(e).astype(np.float32)
        pool.submit([(sid, int(ev.kind[e]), 0, 0, 0.0, 0, v.size)], v)
        o.apply(int(ev.kind[e]), v.astype(np.float64))
        pool.sync()
        _check_stream(pool, sid, o)
    A = pool.stream(sid).matrix()
    np.testing.assert_allclose(A, o.A_view(), rtol=0, atol=1e-6)
    pool.close()


@pytest.mark.parametrize("k", [9, 16, 21, 32])
def test_pool_tensor_core_rotation_matches_fp32_pipes(isvd, k):
    """The tensor-core rotation (exact BF16 digit products, rank buckets 16 and 32) against the
    FP32-pipe rotation and the oracle, on sides that span several 256-row tiles with ragged tails (rows and
    columns interleaved, so both the projection side with z_hat and the other side are rotated)."""
    A0, fm = streams.make_panel(613, 301, 40, seed=60 + k)
    A0 = A0.astype(np.float32)
    f = oracle.truncated_svd(A0.astype(np.float64), k)
    ev = streams.make_events(fm, 613, 10, mix=(0.6, 0.4, 0.0), seed=80 + k)
    pools = [isvd.Pool(k_max=32, flags=isvd.POOL_TC_ROTATIONS), isvd.Pool(k_max=32)]
    sids = [p.admit(A0, k, factors=f) for p in pools]
    o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
    for e in range(len(ev)):
        v = ev.vector(e).astype(np.float32)
        for p, sid in zip(pools, sids):
            p.submit([(sid, int(ev.kind[e]), 0, 0, 0.0, 0, v.size)], v)
        o.apply(int(ev.kind[e]), v.astype(np.float64))
    for p, sid in zip(pools, sids):
        p.sync()
        _check_stream(p, sid, o)
    (U1, s1, V1), (U2, s2, V2) = (p.stream(sid).factors() for p, sid in zip(pools, sids))
    nrm = np.linalg.norm(o.reconstruction())
    assert np.linalg.norm(recon(U1, s1, V1) - recon(U2, s2, V2)) <= 1e-5 * nrm
    for U, V in ((U1, V1), (U2, V2)):
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(U.shape[1])).max() < 1e-5
        assert np.abs(V.T.astype(np.float64) @ V - np.eye(V.shape[1])).max() < 1e-5
    for p in pools:
        p.close()


def test_pool_completion_records_and_sigma_gather(isvd):
    """isvd_pool_poll returns one record per op, each op exactly once and a stream's ops in its
    order; the records carry the rank, residual norm (Eq. row-residual) and sigma_1 each op left
    behind, checked against the oracle op by op. isvd_pool_gather_sigma returns every slot's
    singular values in one array."""
    data = make_streams(7, seed=21, n_events=9, ks=(4, 8, 16, 32), nrange=(30, 120))
    pool = isvd.Pool(k_max=32, flags=isvd.POOL_COMPLETIONS)
    factors = [oracle.truncated_svd(A0.astype(np.float64), k) for A0, _, k in data]
    ids = [pool.admit(A0, k, factors=f) for (A0, _, k), f in zip(data, factors)]
    ops, payload = interleave(ids, data)
    half = len(ops) // 2
    # two submits (seq continues across them); the second payload slice is rebased to 0
    base = min((o[5] for o in ops[half:] if o[1] != streams.ENTRY), default=0)
    ops2 = [(o[0], o[1], o[2], o[3], o[4], o[5] - base if o[1] != streams.ENTRY else 0, o[6]) for o in ops[half:]]
    pool.submit(ops[:half], payload)
    pool.submit(ops2, payload[base:])
    pool.sync()
    rec = pool.poll()
    assert rec.size == len(ops)
    assert sorted(rec["seq"].tolist()) == list(range(len(ops)))
    assert pool.poll().size == 0                      # every record is handed out once
    by_seq = {int(r["seq"]): r for r in rec}
    for sidx, ((A0, ev, k), f) in enumerate(zip(data, factors)):
        o = oracle.OracleISVD(A0.astype(np.float64), k, tol_rel=3e-6, factors=f)
        seqs = [q for q, op in enumerate(ops) if op[0] == ids[sidx]]
        assert len(seqs) == len(ev)
        for e, q in enumerate(seqs):
            kd = int(ev.kind[e])
            if kd == streams.ENTRY:
                o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            else:
                o.apply(kd, ev.vector(e).astype(np.float32).astype(np.float64))
            r = by_seq[q]
            assert r["stream"] == ids[sidx] and r["kind"] == kd and r["status"] == 0
            assert r["r"] == o.r
            assert abs(r["sigma_max"] - o.s[0]) <= 1e-5 * o.s[0]
            if kd == streams.ENTRY:
                assert r["rho"] == 0.0
            else:
                assert abs(r["rho"] - o.rho_last) <= 1e-4 * max(o.rho_last, 1e-3 * o.s[0])
        done = [int(by_seq[q]["done_ns"]) for q in seqs]
        assert done == sorted(done)                   # a stream's ops complete in its order
    G = pool.gather_sigma(32)
    assert G.shape == (pool.slots, 32)
    for sidx, sid in enumerate(ids):
        s = pool.stream(sid).sigma()
        np.testing.assert_array_equal(G[sid, :s.size], s)
        assert np.all(G[sid, s.size:] == 0.0)
    pool.release(ids[0])
    G2 = pool.gather_sigma(8)
    assert np.all(G2[ids[0]] == 0.0)
    plain = isvd.Pool(k_max=8)
    with pytest.raises(isvd.IsvdError) as e:
        plain.poll()
    assert e.value.name == "EINVAL"
    plain.close()
    pool.close()


def test_pool_device_checks_report_nonfinite_per_stream(isvd):
    """With POOL_DEVICE_CHECKS a host payload is not scanned on the host: a NaN in one stream's row
    is caught by the kernels and reported for that stream alone (sticky ENONFINITE at sync, status
    9 in its completion record), while the other streams' updates are exactly those of a pool that
    never saw the bad op. Without the flag the same submit is refused up front, nothing queued."""
    data = make_streams(4, seed=33, n_events=1, mix=(1.0, 0.0, 0.0), ks=(8, 16, 32, 32), nrange=(40, 90))
    pools = [isvd.Pool(k_max=32, flags=isvd.POOL_COMPLETIONS | isvd.POOL_DEVICE_CHECKS),
             isvd.Pool(k_max=32, flags=isvd.POOL_COMPLETIONS)]
    ids = [[p.admit(A0, k) for A0, _, k in data] for p in pools]
    rows = [ev.vector(0).astype(np.float32) for _, ev, _ in data]
    bad = 2
    rows_bad = [r.copy() for r in rows]
    rows_bad[bad][3] = np.nan
    offs = np.cumsum([0] + [r.size for r in rows])
    ops = [(ids[0][s], streams.ROW, 0, 0, 0.0, int(offs[s]), rows[s].size) for s in range(len(rows))]
    pools[0].submit(ops, np.concatenate(rows_bad))
    with pytest.raises(isvd.IsvdError) as e:
        pools[1].submit([(ids[1][s], *o[1:]) for s, o in enumerate(ops)], np.concatenate(rows_bad))
    assert e.value.name == "ENONFINITE"
    good = [s for s in range(len(rows)) if s != bad]
    pay = np.concatenate([rows[s] for s in good])
    goffs = np.cumsum([0] + [rows[s].size for s in good])
    pools[1].submit([(ids[1][s], streams.ROW, 0, 0, 0.0, int(goffs[q]), rows[s].size) for q, s in enumerate(good)], pay)
    with pytest.raises(isvd.IsvdError) as e:
        pools[0].sync()
    assert e.value.name == "ENONFINITE"
    pools[1].sync()
    rec = pools[0].poll()
    assert rec.size == len(rows)
    status = {int(r["stream"]): int(r["status"]) for r in rec}
    assert status[ids[0][bad]] == 9 and all(status[ids[0][s]] == 0 for s in good)
    for s in good:
        a, b = pools[0].stream(ids[0][s]).factors(), pools[1].stream(ids[1][s]).factors()
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    pools[0].release(ids[0][bad])
    pools[0].sync()                                   # the failure stayed with the released stream
    for p in pools:
        p.close()
