"""Allocation-free orthogonality measurement vs the allocating path, through the C ABI.

isvd_orth_error_noalloc serves callers that cannot allocate device memory (memory pools that
forbid new allocations, code that must not synchronise the device, processes whose allocator
belongs to another framework); its scratch is a fixed device array inside the library. This test
checks, on two calls in a row, that it reports the same max|Q^T Q - I| as the existing
isvd_reorthogonalize (which uses the handle's own workspace) for the U and V of a live stream, and
that it agrees with the same quantity computed in float64 NumPy from the downloaded factors, from a
matrix whose rows span many row splits of the Gram kernel at the fixed maximum r = 128, and that a
factor holding a NaN reports NaN.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_24514_gb300 import streams

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_orth_error_matches_reorthogonalize(prec):
    torch = pytest.importorskip("torch")
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    L = pkg.lib()
    fn = L.isvd_orth_error_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]

    A0, fm = streams.make_panel(300, 90, 6, seed=91)
    ev = streams.make_events(fm, 300, 60, mix=(0.6, 0.2, 0.2), seed=92)
    # orth_tol = 1 so the existing monitor only measures and never rewrites U and V.
    g = pkg.ISVD(A0, 12, prec=prec, orth_tol=1.0, orth_every=10**9)
    g.apply_events(ev)
    m, n, r, _ = g.shape()
    dt = torch.float64 if prec == 0 else torch.float32
    Ud = torch.empty((m, r), dtype=dt, device="cuda")
    Vd = torch.empty((n, r), dtype=dt, device="cuda")
    assert L.isvd_get_factors(g._h, C.c_void_p(Ud.data_ptr()), None, C.c_void_p(Vd.data_ptr()), 1) == 0
    err_u, err_v = g.reorthogonalize(force=False)          # existing entry point
    assert err_u > 0 and err_v > 0

    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):                                    # two calls in a row share the scratch
        assert fn(Ud.data_ptr(), m, r, r, prec, out[2 * call].data_ptr(), None) == 0
        assert fn(Vd.data_ptr(), n, r, r, prec, out[2 * call + 1].data_ptr(), None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    tol = 1e-13 if prec == 0 else 1e-9
    for call in range(2):
        assert abs(got[2 * call] - err_u) <= tol + 1e-9 * err_u, (got, err_u)
        assert abs(got[2 * call + 1] - err_v) <= tol + 1e-9 * err_v, (got, err_v)

    # Independent reference: max|Q^T Q - I| of the downloaded factors in float64 NumPy.
    for Q, val in ((Ud, got[2]), (Vd, got[3])):
        Qh = Q.cpu().numpy().astype(np.float64)
        ref = np.abs(Qh.T @ Qh - np.eye(r)).max()
        assert abs(val - ref) <= 1e-13 + 1e-9 * ref, (val, ref)

    # Sizes beyond the fixed scratch are rejected before any device work.
    assert fn(Ud.data_ptr(), m, 129, 129, prec, out.data_ptr(), None) == 2   # ISVD_ESHAPE
    assert fn(None, m, r, r, prec, out.data_ptr(), None) == 1                # ISVD_EINVAL
    g.close()


def _fn():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    fn = pkg.lib().isvd_orth_error_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    return fn


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_many_splits_at_max_rank_matches_numpy(prec):
    """100,000 rows (hundreds of row splits) at r = 128, in a row stride wider than r."""
    torch = pytest.importorskip("torch")
    fn = _fn()
    rows, r, ld = 100_000, 128, 132
    g = np.random.Generator(np.random.PCG64(17))
    Q, _ = np.linalg.qr(g.standard_normal((rows, r)))
    Q[:, 5] *= 1.0 + 3e-6            # a known departure from orthonormality
    dt = np.float64 if prec == 0 else np.float32
    Qs = np.zeros((rows, ld), dt)
    Qs[:, :r] = Q
    Qd = torch.from_numpy(Qs).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        assert fn(Qd.data_ptr(), rows, r, ld, prec, out[call].data_ptr(), None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    Qh = Qs[:, :r].astype(np.float64)
    ref = np.abs(Qh.T @ Qh - np.eye(r)).max()
    assert ref > 5e-6
    for v in got:
        assert abs(v - ref) <= 1e-12, (v, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_reports_nan_for_a_nan_factor(prec):
    torch = pytest.importorskip("torch")
    fn = _fn()
    rows, r = 50, 6
    dt = torch.float64 if prec == 0 else torch.float32
    Q = torch.linalg.qr(torch.randn(rows, r, dtype=torch.float64))[0].to(dt)
    Q[17, 3] = float("nan")
    Qd = Q.cuda()
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    assert fn(Qd.data_ptr(), rows, r, r, prec, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert np.isnan(out.item())
