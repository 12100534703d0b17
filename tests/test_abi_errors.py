"""Argument and input checks of the C ABI that return before any device work (no GPU needed):
shape and rank limits, unknown precisions, NULL arguments, and non-finite host input (the C ABI
rejects NaN/Inf before it allocates or queues anything), through the library's own symbols."""
import ctypes as C

import numpy as np
import pytest

EINVAL, ESHAPE, ENONFINITE = 1, 2, 9
FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def pkg():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as p
    p.lib()
    return p


def create(pkg, A, k, prec, k_max=0):
    cfg = pkg.Config(prec=prec, k_max=k_max)
    h = C.c_void_p()
    m, n = A.shape
    st = pkg.lib().isvd_create(C.byref(cfg), A.ctypes.data, m, n, n, k, 0, C.byref(h))
    assert not h.value  # nothing was created
    return st


@pytest.mark.parametrize("prec,dt", [(FP32, np.float32), (FP64, np.float64)])
@pytest.mark.parametrize("shape,pos", [((3, 5), (0, 0)), ((3, 5), (2, 4)), ((2, 5000), (1, 4095)),
                                       ((2, 5000), (1, 4096)), ((1, 8193), (0, 8192)), ((2, 4096), (1, 4095))])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_create_rejects_nonfinite_host_input(pkg, prec, dt, shape, pos, bad):
    A = np.full(shape, 0.25, dtype=dt)
    A[pos] = bad
    assert create(pkg, A, 2, prec) == ENONFINITE


def test_create_rejects_bad_shapes_and_ranks(pkg):
    A = np.ones((4, 3), np.float32)
    assert create(pkg, A, 0, FP32) == ESHAPE
    assert create(pkg, A, 2, 5) == EINVAL                   # unknown precision
    assert create(pkg, A, 4, FP32, k_max=2) == EINVAL       # k above its capacity
    assert create(pkg, A, 2, FP32, k_max=129) == EINVAL     # capacity above the 128 limit
    assert create(pkg, A.astype(np.float64), 2, FP64, k_max=97) == EINVAL  # FP64 core limit
    cfg = pkg.Config(prec=FP32)
    h = C.c_void_p()
    assert pkg.lib().isvd_create(C.byref(cfg), None, 4, 3, 3, 2, 0, C.byref(h)) == EINVAL
    assert pkg.lib().isvd_create(C.byref(cfg), A.ctypes.data, 4, 3, 2, 2, 0, C.byref(h)) == ESHAPE  # lda < n


def test_noalloc_rejects_arguments_before_device_work(pkg):
    fn = pkg.lib().isvd_orth_error_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    q = np.zeros(16, np.float64)
    out = np.zeros(1, np.float64)
    assert fn(q.ctypes.data, 10, 129, 129, FP64, out.ctypes.data, None) == ESHAPE   # above the fixed scratch
    assert fn(q.ctypes.data, 10, 0, 4, FP64, out.ctypes.data, None) == EINVAL
    assert fn(q.ctypes.data, 10, 4, 3, FP64, out.ctypes.data, None) == EINVAL       # ld < r
    assert fn(q.ctypes.data, -1, 4, 4, FP64, out.ctypes.data, None) == EINVAL
    assert fn(q.ctypes.data, 10, 4, 4, 7, out.ctypes.data, None) == EINVAL          # unknown precision
    assert fn(None, 10, 4, 4, FP32, out.ctypes.data, None) == EINVAL
    assert fn(q.ctypes.data, 10, 4, 4, FP32, None, None) == EINVAL


def test_pool_rejects_arguments_before_device_work(pkg):
    L = pkg.lib()
    h = C.c_void_p()
    for k_max in (0, 129):
        cfg = pkg.PoolConfig(k_max=k_max)
        assert L.isvd_pool_create(C.byref(cfg), C.byref(h)) == EINVAL
        assert not h.value
    assert L.isvd_pool_create(None, C.byref(h)) == EINVAL
    assert L.isvd_pool_submit(None, None, 1, None, 0, 0) == EINVAL


def test_deferred_rotations_reject_null_handle(pkg):
    L = pkg.lib()
    assert L.isvd_set_deferred_rotations(None, 1) == EINVAL
    assert L.isvd_set_deferred_rotations(None, 0) == EINVAL
    assert L.isvd_deferred_pending(None) == 0
