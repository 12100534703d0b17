"""GB300 (sm_103a) engine for the Brand-style incremental SVD of arXiv 2605.24514.

This module is a thin ``ctypes`` binding of ``libisvd.so`` (C ABI in ``include/isvd.h``): it only
marshals arguments. Every step of the update, refresh and metrics paths runs in the library's
CUDA kernels; there is no CPU fallback, and using the engine without the built library raises.

Host inputs are NumPy arrays; device inputs are CUDA tensors (``torch``), passed by pointer.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libisvd.so")

FP64, FP32 = 0, 1
ROW, COL, ENTRY = 0, 1, 2
POLICY_NONE, POLICY_PERIODIC, POLICY_ERROR, POLICY_ANGLE, POLICY_ADAPTIVE_RANK = 0, 1, 2, 4, 8
POLICY_NOVELTY_RANK = 16
POLICY_RANK_SHRINK = 32
METRICS_CHEAP, METRICS_FULL = 0, 1
KCLASS = {"proj": 0, "core": 1, "rotate": 2, "check": 3, "refresh": 4, "reorth": 5}

STATUS = {0: "ok", 1: "EINVAL", 2: "ESHAPE", 3: "EBOUNDS", 4: "ENOMEM", 5: "EBUDGET",
          6: "ENOTCONV", 7: "ETIMEOUT", 8: "ECUDA", 9: "ENONFINITE"}


class IsvdError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Config(C.Structure):
    _fields_ = [("prec", C.c_int32), ("k_max", C.c_int32), ("tol_rel", C.c_double),
                ("row_cap", C.c_int64), ("col_cap", C.c_int64), ("cuda_stream", C.c_void_p),
                ("seed", C.c_uint64), ("orth_tol", C.c_double), ("orth_every", C.c_int64),
                ("rsvd_oversample", C.c_int32), ("rsvd_power_iters", C.c_int32)]


class Policy(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k_min", C.c_int32), ("k_max", C.c_int32),
                ("store_initial_subspace", C.c_int32), ("T_refresh", C.c_int64), ("T_min", C.c_int64),
                ("check_every", C.c_int64), ("gamma", C.c_double), ("theta_max_rad", C.c_double),
                ("tau_evr", C.c_double), ("eta", C.c_double), ("tau_shrink", C.c_double)]


class Metrics(C.Structure):
    _fields_ = [("t", C.c_int64), ("m", C.c_int64), ("n", C.c_int64), ("r", C.c_int32), ("k", C.c_int32),
                ("frob_error", C.c_double), ("frob_opt", C.c_double), ("frob_gap", C.c_double),
                ("frob_ratio", C.c_double), ("angle", C.c_double), ("angle_to_opt", C.c_double),
                ("evr", C.c_double), ("rho_last", C.c_double), ("novelty_last", C.c_double),
                ("orth_err_u", C.c_double), ("orth_err_v", C.c_double), ("N", C.c_double),
                ("refreshes", C.c_int64), ("reorths", C.c_int64), ("t_last", C.c_int64),
                ("core_sweeps", C.c_int32), ("reserved0", C.c_int32),
                ("angle_succ_u", C.c_double), ("angle_succ_v", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PoolConfig(C.Structure):
    _fields_ = [("k_max", C.c_int32), ("flags", C.c_int32), ("max_streams", C.c_int64),
                ("hbm_budget_bytes", C.c_int64), ("cuda_stream", C.c_void_p), ("tol_rel", C.c_double),
                ("orth_every", C.c_int64), ("orth_tol", C.c_double), ("rank_every", C.c_int64),
                ("tau_evr", C.c_double), ("eta_novelty", C.c_double), ("tau_shrink", C.c_double)]


POOL_TC_ROTATIONS = 1
POOL_COMPLETIONS = 2
POOL_DEVICE_CHECKS = 4
COMPLETION_DTYPE = np.dtype([("seq", np.int64), ("stream", np.int32), ("kind", np.int32), ("status", np.int32),
                             ("r", np.int32), ("rho", np.float64), ("sigma_max", np.float64), ("done_ns", np.uint64)])


class Completion(C.Structure):
    _fields_ = [("seq", C.c_int64), ("stream", C.c_int32), ("kind", C.c_int32), ("status", C.c_int32),
                ("r", C.c_int32), ("rho", C.c_double), ("sigma_max", C.c_double), ("done_ns", C.c_uint64)]


class PoolOp(C.Structure):
    _fields_ = [("stream", C.c_int32), ("kind", C.c_int32), ("i", C.c_int64), ("j", C.c_int64),
                ("delta", C.c_double), ("off", C.c_int64), ("len", C.c_int64)]


class Risk(C.Structure):
    _fields_ = [("t", C.c_int64), ("r", C.c_int32), ("reserved", C.c_int32), ("vol", C.c_double),
                ("vol_opt", C.c_double), ("risk_error", C.c_double), ("cov_error", C.c_double),
                ("cov_norm", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


CENTER_CAUSAL, CENTER_EW = 1, 2


class Event(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("i", C.c_int64), ("j", C.c_int64),
                ("delta", C.c_double), ("off", C.c_int64), ("len", C.c_int64)]


_lib = None

_SIGS = {
    "isvd_create": (C.c_int, [C.POINTER(Config), C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                              C.POINTER(C.c_void_p)]),
    "isvd_create_from_factors": (C.c_int, [C.POINTER(Config), C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                           C.POINTER(C.c_void_p)]),
    "isvd_destroy": (None, [C.c_void_p]),
    "isvd_append_row": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "isvd_append_col": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "isvd_update_entry": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_double]),
    "isvd_update_entry_exact": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_double]),
    "isvd_set_deferred_rotations": (C.c_int, [C.c_void_p, C.c_int]),
    "isvd_deferred_pending": (C.c_int, [C.c_void_p]),
    "isvd_apply_events": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int]),
    "isvd_set_policy": (C.c_int, [C.c_void_p, C.POINTER(Policy)]),
    "isvd_refresh": (C.c_int, [C.c_void_p, C.c_int]),
    "isvd_metrics": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Metrics)]),
    "isvd_last_check_metrics": (C.c_int, [C.c_void_p, C.POINTER(Metrics)]),
    "isvd_get_factors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "isvd_get_matrix": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "isvd_get_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32)]),
    "isvd_reorthogonalize": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "isvd_sync": (C.c_int, [C.c_void_p]),
    "isvd_kernel_launches": (C.c_int64, [C.c_void_p]),
    "isvd_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "isvd_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64)]),
    "isvd_latencies": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "isvd_last_error": (C.c_char_p, [C.c_void_p]),
    "isvd_status_string": (C.c_char_p, [C.c_int]),
    "isvd_pool_create": (C.c_int, [C.POINTER(PoolConfig), C.POINTER(C.c_void_p)]),
    "isvd_pool_destroy": (None, [C.c_void_p]),
    "isvd_pool_admit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int64,
                                  C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int32)]),
    "isvd_pool_release": (C.c_int, [C.c_void_p, C.c_int32]),
    "isvd_pool_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int]),
    "isvd_pool_sync": (C.c_int, [C.c_void_p]),
    "isvd_pool_stream": (C.c_void_p, [C.c_void_p, C.c_int32]),
    "isvd_pool_bytes_used": (C.c_int64, [C.c_void_p]),
    "isvd_pool_kernel_launches": (C.c_int64, [C.c_void_p]),
    "isvd_pool_last_error": (C.c_char_p, [C.c_void_p]),
    "isvd_pool_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "isvd_pool_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]),
    "isvd_pool_host_profile": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int64)]),
    "isvd_pool_poll": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "isvd_risk": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(Risk)]),
    "isvd_center_create": (C.c_int, [C.c_int32, C.c_double, C.c_int64, C.c_int32, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "isvd_center_destroy": (None, [C.c_void_p]),
    "isvd_center_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int]),
    "isvd_center_add_assets": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "isvd_center_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "isvd_pool_slots": (C.c_int64, [C.c_void_p]),
    "isvd_pool_gather_sigma": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int]),
}


def lib():
    """Loads ``libisvd.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2605_24514_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """(pointer, on_device) for a NumPy array or a CUDA tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_cuda:
            return a.data_ptr(), 0
        return a.data_ptr(), 1
    raise TypeError(type(a))


class ISVD:
    """One incremental-SVD stream (a ``libisvd`` handle)."""

    def __init__(self, A0, k, prec=FP64, k_max=0, tol_rel=0.0, stream=None, row_cap=0, col_cap=0,
                 seed=0, orth_tol=0.0, orth_every=0, rsvd_oversample=0, rsvd_power_iters=-1, factors=None):
        """``factors`` = (U0, sigma0, V0) host arrays to start from instead of computing the
        truncated SVD of A0 (isvd_create_from_factors)."""
        self.prec = prec
        self.dtype = np.float64 if prec == FP64 else np.float32
        if isinstance(A0, np.ndarray):
            A0 = np.ascontiguousarray(A0, dtype=self.dtype)
        m0, n0 = A0.shape
        cfg = Config(prec=prec, k_max=k_max, tol_rel=tol_rel, row_cap=row_cap, col_cap=col_cap,
                     cuda_stream=stream or 0, seed=seed, orth_tol=orth_tol, orth_every=orth_every,
                     rsvd_oversample=rsvd_oversample, rsvd_power_iters=rsvd_power_iters)
        ptr, dev = _ptr(A0)
        h = C.c_void_p()
        self._h = None
        if factors is None:
            st = lib().isvd_create(C.byref(cfg), ptr, m0, n0, n0, int(k), dev, C.byref(h))
        else:
            U0, s0, V0 = factors
            U0 = np.ascontiguousarray(U0, dtype=self.dtype)
            V0 = np.ascontiguousarray(V0, dtype=self.dtype)
            s0 = np.ascontiguousarray(s0, dtype=np.float64)
            st = lib().isvd_create_from_factors(C.byref(cfg), ptr, m0, n0, n0, U0.ctypes.data, s0.ctypes.data,
                                                V0.ctypes.data, int(s0.size), int(k), dev, C.byref(h))
        if st:
            raise IsvdError(st, "isvd_create")
        self._h = h

    def _check(self, st, what):
        if st:
            raise IsvdError(st, f"{what}: {lib().isvd_last_error(self._h).decode()}")

    def _vec(self, v):
        if isinstance(v, np.ndarray):
            v = np.ascontiguousarray(v, dtype=self.dtype)
        return v

    def append_row(self, x):
        x = self._vec(x)
        p, d = _ptr(x)
        self._check(lib().isvd_append_row(self._h, p, x.shape[0], d), "append_row")

    def append_col(self, y):
        y = self._vec(y)
        p, d = _ptr(y)
        self._check(lib().isvd_append_col(self._h, p, y.shape[0], d), "append_col")

    def update_entry(self, i, j, delta):
        self._check(lib().isvd_update_entry(self._h, int(i), int(j), float(delta)), "update_entry")

    def update_entry_exact(self, i, j, delta):
        """A_ij += delta in the rank-increasing form (both residual directions join the core)."""
        self._check(lib().isvd_update_entry_exact(self._h, int(i), int(j), float(delta)), "update_entry_exact")

    def set_deferred_rotations(self, enable=True):
        """Entry updates rotate small k x k factors R_U, R_V instead of U and V (isvd_set_deferred_rotations)."""
        self._check(lib().isvd_set_deferred_rotations(self._h, 1 if enable else 0), "set_deferred_rotations")

    @property
    def deferred_pending(self):
        return bool(lib().isvd_deferred_pending(self._h))

    def apply_events(self, events, payload=None):
        """Applies a ``streams.EventStream`` (payload converted to the storage type) in one call.
        ``payload`` may be given as a CUDA tensor to keep it on the device."""
        n = len(events)
        arr = (Event * max(n, 1))()
        for e in range(n):
            arr[e].kind = int(events.kind[e])
            arr[e].i = int(events.i[e])
            arr[e].j = int(events.j[e])
            arr[e].delta = float(events.delta[e])
            arr[e].off = int(events.off[e])
            arr[e].len = int(events.length[e])
        if payload is None:
            payload = np.ascontiguousarray(events.payload, dtype=self.dtype)
        p, d = _ptr(payload)
        plen = payload.shape[0] if len(payload.shape) else 0
        self._check(lib().isvd_apply_events(self._h, arr, n, p, plen, d), "apply_events")

    def set_policy(self, kind=POLICY_NONE, T_refresh=0, T_min=0, check_every=0, gamma=1.1,
                   theta_max=np.pi / 2, tau_evr=0.9, k_min=1, k_max=0, store_initial_subspace=False, eta=0.5,
                   tau_shrink=0.99):
        pol = Policy(kind=kind, k_min=k_min, k_max=k_max, store_initial_subspace=int(store_initial_subspace),
                     T_refresh=T_refresh, T_min=T_min, check_every=check_every, gamma=gamma,
                     theta_max_rad=theta_max, tau_evr=tau_evr, eta=eta, tau_shrink=tau_shrink)
        self._check(lib().isvd_set_policy(self._h, C.byref(pol)), "set_policy")

    def refresh(self, store_initial_subspace=False):
        self._check(lib().isvd_refresh(self._h, int(store_initial_subspace)), "refresh")

    def metrics(self, full=True):
        mt = Metrics()
        self._check(lib().isvd_metrics(self._h, METRICS_FULL if full else METRICS_CHEAP, C.byref(mt)), "metrics")
        return mt.as_dict()

    def last_check_metrics(self):
        mt = Metrics()
        self._check(lib().isvd_last_check_metrics(self._h, C.byref(mt)), "last_check_metrics")
        return mt.as_dict()

    def shape(self):
        m, n, r, k = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        self._check(lib().isvd_get_shape(self._h, C.byref(m), C.byref(n), C.byref(r), C.byref(k)), "get_shape")
        return m.value, n.value, r.value, k.value

    def factors(self):
        m, n, r, _ = self.shape()
        U = np.empty((m, r), self.dtype)
        V = np.empty((n, r), self.dtype)
        s = np.empty(r, np.float64)
        self._check(lib().isvd_get_factors(self._h, U.ctypes.data, s.ctypes.data, V.ctypes.data, 0), "get_factors")
        return U, s, V

    def sigma(self):
        """Current singular values (device to host copy of r doubles)."""
        r = self.shape()[2]
        s = np.empty(r, np.float64)
        self._check(lib().isvd_get_factors(self._h, None, s.ctypes.data, None, 0), "get_factors")
        return s

    def matrix(self):
        m, n, _, _ = self.shape()
        A = np.empty((m, n), self.dtype)
        self._check(lib().isvd_get_matrix(self._h, A.ctypes.data, 0), "get_matrix")
        return A

    def risk(self, w=None, full=True):
        """Low-rank covariance and portfolio risk of Section 5.3 (isvd_risk); ``w`` None = 1/n."""
        out = Risk()
        if w is None:
            p, d = None, 0
        else:
            w = self._vec(w)
            p, d = _ptr(w)
        self._check(lib().isvd_risk(self._h, p, d, 1 if full else 0, C.byref(out)), "risk")
        return out.as_dict()

    def reorthogonalize(self, force=False):
        eu, ev = C.c_double(), C.c_double()
        self._check(lib().isvd_reorthogonalize(self._h, int(force), C.byref(eu), C.byref(ev)), "reorthogonalize")
        return eu.value, ev.value

    def sync(self):
        self._check(lib().isvd_sync(self._h), "sync")

    @property
    def launches(self):
        return int(lib().isvd_kernel_launches(self._h))

    def profile(self, enable=True):
        """Starts (or stops) CUDA-event timing of each kernel class and of each update."""
        self._check(lib().isvd_profile(self._h, int(enable)), "profile")

    def profile_read(self):
        """{class: (device ms, algorithmic bytes, launches)} since ``profile()``."""
        out = {}
        for name, c in KCLASS.items():
            ms, by, n = C.c_double(), C.c_double(), C.c_int64()
            self._check(lib().isvd_profile_read(self._h, c, C.byref(ms), C.byref(by), C.byref(n)), "profile_read")
            out[name] = (ms.value, by.value, n.value)
        return out

    def latencies_us(self):
        n = C.c_int64()
        self._check(lib().isvd_latencies(self._h, None, 0, C.byref(n)), "latencies")
        buf = np.empty(max(n.value, 1), np.float64)
        self._check(lib().isvd_latencies(self._h, buf.ctypes.data, buf.size, C.byref(n)), "latencies")
        return buf[:n.value]

    def close(self):
        if self._h:
            lib().isvd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Centering:
    """Causal centering of return rows (Section 5.1, isvd_center_*): CENTER_CAUSAL (expanding mean)
    or CENTER_EW (exponentially weighted mean with forgetting factor ``alpha``)."""

    def __init__(self, n, mode=CENTER_CAUSAL, alpha=0.0, prec=FP64, stream=None):
        self.prec = prec
        self.dtype = np.float64 if prec == FP64 else np.float32
        h = C.c_void_p()
        self._c = None
        st = lib().isvd_center_create(int(mode), float(alpha), int(n), int(prec), stream or 0, C.byref(h))
        if st:
            raise IsvdError(st, "isvd_center_create")
        self._c = h
        self.n = int(n)

    def rows(self, raw):
        """Centers the rows of ``raw`` (rows x n, host array or CUDA tensor) in time order."""
        if isinstance(raw, np.ndarray):
            raw = np.ascontiguousarray(raw, dtype=self.dtype)
            out = np.empty_like(raw)
        else:
            out = raw.new_empty(raw.shape)
        rows, n = raw.shape
        p, d = _ptr(raw)
        q, _ = _ptr(out)
        st = lib().isvd_center_rows(self._c, p, rows, n, q, n, d)
        if st:
            raise IsvdError(st, "isvd_center_rows")
        return out

    def add_assets(self, mu_new):
        mu_new = np.ascontiguousarray(mu_new, dtype=np.float64)
        st = lib().isvd_center_add_assets(self._c, mu_new.ctypes.data, mu_new.size)
        if st:
            raise IsvdError(st, "isvd_center_add_assets")
        self.n += mu_new.size

    def state(self):
        mu = np.empty(self.n, np.float64)
        cnt = C.c_int64()
        st = lib().isvd_center_state(self._c, mu.ctypes.data, C.byref(cnt))
        if st:
            raise IsvdError(st, "isvd_center_state")
        return mu, cnt.value

    def close(self):
        if self._c:
            lib().isvd_center_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Borrowed(ISVD):
    """A pool stream's handle (owned by the pool)."""

    def __init__(self, handle, dtype=np.float32):
        self.prec = FP32
        self.dtype = dtype
        self._h = C.c_void_p(handle)

    def close(self):
        self._h = None


class Pool:
    """Many independent FP32 streams updated by fused per-tick launches (isvd_pool_*)."""

    def __init__(self, k_max=32, max_streams=0, hbm_budget_bytes=0, stream=None, tol_rel=0.0, flags=0,
                 orth_every=0, orth_tol=0.0, rank_every=0, tau_evr=0.9, eta_novelty=0.0, tau_shrink=0.0):
        cfg = PoolConfig(k_max=k_max, flags=flags, max_streams=max_streams, hbm_budget_bytes=hbm_budget_bytes,
                         cuda_stream=stream or 0, tol_rel=tol_rel, orth_every=orth_every, orth_tol=orth_tol,
                         rank_every=rank_every, tau_evr=tau_evr, eta_novelty=eta_novelty, tau_shrink=tau_shrink)
        h = C.c_void_p()
        st = lib().isvd_pool_create(C.byref(cfg), C.byref(h))
        if st:
            raise IsvdError(st, "isvd_pool_create")
        self._p = h

    def _check(self, st, what):
        if st:
            raise IsvdError(st, f"{what}: {lib().isvd_pool_last_error(self._p).decode()}")

    def admit(self, A0, k, row_cap=0, col_cap=0, factors=None):
        A0 = np.ascontiguousarray(A0, dtype=np.float32)
        m0, n0 = A0.shape
        sid = C.c_int32()
        if factors is None:
            st = lib().isvd_pool_admit(self._p, A0.ctypes.data, m0, n0, n0, int(k), row_cap, col_cap, None, None,
                                       None, 0, C.byref(sid))
        else:
            U0 = np.ascontiguousarray(factors[0], dtype=np.float32)
            s0 = np.ascontiguousarray(factors[1], dtype=np.float64)
            V0 = np.ascontiguousarray(factors[2], dtype=np.float32)
            r0 = min(int(k), m0, n0)
            if U0.shape != (m0, r0) or s0.shape != (r0,) or V0.shape != (n0, r0):
                raise ValueError(f"factors must be ({m0}, {r0}), ({r0},), ({n0}, {r0}) for k = {k}")
            st = lib().isvd_pool_admit(self._p, A0.ctypes.data, m0, n0, n0, int(k), row_cap, col_cap, U0.ctypes.data,
                                       s0.ctypes.data, V0.ctypes.data, 0, C.byref(sid))
        self._check(st, "isvd_pool_admit")
        return sid.value

    def admit_device(self, A0, k, row_cap=0, col_cap=0):
        """Admits a stream from a contiguous FP32 CUDA tensor A0 (m0 x n0), computing its truncated SVD."""
        m0, n0 = A0.shape
        sid = C.c_int32()
        st = lib().isvd_pool_admit(self._p, A0.data_ptr(), m0, n0, n0, int(k), row_cap, col_cap, None, None,
                                   None, 1, C.byref(sid))
        self._check(st, "isvd_pool_admit")
        return sid.value

    def release(self, sid):
        self._check(lib().isvd_pool_release(self._p, int(sid)), "isvd_pool_release")

    def submit(self, ops, payload):
        """ops: structured array / list of (stream, kind, i, j, delta, off, len); payload: FP32."""
        n = len(ops)
        arr = (PoolOp * max(n, 1))()
        for e, o in enumerate(ops):
            arr[e].stream, arr[e].kind, arr[e].i, arr[e].j, arr[e].delta, arr[e].off, arr[e].len = o
        if isinstance(payload, np.ndarray):
            payload = np.ascontiguousarray(payload, dtype=np.float32)
        p, d = _ptr(payload)
        self._check(lib().isvd_pool_submit(self._p, arr, n, p, payload.shape[0], d), "isvd_pool_submit")

    def submit_raw(self, arr, n, payload_ptr, payload_len, on_device):
        self._check(lib().isvd_pool_submit(self._p, arr, n, payload_ptr, payload_len, on_device), "isvd_pool_submit")

    def sync(self):
        self._check(lib().isvd_pool_sync(self._p), "isvd_pool_sync")

    POOL_KCLASSES = ("warp8", "warp16", "warp32", "rot8", "rot16", "rot32", "retry", "cta")

    def profile(self, enable=True):
        """Per-launch-class device timing of subsequent submits (CUDA events on each launch's
        own stream); enable=True clears and starts it."""
        self._check(lib().isvd_pool_profile(self._p, 1 if enable else 0), "isvd_pool_profile")

    def profile_read(self):
        """{class: (ms, launches)} of the launches since profile(True)."""
        n = len(self.POOL_KCLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        self._check(lib().isvd_pool_profile_read(self._p, ms, cnt, n), "isvd_pool_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.POOL_KCLASSES)}

    def poll(self, cap=1 << 16):
        """Completion records of finished ops not returned before (pool made with POOL_COMPLETIONS),
        as a NumPy structured array (fields of isvd_completion)."""
        out = np.empty(max(cap, 1), dtype=COMPLETION_DTYPE)
        n = C.c_int64()
        self._check(lib().isvd_pool_poll(self._p, out.ctypes.data, cap, C.byref(n)), "isvd_pool_poll")
        return out[:n.value]

    @property
    def slots(self):
        return int(lib().isvd_pool_slots(self._p))

    def gather_sigma(self, ld, out=None):
        """Singular values of every slot, (slots x ld) doubles zero-padded; ``out`` may be a CUDA
        tensor or a (pinned) host array, filled asynchronously on the pool's stream."""
        if out is None:
            out = np.zeros((self.slots, ld), np.float64)
        ptr, dev = _ptr(out)
        self._check(lib().isvd_pool_gather_sigma(self._p, int(ld), ptr, dev), "isvd_pool_gather_sigma")
        return out

    def host_profile(self):
        """{phase: host microseconds} of the submits since profile(True), and their count."""
        us = (C.c_double * 4)()
        n = C.c_int64()
        self._check(lib().isvd_pool_host_profile(self._p, us, 4, C.byref(n)), "isvd_pool_host_profile")
        return dict(zip(("validate", "order", "stage", "enqueue"), us)), n.value

    def stream(self, sid):
        h = lib().isvd_pool_stream(self._p, int(sid))
        if not h:
            raise IsvdError(1, "no such stream")
        return _Borrowed(h)

    @property
    def bytes_used(self):
        return int(lib().isvd_pool_bytes_used(self._p))

    @property
    def launches(self):
        return int(lib().isvd_pool_kernel_launches(self._p))

    def close(self):
        if self._p:
            lib().isvd_pool_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
