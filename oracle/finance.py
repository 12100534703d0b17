"""CPU oracle of the finance layer (TEST INFRASTRUCTURE ONLY): causal centering of return rows,
low-rank covariance, and the covariance and portfolio-risk errors of Section 5.

Plain FP64 NumPy, written from the paper and shared with nothing on the CUDA path; only ``tests/``
and ``bench.py``'s CPU-baseline leg may import it.

* causal (expanding-mean) centering ........ Section 5.1, Option A (mu_t = mu_{t-1} + (r_t - mu_{t-1}) / t)
* exponentially weighted centering ......... Section 5.1, Option B (mu_t = (1 - a) mu_{t-1} + a r_t)
* sample and low-rank covariance ........... Eqs. (sample-covariance), (cov-from-svd), (low-rank-covariances)
* covariance error ......................... Eq. (cov-error)
* portfolio volatility and risk error ...... Eqs. (portfolio-vol), (risk-error)

Reading (EW start): the recursion of Option B is started from mu_0 = 0, so the first centered row is
(1 - a) r_1; Option A does not depend on its start (mu_1 = r_1 whatever mu_0).
Reading (t): the covariance normalisation 1 / (t - 1) takes t = the number of rows of the centered
matrix the factors describe.
"""
from __future__ import annotations

import numpy as np

CAUSAL, EW = 1, 2


def center_rows(raw, mode, alpha=0.0, mu=None, count=0):
    """Centers the rows of ``raw`` (time x assets) one by one. ``mu`` and ``count`` are the state
    before the first row (a zero mean and no rows by default). Returns (centered, mu, count)."""
    raw = np.asarray(raw, dtype=np.float64)
    mu = np.zeros(raw.shape[1]) if mu is None else np.array(mu, dtype=np.float64, copy=True)
    out = np.empty_like(raw)
    for t in range(raw.shape[0]):
        count += 1
        if mode == CAUSAL:
            mu = mu + (raw[t] - mu) / count
        elif mode == EW:
            mu = (1.0 - alpha) * mu + alpha * raw[t]
        else:
            raise ValueError(mode)
        out[t] = raw[t] - mu
    return out, mu, count


def sample_covariance(R):
    """Eq. (sample-covariance): R^T R / (t - 1) of a centered t x N matrix."""
    R = np.asarray(R, dtype=np.float64)
    return R.T @ R / (R.shape[0] - 1)


def lowrank_covariance(V, s, t):
    """Eq. (low-rank-covariances): V diag(s^2) V^T / (t - 1), formed explicitly (N x N)."""
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return (V * s ** 2) @ V.T / (t - 1)


def covariance_error(V_inc, s_inc, V_opt, s_opt, t):
    """Eq. (cov-error): ||S_inc - S_opt||_F / ||S_opt||_F of the two low-rank covariances."""
    S_inc = lowrank_covariance(V_inc, s_inc, t)
    S_opt = lowrank_covariance(V_opt, s_opt, t)
    return float(np.linalg.norm(S_inc - S_opt) / np.linalg.norm(S_opt))


def portfolio_vol(V, s, t, w):
    """Eq. (portfolio-vol): sqrt(w^T S w) with S the low-rank covariance."""
    w = np.asarray(w, dtype=np.float64)
    return float(np.sqrt(max(w @ lowrank_covariance(V, s, t) @ w, 0.0)))


def risk_error(V_inc, s_inc, V_opt, s_opt, t, w):
    """Eq. (risk-error): |vol_inc - vol_opt| / vol_opt."""
    a = portfolio_vol(V_inc, s_inc, t, w)
    b = portfolio_vol(V_opt, s_opt, t, w)
    return abs(a - b) / b
