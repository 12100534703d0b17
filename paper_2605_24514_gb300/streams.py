"""Seeded synthetic inputs: factor-model return panels and update-event streams.

This module holds no arithmetic of the incremental-SVD method itself. It only draws
random data, so that the CUDA path and the CPU oracle can be fed identical inputs.

The generator follows the factor-model description of the workloads (Section 5 uses a
time x asset return panel; the synthetic stand-in used here has the same structure):

* ``f`` latent factors with volatilities ``0.02 * 0.7**j`` (j = 0..f-1; the decay 0.7 can be
  changed, e.g. to keep many factors above the noise), factor returns
  ``F[t, j] ~ N(0, (0.02*0.7**j)**2)``;
* loadings ``B[i, j] ~ N(0, 1) / sqrt(f)`` for every asset i;
* idiosyncratic noise either ``scale * T_nu`` (unit-scale Student-t, default nu = 4,
  scale 0.01) or Gaussian with a given standard deviation;
* a row (one time step) is ``x_t = B f_t + eps_t``; a new column (one new asset with
  fresh loadings ``b``) is ``y = F b + eps`` over the stored factor history ``F``.

Entry updates pick (i, j) uniformly over the current shape and draw
``delta ~ N(0, sd)`` where the second argument is read as a standard deviation.

Everything is drawn with ``numpy.random.Generator(PCG64(seed))`` in float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ROW, COL, ENTRY = 0, 1, 2


@dataclass
class FactorModel:
    """Stateful factor-model panel generator (keeps loadings and factor history)."""

    n: int
    f: int
    seed: int = 0
    noise: str = "t"          # "t" (Student-t) or "gauss"
    noise_scale: float = 0.01
    nu: float = 4.0
    vol_decay: float = 0.7
    rng: np.random.Generator = field(init=False, repr=False)
    B: np.ndarray = field(init=False, repr=False)
    F: np.ndarray = field(init=False, repr=False)
    t: int = field(init=False, default=0)

    def __post_init__(self):
        self.rng = np.random.Generator(np.random.PCG64(self.seed))
        self.vol = 0.02 * self.vol_decay ** np.arange(self.f)
        self.B = self.rng.standard_normal((self.n, self.f)) / np.sqrt(self.f)
        self.F = np.zeros((64, self.f))

    def _noise(self, size):
        if self.noise == "gauss":
            return self.noise_scale * self.rng.standard_normal(size)
        z = self.rng.standard_normal(size)
        chi2 = self.rng.chisquare(self.nu, size)
        return self.noise_scale * z / np.sqrt(chi2 / self.nu)

    def rows(self, t: int) -> np.ndarray:
        """Draw ``t`` new time steps (rows) over the current asset set."""
        Fn = self.rng.standard_normal((t, self.f)) * self.vol
        if self.t + t > self.F.shape[0]:
            F2 = np.zeros((max(2 * self.F.shape[0], self.t + t), self.f))
            F2[:self.t] = self.F[:self.t]
            self.F = F2
        self.F[self.t:self.t + t] = Fn
        self.t += t
        return Fn @ self.B.T + self._noise((t, self.B.shape[0]))

    def new_asset(self) -> np.ndarray:
        """Draw one new asset (column) over the stored factor history."""
        b = self.rng.standard_normal(self.f) / np.sqrt(self.f)
        self.B = np.vstack([self.B, b[None, :]])
        F = self.F[:self.t]
        return F @ b + self._noise(F.shape[0])


@dataclass
class EventStream:
    """A list of update events with payloads packed in one float64 buffer.

    ``kind[e]`` is ROW, COL or ENTRY. For ROW/COL the payload is
    ``payload[off[e] : off[e] + length[e]]``; for ENTRY, ``i[e], j[e], delta[e]`` hold
    the position and the increment. ``m_after[e], n_after[e]`` are the shape after
    the event.
    """

    kind: np.ndarray
    off: np.ndarray
    length: np.ndarray
    i: np.ndarray
    j: np.ndarray
    delta: np.ndarray
    payload: np.ndarray
    m_after: np.ndarray
    n_after: np.ndarray

    def __len__(self):
        return int(self.kind.size)

    def vector(self, e: int) -> np.ndarray:
        o, l = int(self.off[e]), int(self.length[e])
        return self.payload[o:o + l]

    def slice(self, a: int, b: int) -> "EventStream":
        """Events ``a..b-1`` with payload offsets rebased to 0."""
        off = self.off[a:b]
        base = int(off[0]) if b > a else 0
        end = int(off[-1] + self.length[b - 1]) if b > a else 0
        return EventStream(self.kind[a:b].copy(), (off - base).copy(), self.length[a:b].copy(),
                           self.i[a:b].copy(), self.j[a:b].copy(), self.delta[a:b].copy(),
                           self.payload[base:end].copy(), self.m_after[a:b].copy(),
                           self.n_after[a:b].copy())


def make_panel(m0: int, n0: int, f: int, seed: int, noise: str = "t",
               noise_scale: float = 0.01, vol_decay: float = 0.7) -> tuple[np.ndarray, FactorModel]:
    """Initial panel A0 (m0 x n0) and the generator that continues it."""
    fm = FactorModel(n=n0, f=f, seed=seed, noise=noise, noise_scale=noise_scale, vol_decay=vol_decay)
    return fm.rows(m0), fm


def make_events(fm: FactorModel, m0: int, n_events: int, mix=(1.0, 0.0, 0.0),
                delta_sd: float = 0.005, seed: int = 1) -> EventStream:
    """Draw a stream of ``n_events`` events with kind probabilities ``mix``.

    ``mix`` = (row, col, entry) fractions. Event kinds and entry positions come from a
    second PCG64 stream seeded with ``seed`` so that the panel and the schedule can be
    varied independently.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.asarray(mix, dtype=np.float64)
    p = p / p.sum()
    kinds = rng.choice(3, size=n_events, p=p).astype(np.int32)
    m, n = m0, fm.B.shape[0]
    off = np.zeros(n_events, np.int64)
    length = np.zeros(n_events, np.int64)
    ii = np.zeros(n_events, np.int64)
    jj = np.zeros(n_events, np.int64)
    dd = np.zeros(n_events, np.float64)
    m_after = np.zeros(n_events, np.int64)
    n_after = np.zeros(n_events, np.int64)
    chunks = []
    pos = 0
    for e, kd in enumerate(kinds):
        if kd == ROW:
            v = fm.rows(1)[0]
            off[e], length[e] = pos, v.size
            chunks.append(v)
            pos += v.size
            m += 1
        elif kd == COL:
            v = fm.new_asset()
            assert v.size == m
            off[e], length[e] = pos, v.size
            chunks.append(v)
            pos += v.size
            n += 1
        else:
            off[e] = pos   # zero-length payload at the current position
            ii[e] = rng.integers(0, m)
            jj[e] = rng.integers(0, n)
            dd[e] = delta_sd * rng.standard_normal()
        m_after[e], n_after[e] = m, n
    payload = np.concatenate(chunks) if chunks else np.zeros(0)
    return EventStream(kinds, off, length, ii, jj, dd, payload, m_after, n_after)


def workload(name: str, seed: int = 0, n_events: int | None = None):
    """Named workloads: returns ``(A0, events, k, extra)``.

    * ``"panel-200x50-k10"``: 200x50 panel, 5 factors, k=10, 1,000 row appends then
      200 entry updates with delta sd 0.005.
    * ``"panel-2000x1000-k64"``: 2,000x1,000 panel, 20 factors, k=64, mixed updates
      70% row / 10% column / 20% entry (delta sd 0.005).
    * ``"tiny"``: 12x8 panel, 3 factors, k=4, mixed 60/20/20 updates.
    """
    if name == "panel-200x50-k10":
        A0, fm = make_panel(200, 50, 5, seed)
        ne = 1200 if n_events is None else n_events
        nrow = min(1000, ne)
        ev1 = make_events(fm, 200, nrow, mix=(1, 0, 0), seed=seed + 1000)
        if ne > nrow:
            ev2 = make_events(fm, 200 + nrow, ne - nrow, mix=(0, 0, 1), seed=seed + 2000)
            ev = concat_events(ev1, ev2)
        else:
            ev = ev1
        return A0, ev, 10, {"f": 5}
    if name == "panel-2000x1000-k64":
        A0, fm = make_panel(2000, 1000, 20, seed)
        ne = 50000 if n_events is None else n_events
        ev = make_events(fm, 2000, ne, mix=(0.7, 0.1, 0.2), seed=seed + 1000)
        return A0, ev, 64, {"f": 20}
    if name == "tiny":
        A0, fm = make_panel(12, 8, 3, seed)
        ne = 40 if n_events is None else n_events
        ev = make_events(fm, 12, ne, mix=(0.6, 0.2, 0.2), seed=seed + 1000)
        return A0, ev, 4, {"f": 3}
    raise KeyError(name)


def concat_events(a: EventStream, b: EventStream) -> EventStream:
    shift = a.payload.size
    return EventStream(np.concatenate([a.kind, b.kind]), np.concatenate([a.off, b.off + shift]),
                       np.concatenate([a.length, b.length]), np.concatenate([a.i, b.i]),
                       np.concatenate([a.j, b.j]), np.concatenate([a.delta, b.delta]),
                       np.concatenate([a.payload, b.payload]),
                       np.concatenate([a.m_after, b.m_after]), np.concatenate([a.n_after, b.n_after]))


def batched_panels(n_streams: int, seed: int = 0, n_lo: int = 50, n_hi: int = 500,
                   ks=(8, 16, 32), f: int = 5):
    """Independent streams for the batched workload: n ~ U[n_lo, n_hi], m0 = 2n,
    k drawn uniformly from ``ks``. Returns a list of (A0, FactorModel, k)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n_streams):
        n = int(rng.integers(n_lo, n_hi + 1))
        k = int(rng.choice(np.asarray(ks)))
        A0, fm = make_panel(2 * n, n, f, seed * 1_000_003 + s + 1)
        out.append((A0, fm, k))
    return out
