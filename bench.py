#!/usr/bin/env python
"""Throughput and latency of incremental-SVD updates on one GB300 (or N replicas).

Default workload ``batched-4096``: 4,096 independent FP32-bulk streams, each a factor-model panel
(n ~ U[50, 500] assets, m0 = 2n rows, 5 factors, Student-t noise, k ~ {8, 16, 32}); one step = one
tick = one row append on every stream through the pool's fused launch, compared with the plain GPU
form (the same streams driven through the per-stream single-stream kernels, one launch sequence
per stream update). Error ratios of a sample of streams are measured after the timed region.

Workload ``panel-2000x1000-k64``: one FP32-bulk stream started from a 2,000 x 1,000 factor-model panel
(20 factors, Student-t noise), k = 64, mixed updates 70% row appends / 10% column appends /
20% rank-1 entry updates (delta sd 0.005), error-threshold refresh (ratio > 1.05) and
angle-threshold refresh (largest principal angle to the optimal subspace > 5 degrees) checked
every 250 updates, loss-of-orthogonality monitor every 256 updates. A "step" is one batch of
``--batch`` consecutive events of that stream through the whole path (projection, core SVD,
rotations, dense-A bookkeeping, policy checks, refreshes, re-orthogonalisation).

Workload ``tall-200000x20000``: one dense FP32 200,000 x 20,000 stream (50-factor model plus
N(0, 1e-4) noise, k = 64 by default, ``--k`` up to 128); a step is 100 rank-1 entry updates and one
row append, timed with deferred rotations (``isvd_set_deferred_rotations``) and then in the plain
form on the same handle.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on the same stream.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_24514_gb300 import streams  # noqa: E402

WORKLOADS = {
    "panel-2000x1000-k64": dict(prec="fp32", check_every=250, gamma=1.05, theta_deg=5.0, batch=500,
                                desc="2000x1000 factor panel (20 factors, t4 noise), k=64, 70/10/20 row/col/entry, "
                                     "FP32 bulk + FP64 core/rho/sigma, refresh on ratio>1.05 or angle>5deg"),
    "batched-4096": dict(prec="fp32", batch=4096, streams=4096, n_lo=50, n_hi=500, ks=(8, 16, 32),
                         desc="4096 independent factor-model streams, n ~ U[50,500], m0 = 2n, k ~ {8,16,32}, "
                              "one row append per stream per tick, FP32 bulk + FP64-class core; batched pool path "
                              "vs per-stream single-stream kernels (plain GPU form)"),
    "serving": dict(prec="fp32", streams=2000, n_lo=100, n_hi=2000, k_lo=8, k_hi=64, mix=(0.6, 0.1, 0.3),
                    rate=1e6, requests=200_000, budget_gb_per_20000=120.0, rank_every=100, tau_evr=0.9, f=10,
                    desc="serving loop: streams with n log-uniform in [100, 2000], m0 = 2n, k uniform in [8, 64], "
                         "Poisson arrivals, row/col/entry 60/10/30, admission under an HBM budget (120 GB per "
                         "20,000 streams), adaptive rank (EVR < 0.9, capped at each stream's rank bucket), "
                         "continuous batching: each submit takes the requests that have arrived"),
    "tall-200000x20000": dict(prec="fp32", m=200_000, n=20_000, f=50, noise_sd=1e-4, k=64, entries_per_append=100,
                              delta_sd=0.005,
                              desc="one dense FP32 200,000 x 20,000 stream from a 50-factor model plus N(0, 1e-4) "
                                   "noise; each step = 100 rank-1 entry updates (delta sd 0.005) then one row "
                                   "append; deferred rotations (U = U0 R_U) against the plain form on the same "
                                   "handle; no refresh policy; orthogonality monitor every 256 updates"),
    "panel-200x50-k10": dict(prec="fp64", check_every=50, T_refresh=250, batch=200,
                             desc="200x50 factor panel (5 factors), k=10, 1000 row appends then 200 entry "
                                  "updates, FP64, periodic refresh 250, metrics every 50"),
}
HBM_PEAK_FALLBACK = 6800.0
# DRAM bytes (read + write) of one launch of the default workload (4,096 streams), from the one-pass
# ncu capture of dram__bytes_read.sum and dram__bytes_write.sum summarised under profiles/ (tick 3;
# ticks differ by about 1%). Set to None whenever the kernel changes until it is captured again.
DRAM_TRAFFIC = {"k_pool_rotate<32>": 247250000, "k_pool_rotate_tc<32>": None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return HBM_PEAK_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device="cuda") -> float:
    """Max over ranks of a per-rank float (the timed region's duration), identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Replica r runs its own seeded stream(s); ranks never share inputs."""
    return 1000 + 7919 * rank


def make_stream(name, seed, n_events):
    A0, ev, k, extra = streams.workload(name, seed=seed, n_events=n_events)
    return A0, ev, k


def run_gb300(args):
    import torch

    import paper_2605_24514_gb300 as pkg
    from paper_2605_24514_gb300 import build as b

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    W = WORKLOADS[args.workload]
    B = args.batch or W["batch"]
    K, Wm = args.steps, args.warmup
    n_ev = (Wm + 2 * K) * B
    A0, ev, k = make_stream(args.workload, seed=rank_seed(rank), n_events=n_ev)
    prec = pkg.FP32 if W["prec"] == "fp32" else pkg.FP64
    dt = np.float32 if prec == pkg.FP32 else np.float64
    st = torch.cuda.Stream()
    g = pkg.ISVD(A0, k, prec=prec, k_max=k, stream=st.cuda_stream, seed=rank)
    if "gamma" in W:
        g.set_policy(kind=pkg.POLICY_ERROR | pkg.POLICY_ANGLE, check_every=W["check_every"], gamma=W["gamma"],
                     theta_max=np.deg2rad(W["theta_deg"]))
    else:
        g.set_policy(kind=pkg.POLICY_PERIODIC, T_refresh=W["T_refresh"], check_every=W["check_every"])
    payload = torch.from_numpy(ev.payload.astype(dt)).to("cuda")   # resident in HBM
    slices = []
    for s in range(Wm + 2 * K):
        a, e = s * B, (s + 1) * B
        sl = ev.slice(a, e)
        base = int(ev.off[a]) if e > a else 0
        slices.append((sl, base, base + sl.payload.size))
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")

    def step_dev(i):
        sl, lo, hi = slices[i]
        g.apply_events(sl, payload=payload[lo:hi])

    for i in range(Wm):
        step_dev(i)
    g.sync()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    g.profile(True)
    l0 = g.launches
    ratios = []
    clocks.start()
    evs = []
    torch.cuda.nvtx.range_push("timed")
    for i in range(Wm, Wm + K):
        flush.zero_()                       # evict L2 (129 MB) between steps, outside the timing
        st.wait_stream(torch.cuda.current_stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step_dev(i)
        e1.record(st)
        evs.append((e0, e1))
        ratios.append(g.last_check_metrics()["frob_ratio"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = g.launches - l0
    ms = sum(a.elapsed_time(b_) for a, b_ in evs)
    prof = g.profile_read()
    lat = g.latencies_us()
    g.profile(False)
    ms = reduce_max(ms, world)
    value = world * K * B / (ms / 1e3)

    # End to end through the public API with host buffers: each step copies its payload from
    # pinned host memory and reads sigma back.
    e2e = None
    if not args.no_e2e:
        pinned = []
        for i in range(Wm + K, Wm + 2 * K):
            sl, lo, hi = slices[i]
            h = torch.empty(hi - lo, dtype=torch.float32 if dt == np.float32 else torch.float64).pin_memory()
            h.copy_(torch.from_numpy(ev.payload[lo:hi].astype(dt)))
            pinned.append(h)
        g.sync()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for j, i in enumerate(range(Wm + K, Wm + 2 * K)):
            sl, lo, hi = slices[i]
            g.apply_events(sl, payload=pinned[j].numpy())
            sig = g.sigma()
            h2d += pinned[j].numel() * pinned[j].element_size() + 48 * len(sl)
            d2h += sig.nbytes
        torch.cuda.synchronize()
        el = reduce_max(time.perf_counter() - t0, world)
        e2e = {"value": world * K * B / el, "unit": "updates/s", "h2d_bytes_per_step": int(h2d // K),
               "d2h_bytes_per_step": int(d2h // K)}

    if rank != 0:
        return None
    peak, peak_src = measured_peaks()
    # Dominant kernel class by device time; HBM roofline from algorithmic bytes / its time.
    dom = max(prof, key=lambda c: prof[c][0])
    rot_ms, rot_bytes, rot_n = prof["rotate"]
    classes = {c: {"ms": round(v[0], 3), "launches": int(v[2]),
                   "us_per_launch": round(1e3 * v[0] / v[2], 3) if v[2] else None,
                   "GBps": round(v[1] / (v[0] * 1e6), 1) if v[0] > 0 and v[1] > 0 else None}
               for c, v in prof.items()}
    roof_cls = dom if prof[dom][1] > 0 else "rotate"
    r_ms, r_bytes, r_n = prof[roof_cls]
    achieved = r_bytes / (r_ms * 1e6) if r_ms > 0 else 0.0
    out = {
        "metric": "iSVD updates/s and p50/p99 update latency at err ratio<=1.05 vs plain GPU form",
        "value": round(value, 1),
        "unit": "updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": round(ms / K, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == pkg.FP32 else "f64",
        "data": "synthetic (seeded factor-model panel and update stream)",
        "config": {"workload": args.workload, "desc": W["desc"], "events_per_step": B,
                   "m_n_end": [int(ev.m_after[(Wm + K) * B - 1]), int(ev.n_after[(Wm + K) * B - 1])],
                   "form": "per-update kernel launches on one CUDA stream (no graph, no batching)",
                   "l2": "flushed between steps (256 MB device write, untimed)",
                   "latency_us": {"p50": round(float(np.percentile(lat, 50)), 2),
                                  "p99": round(float(np.percentile(lat, 99)), 2),
                                  "mean": round(float(np.mean(lat)), 2), "n": int(lat.size)},
                   "err_ratio_at_checks_max": (None if not np.isfinite(np.nanmax(ratios)) else
                                               round(float(np.nanmax(ratios)), 5)) if ratios else None,
                   "kernel_classes": classes,
                   "parallelism": "replicas" if world > 1 else "single stream"},
        "roofline": {"kernel": roof_cls, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                     "dominant_class": dom},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_budget)
    return out


def _tall_steps(W, m0, n0, f, Bl, vol, steps, seed):
    """Per step: ``entries_per_append`` entry updates (positions uniform over the current shape,
    delta ~ N(0, delta_sd^2)) and one factor-model row; one EventStream per step."""
    rng = np.random.default_rng(seed)
    per = W["entries_per_append"]
    out = []
    m = m0
    for _ in range(steps):
        kind = np.full(per + 1, streams.ENTRY, np.int32)
        kind[-1] = streams.ROW
        ii = np.zeros(per + 1, np.int64)
        jj = np.zeros(per + 1, np.int64)
        dd = np.zeros(per + 1, np.float64)
        ii[:per] = rng.integers(0, m, per)
        jj[:per] = rng.integers(0, n0, per)
        dd[:per] = W["delta_sd"] * rng.standard_normal(per)
        x = Bl @ (vol * rng.standard_normal(f)) + W["noise_sd"] * rng.standard_normal(n0)
        off = np.zeros(per + 1, np.int64)
        length = np.zeros(per + 1, np.int64)
        length[-1] = n0
        m_after = np.full(per + 1, m, np.int64)
        m_after[-1] = m + 1
        out.append(streams.EventStream(kind, off, length, ii, jj, dd, x, m_after, np.full(per + 1, n0, np.int64)))
        m += 1
    return out


def run_tall(args):
    """One tall FP32 stream: steps of entry updates and a row append, timed with deferred
    rotations and then in the plain form on the same handle."""
    import torch

    import paper_2605_24514_gb300 as pkg
    from paper_2605_24514_gb300 import build as b

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    W = WORKLOADS[args.workload]
    m0, n0, f = args.m or W["m"], args.n or W["n"], W["f"]
    k = args.k or W["k"]
    K, Wm = args.steps, args.warmup
    seed = rank_seed(rank)
    rng = np.random.default_rng(seed)
    vol = 0.02 * 0.7 ** np.arange(f)
    Bl = rng.standard_normal((n0, f)) / np.sqrt(f)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    # A0 = F B^T + noise, drawn on the device in row chunks (inputs only; the method never runs here)
    A0 = torch.empty(m0, n0, dtype=torch.float32, device="cuda")
    Bt = torch.tensor(Bl.T, dtype=torch.float32, device="cuda")
    volt = torch.tensor(vol, dtype=torch.float32, device="cuda")
    for a in range(0, m0, 20000):
        e = min(m0, a + 20000)
        F = torch.randn(e - a, f, generator=gen, device="cuda") * volt
        A0[a:e] = F @ Bt + W["noise_sd"] * torch.randn(e - a, n0, generator=gen, device="cuda")
    del Bt
    n_steps = 2 * Wm + 3 * K
    steps = _tall_steps(W, m0, n0, f, Bl, vol, n_steps, seed + 1)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = pkg.ISVD(A0, k, prec=pkg.FP32, k_max=k, stream=st.cuda_stream, seed=rank, row_cap=m0 + n_steps + 8,
                 col_cap=n0)
    g.sync()
    create_s = time.perf_counter() - t0
    del A0
    torch.cuda.empty_cache()
    payload = [torch.from_numpy(s.payload.astype(np.float32)).to("cuda") for s in steps]
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
    B = len(steps[0])

    def timed(first, count):
        evs = []
        for i in range(first, first + count):
            flush.zero_()
            st.wait_stream(torch.cuda.current_stream())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g.apply_events(steps[i], payload=payload[i])
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b_) for a, b_ in evs)

    # deferred form: warm-up, then the timed steps with profiling and clocks
    g.set_deferred_rotations(True)
    timed(0, Wm)
    clocks = Clocks(local)
    g.profile(True)
    l0 = g.launches
    clocks.start()
    ms = timed(Wm, K)
    clk = clocks.stop()
    launches = g.launches - l0
    prof = g.profile_read()
    g.profile(False)
    ms = reduce_max(ms, world)
    value = world * K * B / (ms / 1e3)
    # end to end: payload from pinned host memory, sigma read back, per step
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(steps[i].payload.astype(np.float32)).pin_memory() for i in range(Wm + K, Wm + 2 * K)]
        g.sync()
        t0 = time.perf_counter()
        d2h = 0
        for j, i in enumerate(range(Wm + K, Wm + 2 * K)):
            g.apply_events(steps[i], payload=pinned[j].numpy())
            d2h += g.sigma().nbytes
        torch.cuda.synchronize()
        el = reduce_max(time.perf_counter() - t0, world)
        e2e = {"value": world * K * B / el, "unit": "updates/s", "h2d_bytes_per_step": int(4 * n0 + 48 * B),
               "d2h_bytes_per_step": int(d2h // K)}
    # plain form on the same handle
    g.set_deferred_rotations(False)
    timed(Wm + 2 * K, Wm)
    ms_plain = reduce_max(timed(2 * Wm + 2 * K, K), world)
    eu, ev_ = g.reorthogonalize(force=False)
    if rank != 0:
        return None
    peak, peak_src = measured_peaks()
    classes = {c: {"ms": round(v[0], 3), "launches": int(v[2]),
                   "us_per_launch": round(1e3 * v[0] / v[2], 3) if v[2] else None,
                   "GBps": round(v[1] / (v[0] * 1e6), 1) if v[0] > 0 and v[1] > 0 else None}
               for c, v in prof.items()}
    dom = max(prof, key=lambda c: prof[c][0])
    r_ms, r_bytes, _ = prof["rotate"]
    achieved = r_bytes / (r_ms * 1e6) if r_ms > 0 else 0.0
    out = {
        "metric": "iSVD updates/s of one tall stream, deferred rotations vs the plain form",
        "value": round(value, 1),
        "unit": "updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": round(ms / K, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded 50-factor model drawn on the device, update stream from the same model)",
        "config": {"workload": args.workload, "desc": W["desc"], "m0": m0, "n0": n0, "k": k, "events_per_step": B,
                   "form": "deferred rotations, per-update kernel launches on one CUDA stream",
                   "plain_form_updates_per_s": round(world * K * B / (ms_plain / 1e3), 1),
                   "speedup_vs_plain_form": round(ms_plain / ms, 3),
                   "create_s": round(create_s, 2),
                   "orth_err_end": [eu, ev_],
                   "l2": "flushed between steps (256 MB device write, untimed); U, V and A exceed L2",
                   "kernel_classes": classes, "dominant_class": dom,
                   "parallelism": "replicas" if world > 1 else "single stream"},
        "roofline": {"kernel": "rotate", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                     "note": "the fold and append rotations; the deferred entry updates move k x k data only"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline_tall(W, k, budget_s=args.cpu_budget)
    return out


def cpu_baseline_tall(W, k, budget_s=15.0):
    """The oracle on the same step pattern at a reduced shape (20,000 x 2,000): its dense FP64 A
    and per-update SVDs of the full shape do not fit a bounded CPU sample."""
    import oracle
    m0, n0, f = 20_000, 2_000, W["f"]
    rng = np.random.default_rng(5)
    vol = 0.02 * 0.7 ** np.arange(f)
    Bl = rng.standard_normal((n0, f)) / np.sqrt(f)
    A0 = (rng.standard_normal((m0, f)) * vol) @ Bl.T + W["noise_sd"] * rng.standard_normal((m0, n0))
    A0 = A0.astype(np.float32).astype(np.float64)
    steps = _tall_steps(W, m0, n0, f, Bl, vol, 50, 6)
    t0 = time.perf_counter()
    o = oracle.OracleISVD(A0, k, tol_rel=3e-6)
    t1 = time.perf_counter()
    n = 0
    for sl in steps:
        for e in range(len(sl)):
            if sl.kind[e] == streams.ENTRY:
                o.update_entry(sl.i[e], sl.j[e], sl.delta[e])
            else:
                o.append_row(sl.vector(e).astype(np.float32).astype(np.float64))
            n += 1
            if time.perf_counter() - t1 > budget_s:
                break
        if time.perf_counter() - t1 > budget_s:
            break
    el = time.perf_counter() - t1
    return {"value": round(n / el, 3), "unit": "updates/s", "cores": _blas_threads(), "kind": "oracle",
            "sample": f"{n} events of the same step pattern on a 20,000 x 2,000 panel at k = {k} "
                      f"(create {t1 - t0:.1f} s excluded; time budget {budget_s:.0f} s)"}


def run_batched(args):
    """Batched workload: one step = one tick = one row append on every stream."""
    import ctypes as C

    import torch

    import paper_2605_24514_gb300 as pkg
    from paper_2605_24514_gb300 import build as b

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    W = WORKLOADS[args.workload]
    S = args.streams or W["streams"]
    K, Wm = args.steps, args.warmup
    plain_ticks = args.plain_ticks
    n_lat = args.lat_ticks
    t_lat = Wm + K
    t_plain = t_lat + n_lat
    t_e2e = t_plain + (plain_ticks + 1 if plain_ticks > 0 else 0)
    T = t_e2e + (K if not args.no_e2e else 0)
    rng = np.random.Generator(np.random.PCG64(rank_seed(rank)))
    ns = rng.integers(W["n_lo"], W["n_hi"] + 1, size=S)
    ks = rng.choice(np.asarray(W["ks"]), size=S)
    st = torch.cuda.Stream()
    pool = pkg.Pool(k_max=int(max(W["ks"])), stream=st.cuda_stream,
                    flags=pkg.POOL_COMPLETIONS | pkg.POOL_DEVICE_CHECKS |
                    (pkg.POOL_TC_ROTATIONS if args.tc_rotations else 0))
    t0 = time.perf_counter()
    ids, rows, payload_parts, offs = [], [], [], []
    for sidx in range(S):
        n = int(ns[sidx])
        A0, fm = streams.make_panel(2 * n, n, 5, seed=rank_seed(rank) * 1_000_003 + sidx + 1)
        ids.append(pool.admit(A0.astype(np.float32), int(ks[sidx]), row_cap=2 * n + T + 8, col_cap=n + 2))
        rows.append(fm.rows(T).astype(np.float32))
    setup_s = time.perf_counter() - t0
    # Tick-major payload: tick t holds row t of every stream.
    payload = np.concatenate([rows[sidx][t] for t in range(T) for sidx in range(S)])
    tick_len = int(np.sum(ns))
    starts = np.concatenate([[0], np.cumsum(ns)[:-1]])

    def tick_ops(t):
        arr = (pkg.PoolOp * S)()
        for sidx in range(S):
            arr[sidx].stream = ids[sidx]
            arr[sidx].kind = 0
            arr[sidx].off = int(starts[sidx])
            arr[sidx].len = int(ns[sidx])
        return arr

    ops = tick_ops(0)
    pay_dev = torch.from_numpy(payload).to("cuda")

    def tick_dev(t):
        base = t * tick_len
        pool.submit_raw(ops, S, pay_dev[base:base + tick_len].data_ptr(), tick_len, 1)

    for t in range(Wm):
        tick_dev(t)
    pool.sync()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    # Algorithmic bytes of one tick: every stream's U and V read and written once, plus x read
    # and the new row of A written.
    ms_, ns_, ks_ = 2 * ns + Wm, ns, ks
    clocks = Clocks(local)
    l0 = pool.launches
    clocks.start()
    evs, tick_bytes, host_s = [], [], []
    # Algorithmic bytes per launch of each kernel class (row append, stream of n columns, m rows
    # before the update, rank k = its bucket): the rotation reads and writes U and V once and
    # reads x once; the projection + core reads V and x twice (CGS2) and writes the new rows of
    # A and U.
    class_bytes = {}
    for kb in W["ks"]:
        sel = ks == kb
        rot, warp = 0.0, 0.0
        for t in range(Wm, Wm + K):
            m_now = 2 * ns[sel] + t
            rot += float(np.sum((2.0 * (m_now + ns[sel]) * kb + ns[sel]) * 4))
            warp += float(np.sum((2.0 * ns[sel] * kb + 3.0 * ns[sel] + kb) * 4))
        class_bytes[f"rot{kb}"] = rot / K
        class_bytes[f"warp{kb}"] = warp / K
    pool.profile(True)
    torch.cuda.nvtx.range_push("timed")
    for t in range(Wm, Wm + K):
        m_now = 2 * ns + t
        tick_bytes.append(float(np.sum((2.0 * (m_now + ns) * ks + 2.0 * ns) * 4)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h0 = time.perf_counter()
        tick_dev(t)
        host_s.append(time.perf_counter() - h0)
        e1.record(st)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    prof = pool.profile_read()
    host_phases, host_n = pool.host_profile()
    pool.profile(False)
    launches = pool.launches - l0
    tick_ms = np.array([a.elapsed_time(b_) for a, b_ in evs])
    ms = float(tick_ms.sum())
    pool.sync()
    ms = reduce_max(ms, world)
    value = world * K * S / (ms / 1e3)
    # Update latency: every update of a tick completes with it, so the latency of an update
    # submitted at a tick boundary is that tick's device time; L more ticks, each timed alone.
    lat_ms = []
    for t in range(t_lat, t_lat + n_lat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        tick_dev(t)
        e1.record(st)
        lat_ms.append((e0, e1))
    torch.cuda.synchronize()
    lat_ms = np.array([a.elapsed_time(b_) for a, b_ in lat_ms])
    while pool.poll().size:                       # drop the records of the ticks so far
        pass
    # Plain GPU form: the same streams, next ticks, one single-stream launch sequence per stream
    # (one untimed warm-up tick, then plain_ticks timed ones).
    handles = [pool.stream(i) for i in ids]

    def plain_tick(t):
        base = t * tick_len
        for sidx in range(S):
            off = base + int(starts[sidx])
            handles[sidx].append_row(pay_dev[off:off + int(ns[sidx])])

    plain_value, plain_spread = None, None
    if plain_ticks > 0:
        plain_tick(t_plain)
        torch.cuda.synchronize()
        pms = []
        torch.cuda.nvtx.range_push("plain")
        for t in range(t_plain + 1, t_plain + 1 + plain_ticks):
            pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pe0.record(st)
            plain_tick(t)
            pe1.record(st)
            pms.append((pe0, pe1))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        pms = np.array([a.elapsed_time(b_) for a, b_ in pms])
        plain_value = plain_ticks * S / (float(pms.sum()) / 1e3)
        plain_spread = [round(float(pms.min()), 2), round(float(pms.max()), 2)]
    e2e = None
    if not args.no_e2e:
        # End to end through the C ABI: each tick's payload comes from pinned host memory, and each
        # tick's results go back to the host: every stream's singular values (one gather, one copy)
        # and every op's completion record. Ticks are pipelined: tick q+1 is submitted before the
        # results of tick q are read.
        pinned = torch.from_numpy(payload[t_e2e * tick_len:(t_e2e + K) * tick_len]).pin_memory()
        sig_out = [torch.empty((pool.slots, 32), dtype=torch.float64).pin_memory() for _ in range(2)]
        pool.sync()
        while pool.poll().size:
            pass
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        pool.profile(True)                          # host phase times of the e2e submits
        t0 = time.perf_counter()
        n_rec = 0
        t_sub = t_gat = t_pol = 0.0
        for q in range(K):
            seg = pinned[q * tick_len:(q + 1) * tick_len]
            a = time.perf_counter()
            pool.submit_raw(ops, S, seg.data_ptr(), tick_len, 0)
            b_ = time.perf_counter()
            pool.gather_sigma(32, out=sig_out[q % 2].numpy())
            c_ = time.perf_counter()
            n_rec += pool.poll().size
            t_sub += b_ - a
            t_gat += c_ - b_
            t_pol += time.perf_counter() - c_
        pool.sync()
        while True:
            got = pool.poll().size
            if not got:
                break
            n_rec += got
        el = reduce_max(time.perf_counter() - t0, world)
        assert n_rec == K * S, (n_rec, K * S)
        e2e_phases, _ = pool.host_profile()
        pool.profile(False)
        d2h = pool.slots * 32 * 8 + S * 48
        e2e = {"value": world * K * S / el, "unit": "updates/s",
               "h2d_bytes_per_step": int(tick_len * 4 + S * 136), "d2h_bytes_per_step": int(d2h),
               "results": "all streams' sigma (gather, one D2H copy) and one completion record per update, per tick",
               "host_us_per_step": {"submit": round(1e6 * t_sub / K, 1), "gather": round(1e6 * t_gat / K, 1),
                                    "poll": round(1e6 * t_pol / K, 1),
                                    "submit_phases": {k: round(v / K, 1) for k, v in e2e_phases.items()}}}
    # Error ratio (Section 2.5) of a sample of streams after all ticks; the CPU-baseline leg replays
    # the same streams through the oracle and compares.
    sample_ids = list(range(min(S, args.acc_streams)))
    gpu_ratios = [handles[sidx].metrics(full=True)["frob_ratio"] for sidx in sample_ids]
    sweeps = [handles[sidx].metrics(full=False)["core_sweeps"] for sidx in range(0, S, max(1, S // 256))]
    if rank != 0:
        return None
    peak, peak_src = measured_peaks()
    ach_tick = float(np.sum(tick_bytes)) / (ms * 1e6)
    # Dominant kernel for the HBM roofline: the launch class that moves the most algorithmic bytes
    # per tick (the k = 32 rotation here, also the top share of the ncu launch list); its time is
    # the live CUDA-event time of its launches on their own stream in the timed region.
    dom = max((c for c in class_bytes if prof.get(c, (0.0, 0))[1] > 0), key=lambda c: class_bytes[c])
    dom_ms, dom_n = prof[dom]
    ach = class_bytes.get(dom, 0.0) / (dom_ms / dom_n * 1e6) if dom in class_bytes else 0.0
    tc = "_tc" if args.tc_rotations else ""
    kernel_names = {"warp8": "k_pool_warp<8>", "warp16": "k_pool_warp<16>", "warp32": "k_pool_warp<32>",
                    "rot8": "k_pool_rotate<8>", "rot16": f"k_pool_rotate{tc}<16>", "rot32": f"k_pool_rotate{tc}<32>",
                    "retry": "k_pool_retry<32>", "cta": "k_pool_tick"}
    out = {
        "metric": "iSVD updates/s and p50/p99 update latency at err ratio<=1.05 vs plain GPU form",
        "value": round(value, 1), "unit": "updates/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": round(ms / K, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded factor-model panels and rows)",
        "config": {"workload": args.workload, "desc": W["desc"], "streams": S, "events_per_step": S,
                   "k_mix": {str(k): int(np.sum(ks == k)) for k in W["ks"]},
                   "form": "per rank bucket (8/16/32) on its own CUDA stream, so that the buckets' ticks overlap; per tick and bucket a warp-per-update projection + core launch, a persistent rotation launch, a hand-back launch and a completion-record launch",
                   "plain_form_updates_per_s": round(plain_value, 1) if plain_value else None,
                   "plain_form_ticks": plain_ticks, "plain_form_tick_ms_min_max": plain_spread,
                   "speedup_vs_plain": round(value / plain_value, 2) if plain_value else None,
                   "l2": "working set per tick larger than L2 (no flush needed)",
                   "latency_us": {"p50": round(float(np.percentile(lat_ms, 50)) * 1e3, 1) if lat_ms.size else None,
                                  "p99": round(float(np.percentile(lat_ms, 99)) * 1e3, 1) if lat_ms.size else None,
                                  "max": round(float(lat_ms.max()) * 1e3, 1) if lat_ms.size else None,
                                  "ticks": int(lat_ms.size),
                                  "note": "device time of a tick, measured alone; every update of a tick "
                                          "completes with it"},
                   "err_ratio_gpu_sample": [round(float(r), 6) for r in gpu_ratios],
                   "host_submit_us_per_tick": round(float(np.mean(host_s)) * 1e6, 1),
                   "host_submit_phases_us": {k: round(v / max(host_n, 1), 1) for k, v in host_phases.items()},
                   "core_fast_path_frac": round(float(np.mean(np.asarray(sweeps) >= 100)), 4) if sweeps else None,
                   "core_corrected_weights_frac": round(float(np.mean(np.asarray(sweeps) == 102)), 4) if sweeps else None,
                   "setup_s": round(setup_s, 1), "parallelism": "replicas" if world > 1 else "streams in one pool"},
        "roofline": {"kernel": kernel_names[dom], "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": DRAM_TRAFFIC.get(kernel_names[dom]),
                     "algorithmic_bytes_per_launch": round(class_bytes.get(dom, 0.0)),
                     "ms_per_launch": round(dom_ms / dom_n, 4),
                     "tick_achieved_gbs": round(ach_tick, 1),
                     "kernel_ms_per_tick": {c: round(v[0] / K, 4) for c, v in prof.items() if v[1] > 0},
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    pool.close()
    if not args.no_cpu_baseline and world == 1:
        cb, orc_ratios = cpu_baseline_batched(args, T, sample_ids)
        out["cpu_baseline"] = cb
        rel = [abs(g / o - 1.0) for g, o in zip(gpu_ratios, orc_ratios)]
        out["config"]["accuracy"] = {
            "err_ratio_oracle_sample": [round(float(r), 6) for r in orc_ratios],
            "max_rel_diff_vs_oracle": float(max(rel)) if rel else None,
            "ok": bool(all(np.isfinite(gpu_ratios)) and max(gpu_ratios) <= 1.05 and max(rel) <= 0.01),
            "rule": "every sampled ratio finite and <= 1.05, and within 1% of the oracle's on the same stream"}
    return out


def _serving_inputs(W, S, N, seed, torch):
    """Synthetic serving workload, drawn on the device with torch (input generation only): per stream
    a factor-model panel A0 (2n x n), and the scripted requests that the Poisson arrivals draw from:
    rows x = B f + eps, new assets y = F b + eps over the stream's factor history, entry increments
    delta ~ N(0, 0.005) at uniform positions. Returns panels, stream parameters, the arrival-ordered
    request table and one device payload buffer."""
    dev = "cuda"
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    f = W["f"]
    ns = np.exp(rng.uniform(np.log(W["n_lo"]), np.log(W["n_hi"]), size=S)).astype(np.int64)
    ks = rng.integers(W["k_lo"], W["k_hi"] + 1, size=S)
    arr = np.cumsum(rng.exponential(1.0 / W["rate"], size=N))        # arrival times (s)
    who = rng.integers(0, S, size=N)                                  # stream of each arrival
    kinds = rng.choice(3, size=N, p=np.asarray(W["mix"]))
    vol = torch.tensor(0.02 * 0.7 ** np.arange(f), device=dev, dtype=torch.float32)

    def noise(shape):
        z = torch.randn(shape, generator=g, device=dev)
        c = torch.distributions.Chi2(torch.tensor(4.0, device=dev)).sample(shape)
        return 0.01 * z / torch.sqrt(c / 4.0)

    panels, pay, offs, lens = [], [], np.zeros(N, np.int64), np.zeros(N, np.int64)
    ii, jj, dd = np.zeros(N, np.int64), np.zeros(N, np.int64), np.zeros(N)
    pos = 0
    order = np.argsort(who, kind="stable")
    bounds = np.searchsorted(who[order], np.arange(S + 1))
    for sidx in range(S):
        n = int(ns[sidx])
        mine = order[bounds[sidx]:bounds[sidx + 1]]                   # this stream's arrivals, in order
        n_rows = int(np.sum(kinds[mine] == 0))
        B = torch.randn((n, f), generator=g, device=dev) / np.sqrt(f)
        Fh = torch.randn((2 * n + n_rows, f), generator=g, device=dev) * vol
        panels.append((Fh[:2 * n] @ B.T + noise((2 * n, n))).contiguous())
        rows = Fh[2 * n:] @ B.T + noise((n_rows, n))
        m, ncol, ri = 2 * n, n, 0
        for q in mine:
            kd = int(kinds[q])
            if kd == 0:
                v = rows[ri, :ncol] if ncol == n else torch.cat(
                    [rows[ri], torch.randn(ncol - n, generator=g, device=dev) * 0.01])
                ri += 1
                m += 1
            elif kd == 1:
                b = torch.randn((f,), generator=g, device=dev) / np.sqrt(f)
                v = Fh[:m] @ b + noise((m,)) if m <= Fh.shape[0] else None
                if v is None:
                    kinds[q] = 2
                    kd = 2
                else:
                    ncol += 1
            if kd == 2:
                ii[q], jj[q], dd[q] = rng.integers(0, m), rng.integers(0, ncol), 0.005 * rng.standard_normal()
                continue
            pay.append(v.reshape(-1))
            offs[q], lens[q] = pos, v.numel()
            pos += v.numel()
    payload = torch.cat(pay) if pay else torch.zeros(1, device=dev)
    return panels, ns, ks, arr, who, kinds, offs, lens, ii, jj, dd, payload


def run_serving(args):
    """Serving loop with continuous batching: Poisson arrivals over many streams; every pass of the
    host loop submits the requests that have arrived since the previous pass (one submit, which the
    pool splits into ticks so that a stream's requests keep their order) and polls completion
    records. Latency of a request = its completion (device clock mapped to the host clock) minus its
    arrival time. The timed quantity is the whole run: requests / (last completion - first arrival)."""
    import torch

    import paper_2605_24514_gb300 as pkg
    from paper_2605_24514_gb300 import build as b

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    W = WORKLOADS["serving"]
    S = args.streams or W["streams"]
    N = args.requests or W["requests"]
    rate = args.rate or W["rate"]
    W = dict(W, rate=rate)
    t_setup = time.perf_counter()
    panels, ns, ks, arr, who, kinds, offs, lens, ii, jj, dd, payload = _serving_inputs(W, S, N, rank_seed(rank), torch)
    budget = int(W["budget_gb_per_20000"] * 2**30 * S / 20000)
    st = torch.cuda.Stream()
    pool = pkg.Pool(k_max=int(W["k_hi"]), hbm_budget_bytes=budget, stream=st.cuda_stream,
                    flags=pkg.POOL_COMPLETIONS, rank_every=W["rank_every"], tau_evr=W["tau_evr"])
    ids = np.full(S, -1, np.int64)
    cap_extra = np.bincount(who, minlength=S)
    for sidx in range(S):
        A0 = panels[sidx]
        m0, n0 = A0.shape
        try:
            ids[sidx] = pool.admit_device(A0, int(ks[sidx]), row_cap=m0 + int(cap_extra[sidx]) + 2,
                                          col_cap=n0 + int(cap_extra[sidx]) + 2)
        except pkg.IsvdError as e:
            if e.name != "EBUDGET":
                raise
    del panels
    admitted = ids >= 0
    keep = admitted[who]                       # requests of refused streams are dropped
    arr, who, kinds, offs, lens = arr[keep], who[keep], kinds[keep], offs[keep], lens[keep]
    ii, jj, dd = ii[keep], jj[keep], dd[keep]
    N = int(arr.size)
    op_t = np.dtype([("stream", np.int32), ("kind", np.int32), ("i", np.int64), ("j", np.int64),
                     ("delta", np.float64), ("off", np.int64), ("len", np.int64)])
    ops = np.zeros(N, op_t)
    ops["stream"], ops["kind"], ops["i"], ops["j"] = ids[who], kinds, ii, jj
    ops["delta"], ops["off"], ops["len"] = dd, offs, lens
    pool.sync()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    # Clock mapping: host monotonic ns = device globaltimer ns + offset, offset taken as the smallest
    # (host time a record was seen - its device stamp) over the run (records seen right away).
    done_dev = np.zeros(N, np.uint64)
    seen_host = np.zeros(N, np.int64)
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter_ns()
    i = n_done = 0
    submits = 0
    while n_done < N:
        now = (time.perf_counter_ns() - t0) * 1e-9
        j = int(np.searchsorted(arr, now, side="right"))
        if j > i:
            seg = ops[i:j]
            pool.submit_raw(seg.ctypes.data, j - i, payload.data_ptr(), int(payload.numel()), 1)
            submits += 1
            i = j
        rec = pool.poll()
        if rec.size:
            h = time.perf_counter_ns()
            q = rec["seq"]
            done_dev[q] = rec["done_ns"]
            seen_host[q] = h
            n_done += rec.size
            assert np.all(rec["status"] == 0), "device error in a served request"
    clk = clocks.stop()
    pool.sync()
    offset = int(np.min(seen_host - done_dev.astype(np.int64)))
    done_host = done_dev.astype(np.int64) + offset
    lat_us = (done_host - t0 - (arr * 1e9).astype(np.int64)) / 1e3
    span_s = (done_host.max() - t0) * 1e-9 - float(arr[0])
    value = N / span_s
    kk = np.array([pool.stream(int(x)).shape()[3] for x in ids[admitted]])
    out = {
        "metric": "iSVD updates/s and p50/p99 update latency at err ratio<=1.05 vs plain GPU form",
        "value": round(value, 1), "unit": "updates/s", "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": round(span_s * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (factor-model panels and requests drawn on the device)",
        "config": {"workload": "serving", "desc": W["desc"], "streams": S, "streams_admitted": int(admitted.sum()),
                   "hbm_budget_bytes": budget, "pool_bytes_used": pool.bytes_used, "requests": N,
                   "offered_rate_per_s": rate, "submits": submits,
                   "kind_mix": {k: int(np.sum(kinds == c)) for c, k in enumerate(("row", "col", "entry"))},
                   "latency_us": {"p50": round(float(np.percentile(lat_us, 50)), 1),
                                  "p99": round(float(np.percentile(lat_us, 99)), 1),
                                  "max": round(float(lat_us.max()), 1),
                                  "note": "arrival (Poisson schedule, host clock) to the op's completion record "
                                          "(device clock mapped to the host clock)"},
                   "k_final_mean": round(float(kk.mean()), 2) if kk.size else None,
                   "setup_s": round(setup_s, 1)},
        "gpu_launches": int(pool.launches),
        "clocks": clk,
    }
    pool.close()
    return out if rank == 0 else None


def _batched_sample(args, n_streams, ticks):
    """Streams of the batched workload for the CPU oracle (same generator, same seeds, the same
    rows: a stream's rows are drawn as one block of ``ticks`` rows, as on the GPU side)."""
    W = WORKLOADS["batched-4096"]
    rng = np.random.Generator(np.random.PCG64(rank_seed(0)))
    S = args.streams or W["streams"]
    ns = rng.integers(W["n_lo"], W["n_hi"] + 1, size=S)
    ks = rng.choice(np.asarray(W["ks"]), size=S)
    out = []
    for sidx in range(min(n_streams, S)):
        n = int(ns[sidx])
        A0, fm = streams.make_panel(2 * n, n, 5, seed=rank_seed(0) * 1_000_003 + sidx + 1)
        out.append((A0.astype(np.float32).astype(np.float64), fm.rows(ticks).astype(np.float32).astype(np.float64),
                    int(ks[sidx])))
    return out


def cpu_baseline_batched(args, ticks, sample_ids):
    """The oracle on a sample of the batched workload: the first streams, every tick the GPU ran
    (in tick order); returns the timing and the oracle's error ratio of each sampled stream."""
    import oracle
    data = _batched_sample(args, len(sample_ids), ticks)
    engines = [oracle.OracleISVD(A0, k, tol_rel=3e-6) for A0, _, k in data]
    t0 = time.perf_counter()
    for t in range(ticks):
        for (A0, rows, k), o in zip(data, engines):
            o.append_row(rows[t])
    el = time.perf_counter() - t0
    n = ticks * len(data)
    ratios = [o.metrics().frob_ratio for o in engines]
    return ({"value": round(n / el, 3), "unit": "updates/s", "cores": _blas_threads(), "kind": "oracle",
             "sample": f"{n} row appends: the first {len(data)} streams of the same workload over all {ticks} "
                       f"ticks the GPU ran, in tick order"}, ratios)


def oracle_policy(W):
    import oracle
    if "gamma" in W:
        return oracle.Policy(kind=oracle.POLICY_ERROR | oracle.POLICY_ANGLE, check_every=W["check_every"],
                             gamma=W["gamma"], theta_max=np.deg2rad(W["theta_deg"]))
    return oracle.Policy(kind=oracle.POLICY_PERIODIC, T_refresh=W["T_refresh"], check_every=W["check_every"])


def cpu_baseline(args, budget_s=15.0):
    """The oracle (as it stands) on a time-bounded prefix of the same stream."""
    import oracle
    W = WORKLOADS[args.workload]
    A0, ev, k = make_stream(args.workload, seed=0, n_events=4000)
    dt = np.float32 if W["prec"] == "fp32" else np.float64
    o = oracle.OracleISVD(A0.astype(dt).astype(np.float64), k, tol_rel=3e-6 if dt == np.float32 else 1e-10,
                          policy=oracle_policy(W))
    t0 = time.perf_counter()
    n = 0
    while n < len(ev) and time.perf_counter() - t0 < budget_s:
        kd = int(ev.kind[n])
        if kd == oracle.ENTRY:
            o.update_entry(ev.i[n], ev.j[n], ev.delta[n])
        else:
            o.apply(kd, ev.vector(n).astype(dt).astype(np.float64))
        n += 1
    el = time.perf_counter() - t0
    return {"value": round(n / el, 3), "unit": "updates/s", "cores": _blas_threads(), "kind": "oracle",
            "sample": f"first {n} events of the same stream (time budget {budget_s:.0f} s, policy checks included)"}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return int(max(th))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    """The oracle timed per step on a bounded sample of the same workload."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    import oracle
    W = WORKLOADS[args.workload]
    if args.workload.startswith("batched"):
        nst = args.ref_batch
        data = _batched_sample(args, nst, args.warmup + args.steps)
        engines = [oracle.OracleISVD(A0, k, tol_rel=3e-6) for A0, _, k in data]
        for t in range(args.warmup):
            for (A0, rows, k), o in zip(data, engines):
                o.append_row(rows[t])
        t0 = time.perf_counter()
        for t in range(args.warmup, args.warmup + args.steps):
            for (A0, rows, k), o in zip(data, engines):
                o.append_row(rows[t])
        el = time.perf_counter() - t0
        value = args.steps * len(data) / el
        sample = f"{len(data)} streams of the same workload per step (one row append each), {args.steps} steps"
        return {"impl": "reference", "metric": "iSVD updates/s and p50/p99 update latency at err ratio<=1.05 vs plain GPU form",
                "value": round(value, 3), "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded factor-model panels and rows)",
                "config": {"workload": args.workload, "desc": W["desc"], "events_per_step": len(data)},
                "cpu_baseline": {"value": round(value, 3), "unit": "updates/s", "cores": _blas_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": round(value, 3), "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
    if args.workload.startswith("tall"):
        cb = cpu_baseline_tall(W, args.k or W["k"], budget_s=args.cpu_budget)
        return {"impl": "reference", "metric": "iSVD updates/s of one tall stream, deferred rotations vs the plain form",
                "value": cb["value"], "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 50-factor model panel and updates)",
                "config": {"workload": args.workload, "desc": W["desc"]}, "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    Bref = args.ref_batch
    n_ev = (args.warmup + args.steps) * Bref
    A0, ev, k = make_stream(args.workload, seed=0, n_events=n_ev)
    dt = np.float32 if W["prec"] == "fp32" else np.float64
    o = oracle.OracleISVD(A0.astype(dt).astype(np.float64), k, tol_rel=3e-6 if dt == np.float32 else 1e-10,
                          policy=oracle_policy(W))

    def step(s):
        for e in range(s * Bref, (s + 1) * Bref):
            kd = int(ev.kind[e])
            if kd == oracle.ENTRY:
                o.update_entry(ev.i[e], ev.j[e], ev.delta[e])
            else:
                o.apply(kd, ev.vector(e).astype(dt).astype(np.float64))

    for s in range(args.warmup):
        step(s)
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        step(s)
    el = time.perf_counter() - t0
    value = args.steps * Bref / el
    cores = _blas_threads()
    sample = f"{Bref} events per step of the same stream, events {args.warmup * Bref}..{n_ev - 1}"
    return {"impl": "reference", "metric": "iSVD updates/s and p50/p99 update latency at err ratio<=1.05 vs plain GPU form",
            "value": round(value, 3), "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded factor-model panel and update stream)",
            "config": {"workload": args.workload, "desc": W["desc"], "events_per_step": Bref},
            "cpu_baseline": {"value": round(value, 3), "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="batched-4096", choices=list(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--ref-batch", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--streams", type=int, default=0)
    ap.add_argument("--plain-ticks", type=int, default=3)
    ap.add_argument("--lat-ticks", type=int, default=100)
    ap.add_argument("--acc-streams", type=int, default=8)
    ap.add_argument("--requests", type=int, default=0, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=0.0, help="serving: offered requests per second")
    ap.add_argument("--m", type=int, default=0, help="tall workload: initial rows")
    ap.add_argument("--n", type=int, default=0, help="tall workload: columns")
    ap.add_argument("--k", type=int, default=0, help="tall workload: working rank")
    ap.add_argument("--tc-rotations", action="store_true",
                    help="batched workload: rotate rank buckets 16 and 32 on the tensor cores")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload.startswith("batched"):
        out = run_batched(args)
    elif args.workload == "serving":
        out = run_serving(args)
    elif args.workload.startswith("tall"):
        out = run_tall(args)
    else:
        out = run_gb300(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
