"""Host-side contracts that need no GPU: the build covers every CUDA translation unit, and the
bench's reference arm (the CPU oracle timed on a bounded sample) prints one well-formed JSON line,
once, also when launched as two ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_build_compiles_every_translation_unit():
    from paper_2605_24514_gb300 import build
    on_disk = sorted(f for f in os.listdir(build.CSRC) if f.endswith(".cu"))
    assert sorted(build.SOURCES) == on_disk
    assert len(set(build.SOURCES)) == len(build.SOURCES)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-batch", "4"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "batched-4096"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks on the host: rank 0 alone runs the reference arm and prints its line; the other
    rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--ref-batch", "4"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0


def test_tall_step_generator_matches_its_contract():
    """The tall workload's steps: entry updates inside the current shape, then one row of n
    columns; the row count grows by one per step."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_24514_gb300 import streams
    W = bench.WORKLOADS["tall-200000x20000"]
    f = W["f"]
    vol = 0.02 * 0.7 ** np.arange(f)
    Bl = np.random.default_rng(0).standard_normal((300, f)) / np.sqrt(f)
    steps = bench._tall_steps(W, 1000, 300, f, Bl, vol, 4, 1)
    per = W["entries_per_append"]
    for s, sl in enumerate(steps):
        assert len(sl) == per + 1
        assert (sl.kind[:per] == streams.ENTRY).all() and sl.kind[per] == streams.ROW
        assert (sl.i[:per] < 1000 + s).all() and (sl.j[:per] < 300).all()
        assert sl.vector(per).shape == (300,) and np.isfinite(sl.payload).all()
        assert sl.m_after[per] == 1000 + s + 1


def test_tall_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "tall-200000x20000", "--steps", "2", "--warmup", "3", "--cpu-budget", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"] == "tall-200000x20000"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
