"""Bookkeeping of bench.py on the CPU: algorithmic bytes, the traffic record's
source-hash check, the whole-job timing reduction at one rank, and the
reference arm's JSON line."""
import json
import os

import numpy as np

import bench
from workloads import banded_imdp


def test_algorithmic_bytes_formula():
    m = banded_imdp(100, 2, 100 * 2 * 10 + 1, seed=3)
    assert bench.algorithmic_bytes_per_iteration(m) == 20 * m.nnz + 12 * m.n_cols + 20 * m.n_states
    assert bench.algorithmic_bytes_per_iteration(m, "f32") == 12 * m.nnz + 16 * m.n_cols + 20 * m.n_states


def test_traffic_record_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "paper_2401_04068_gb300" / "csrc").mkdir(parents=True)
    for f in ("bellman.cu", "imdp_internal.h"):
        (root / "paper_2401_04068_gb300" / "csrc" / f).write_text("kernel " + f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.bellman_source_hash()
    rec = {"w": {"source_hash": h, "dram_bytes_per_launch": 123}, "old": {"source_hash": "0" * 16,
                                                                          "dram_bytes_per_launch": 9}}
    (root / "profiles" / "bellman_step_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("w") == 123
    assert bench.recorded_traffic("old") is None  # taken on another kernel source
    assert bench.recorded_traffic("missing") is None
    (root / "paper_2401_04068_gb300" / "csrc" / "bellman.cu").write_text("changed")
    assert bench.recorded_traffic("w") is None


def test_committed_traffic_record_is_well_formed():
    p = os.path.join(bench.ROOT, "profiles", "bellman_step_traffic.json")
    rec = json.load(open(p))
    for name, r in rec.items():
        assert len(r["source_hash"]) == 16 and r["dram_bytes_per_launch"] > 0
    assert np.isfinite(bench.measured_peak_hbm()[0])


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference runs the oracle on the host: one JSON line with the
    # keys the measurement contract names (a small batch and budget keep it short)
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--models", "32", "--ref-budget", "0.5"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "pendulum240_x4096" and d["config"]["models"] == 32
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_algorithmic_bytes_leave_out_fixed_states():
    # the reach targets' columns are read by no launch: their transitions,
    # columns and states leave the byte count
    m = banded_imdp(50, 2, 50 * 2 * 6 + 50 * 2 + 1, seed=3)
    full = bench.algorithmic_bytes_per_iteration(m)
    g = np.asarray(m.goal)
    ent = sum(int(m.colptr[m.stateptr[s + 1]] - m.colptr[m.stateptr[s]]) for s in g)
    cols = sum(int(m.stateptr[s + 1] - m.stateptr[s]) for s in g)
    assert bench.algorithmic_bytes_per_iteration(m, fixed=g) == full - 20 * ent - 12 * cols - 20 * len(g)
