"""The measurement contract on the CPU: the reference arm (the oracle timed on the host) prints
one JSON line with the keys the benchmark contract names, and the ensemble's input recipe
(C4) draws instances of the stated shapes."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == d["unit"] == "particle-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("streamer")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_refuses_fewer_than_three_warmup_steps():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_ensemble_recipe_shapes():
    sys.path.insert(0, ROOT)
    from paper_1604_07713_gb300 import workloads as W
    members = W.ensemble(256)
    nx = np.array([m[1]["nx0"] for m in members])
    ny = np.array([m[1]["ny0"] for m in members])
    assert len(members) == 256 and np.all(nx % 16 == 0) and nx.min() >= 64 and nx.max() <= 512
    assert np.all(ny == 16) and len(np.unique(nx)) > 10  # uneven sizes
    volts = np.array([m[0]["phi_left_amp"] for m in members])
    ng = np.array([m[0]["gas_density"] for m in members])
    assert volts.min() >= 100.0 and volts.max() <= 400.0
    assert ng.min() >= 3e20 * (1 - 1e-12) and ng.max() <= 3e21 * (1 + 1e-12)
    ppc = np.array([m[3] // (2 * m[1]["nx0"] * 16) for m in members])
    assert ppc.min() >= 20 and ppc.max() <= 200
    total = sum(m[3] for m in members)
    assert 2.0e8 < total < 3.2e8  # ~2.6e8 particles in all
    assert sorted(m[0]["instance"] for m in members) == list(range(256))
