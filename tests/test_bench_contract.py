"""The benchmark's JSON contract on the CPU: the reference arm (the FP64 oracle
timed on host cores) prints one line with the keys and units the GPU arm uses,
and the algorithmic bytes of a sweep follow their stated formula."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--scale", "12"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0 and d["vs_baseline"] is None
    assert "workload" in d["config"] and "scale 12" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the unit is nnz * R * k per second: value * seconds per step = nnz * R * k (k = 1 per step)
    nnz, R = d["config"]["nnz"], 32
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - nnz * R) <= 1e-6 * nnz * R


def test_algorithmic_bytes_of_a_sweep():
    import bench
    from paper_1601_05527_gb300 import graphgen
    g = graphgen.rmat(10, 8, seed=3)
    n_active = int((g.degrees() > 0).sum())
    for storage, s in (("fp32", 4), ("bf16", 2), ("fp16", 2)):
        b, na = bench.algorithmic_bytes_per_sweep(g, storage)
        assert na == n_active
        # column indices, row pointers, inverse degrees, one read and one write of each active row
        assert b == g.nnz * 4 + (g.n + 1) * 4 + g.n * 4 + 2 * n_active * bench.R * s
    assert np.isclose(bench.algorithmic_bytes_per_sweep(g, "fp32")[0] - bench.algorithmic_bytes_per_sweep(g, "bf16")[0],
                      2 * n_active * bench.R * 2)
