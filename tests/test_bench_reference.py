"""The reference arm of bench.py (the CPU oracle timed on the host cores) on a small workload: one
JSON line with the contract's keys, its own figure as cpu_baseline and e2e, and nothing from ranks
other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "2", "--warmup", "1", "--n-laplace", "24", "--n-elasticity", "12"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *ARGS], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    out = _run({"RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == "GDoF/s"
    assert "Laplace 24^3" in d["config"]["workload"] and "elasticity 12^3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    out = _run({"RANK": "1"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_one_core_oracle_sample():
    """The one-core leg of cpu_baseline: the oracle's apply on bottom slabs of both workloads, its
    rate scaled by the full problems' free DoF per cell."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2308_09839_gb300 import inputs
    pL = inputs.cartesian_laplace_256(n=12)
    pE = inputs.cartesian_elasticity_160(n=6)
    rate, secs, desc = bench.oracle_sample_rate([pL, pE], [2, 1])
    assert rate > 0 and secs > 0
    assert "laplace 12x12x2 cells x1" in desc and "elasticity 6x6x1 cells x1" in desc
