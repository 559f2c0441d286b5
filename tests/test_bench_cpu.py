"""The bench's reference arm (the oracle on the host cores) keeps the JSON
contract on CPU: one line on rank 0, nothing on the other ranks, and a
bounded sample whatever --steps is."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=300, env=e, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


@pytest.mark.parametrize("workload", ["fluid", "ensemble", "adjoint"])
def test_reference_arm_prints_one_contract_line(workload):
    extra = ["--adj-n", "32"] if workload == "adjoint" else []
    lines = run_bench("--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "1",
                      "--cpu-n", "10", *extra)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["steps"] == 1 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    if workload == "adjoint":
        assert d["metric"] == bench.adjoint_metric(100)
    else:
        assert d["metric"] == bench.METRIC


def test_reference_arm_is_silent_on_other_ranks():
    lines = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-n", "10",
                      env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []


def test_reference_sample_shrinks_to_the_time_budget():
    B = bench.REFERENCE_BUDGET_S
    assert bench._bounded_n(32, B / 50, 50) == 32  # fits exactly
    n = bench._bounded_n(32, 10.0, 100)  # 1000 s of work at n = 32
    assert 10 <= n < 32
    assert 100 * 10.0 * (n / 32) ** 6 <= B  # cost ~ n^6
    assert 100 * 10.0 * ((n + 1) / 32) ** 6 > B
    assert bench._bounded_n(32, 1e6, 100) == 10  # never below the smallest valid lattice


def test_default_run_lengths_follow_the_workloads(monkeypatch):
    for argv, steps in ((["bench.py"], 1000), (["bench.py", "--workload", "ensemble"], 500),
                        (["bench.py", "--workload", "adjoint"], 5), (["bench.py", "--steps", "7"], 7)):
        monkeypatch.setattr(sys, "argv", argv)
        assert bench.parse().steps == steps
