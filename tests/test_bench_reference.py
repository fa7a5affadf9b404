"""bench.py --impl reference (the FP64 oracle timed on host cores) prints one JSON line
with the keys of the benchmark line: metric, unit and config match the GPU arm's, and
the line carries its cpu_baseline and an e2e object without host-device traffic."""
import json
import os
import subprocess
import sys

from conftest import ROOT


def _run(extra_env=None, gpus=1):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--gpus", str(gpus)], capture_output=True, text=True, timeout=300,
                          cwd=ROOT, env=env)


def test_reference_arm_prints_one_contract_line():
    res = _run()
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "sweeps/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("grid19_n2429_r49")
    # the config describes the sample each step actually times: its sweep count is the one
    # the step ran, and ms_per_step divided by it is the time per sweep
    import bench
    assert d["config"]["iters"] == bench.REFERENCE_ITERS
    assert d["config"]["sweeps_per_step"] == sum(bench._schedule_py(d["config"]["levels"], bench.REFERENCE_ITERS))
    assert abs(d["value"] - d["config"]["sweeps_per_step"] / (d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]
    assert "l2" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks():
    # launched like the GPU arm with two ranks: rank 1 exits 0 without work, rank 0 prints the
    # line with the same config as the GPU arm's (replicas)
    r1 = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, gpus=2)
    assert r1.returncode == 0 and not r1.stdout.strip()
    r0 = _run({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"}, gpus=2)
    assert r0.returncode == 0, r0.stderr[-2000:]
    d = json.loads([l for l in r0.stdout.splitlines() if l.strip().startswith("{")][0])
    assert d["n_gpus"] == 2 and d["config"]["parallelism"] == "replicas"
