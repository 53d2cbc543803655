"""The reference arm of bench.py (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys and the same config as the GPU arm;
under several ranks only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--ref-step-s", "0.5", *args]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    return [ln for ln in res.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_json_line():
    import argparse

    import bench
    import workloads as W
    lines = run(None, "--workload", "plain_box")
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    args = argparse.Namespace(workload="plain_box", rtol=1e-13, energy_rtol=1e-10, inner_rtol=1e-3,
                              inner_max=None, fcg_window=16, precond=None)
    assert d["config"] == json.loads(json.dumps(bench.bench_config(args, [W.plain_box()], 1)))


def test_reference_arm_prints_on_rank_zero_only():
    assert run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--workload", "plain_box") == []
