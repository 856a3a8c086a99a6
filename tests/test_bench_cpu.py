"""bench.py's reference arm (the oracle on the host cores) and its JSON line, on CPU: rank 0 prints one line
with the contract's keys; another rank of a multi-rank launch does no work and prints nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "water8",
        "--steps", "2", "--warmup", "3"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run(ARGS, env=env, capture_output=True, text=True, timeout=600, check=True)


def test_reference_arm_prints_one_contract_line():
    out = _run({"WORLD_SIZE": "1", "RANK": "0"}).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    assert line["steps"] == 2 and line["warmup"] == 3 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("water8")


def test_reference_arm_other_ranks_do_nothing():
    res = _run({"WORLD_SIZE": "2", "RANK": "1"})
    assert res.stdout.strip() == ""
