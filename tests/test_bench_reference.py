"""bench.py's reference arm (--impl reference): the oracle timed on the host
cores, one JSON line with the keys of the bench contract (CPU only; one
128 x 128 oracle step, scaled to the 1024 x 1024 metric by the node ratio)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip()


def test_reference_line_has_the_contract_keys():
    lines = run().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1
    # ms_per_step is the wall time of one sampled step; value scales its rate by the node ratio
    ratio = (d["config"]["sampled_n"] + 1) ** 2 / (d["config"]["n"] + 1) ** 2
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - ratio) < 1e-3 * ratio
    assert d["config"]["workload"] == "film1024_mixed" and d["config"]["sampled_n"] < d["config"]["n"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == ""
