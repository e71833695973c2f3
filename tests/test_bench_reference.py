"""The oracle arm of bench.py (`--impl reference`) on CPU: it prints one JSON
line with the headline metric, a cpu_baseline describing the run and an e2e
block with no copies, its claimed step time fits inside the process's own
wall clock, and under torchrun every rank but 0 exits without work."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, steps=2, warmup=3):
    env = dict(os.environ)
    env.update(env_extra)
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "sara64_fp64", "--steps", str(steps), "--warmup", str(warmup)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r, time.perf_counter() - t0


def test_reference_arm_line():
    r, wall = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "SDMM iters/s" and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("sara64_fp64")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the timed steps happened inside this process's lifetime
    assert d["ms_per_step"] * d["steps"] / 1e3 <= wall


def test_reference_arm_other_ranks_do_nothing():
    r, _ = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
