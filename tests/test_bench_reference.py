"""bench.py --impl reference: the CPU oracle timed as the reference arm.

The line must be self-consistent and agree with a clock around the run: a
step is one bounded oracle sample, ms_per_step its measured time, and value
the full-size evaluations those samples stand for over that time.  Under
torchrun only rank 0 prints.
"""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra, steps=1, warmup=0):
    env = dict(os.environ, **env_extra)
    t0 = time.perf_counter()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", str(steps),
                        "--warmup", str(warmup)], env=env, capture_output=True, text=True, timeout=600)
    return p, time.perf_counter() - t0


def test_reference_line_matches_its_clock():
    p, wall = run({}, steps=2)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["higher_is_better"] is True
    for key in ("metric", "unit", "config", "cpu_baseline", "e2e", "ms_per_step", "evals_per_step"):
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    # value = full-size evaluations per step over the measured step time
    rate = line["evals_per_step"] / (line["ms_per_step"] / 1000.0)
    assert abs(rate - line["value"]) <= 1e-9 * line["value"]
    # the timed steps fit inside the process's own wall time
    assert line["steps"] * line["ms_per_step"] / 1000.0 <= wall
    assert 0 < line["evals_per_step"] < 1


def test_reference_other_ranks_print_nothing():
    p, _ = run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
