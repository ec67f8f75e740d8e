"""The benchmark's JSON line contract, checked on the CPU through the reference
arm (the oracle on a bounded sample): one line with the metric, value, unit,
step counts, the reference marker and the CPU-baseline and end-to-end objects."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "moves/s" and d["higher_is_better"] is True and d["steps"] == 1
    assert d["value"] > 0 and d["config"]["workload"].startswith("n70_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_local_search_busy_time_is_the_union_of_the_launch_intervals():
    """The benchmark's kernel time when launches of several runs overlap: the
    length of the union of their [start, end] intervals."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.union_ms([]) == 0.0
    assert bench.union_ms([(0, 1), (2, 3)]) == 2.0                    # disjoint: the sum
    assert bench.union_ms([(0, 4), (1, 2), (3, 5)]) == 5.0             # nested and chained
    assert bench.union_ms([(3, 5), (0, 1), (0.5, 3)]) == 5.0           # order does not matter
    assert bench.union_ms([(1, 1), (2, 1.5)]) == 0.0                   # empty intervals
    import random
    rnd = random.Random(5)
    iv = [(a, a + rnd.uniform(0, 3)) for a in (rnd.uniform(0, 20) for _ in range(40))]
    grid = [k * 0.001 for k in range(26000)]
    covered = sum(1 for t in grid if any(a <= t < b for a, b in iv)) * 0.001
    assert abs(bench.union_ms(iv) - covered) < 0.05
