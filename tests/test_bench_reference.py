"""bench.py's reference arm (the oracle timed on the host cores) prints one JSON
line with the contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
                "cpu_baseline"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["higher_is_better"] is True and line["unit"] == "intersections/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert "workload" in line["config"]


def test_fill_mixed_equals_the_chunked_generator():
    """bench.py writes the headline workload chunk by chunk from a process
    pool; the result is the same array as the generator's own chunked form."""
    import multiprocessing as mp

    import numpy as np

    import bench
    from paper_2510_09892_gb300 import workloads as W
    n = W.CHUNK + 7
    A, B, z = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    with mp.get_context("spawn").Pool(2) as pool:
        bench.fill_mixed(pool, 1234, A, B, z)
    A2, B2, z2 = W.mixed_arcs(n, seed=1234)
    assert np.array_equal(A, A2) and np.array_equal(B, B2) and np.array_equal(z, z2)


def test_cpu_loop_rate_counts_every_hit():
    """The all-core FP64 loop splits the arcs over threads and counts the same
    hits as one serial call of the step reference."""
    import numpy as np

    import bench
    from oracle import steps
    from paper_2510_09892_gb300 import workloads as W
    A, B, z = W.uniform_arcs(5000, seed=3)
    c, _ = steps.direct(A, B, z)
    r = bench.cpu_loop_rate(steps.direct, A, B, z, threads=3, chunk=700)
    assert r["arcs"] == 5000 and r["cores"] == 3
    assert abs(r["value"] / r["arcs_per_s"] - np.clip(c, 0, None).sum() / 5000) < 1e-12
