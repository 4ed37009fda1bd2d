"""The benchmark's reference arm (the CPU oracle timed on a bounded sample of
the workload) runs without a GPU: one JSON line with the arm's keys on
rank 0, nothing on the other ranks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, rank=0):
    env = dict(os.environ, RANK=str(rank))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", *args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    return [l for l in p.stdout.splitlines() if l.strip()]


@pytest.mark.parametrize("args,dtype", [
    (["--trees", "16", "--target", "100000"], "f32"),
    (["--workload", "uneven", "--funcset", "mux11", "--trees", "64", "--target", "20000"], "u64"),
    (["--workload", "uneven", "--funcset", "int32", "--trees", "64", "--target", "20000"], "i32"),
])
def test_reference_arm_prints_one_line(args, dtype):
    import bench
    lines = _run(args)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GPop/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"], d["dtype"]) == (2, 1, 1, dtype)
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GPop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert _run(["--trees", "16", "--target", "100000"], rank=1) == []
