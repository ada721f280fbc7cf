"""Host logic of bench.py that runs without a GPU: the reference arm's JSON line (the oracle on
the host cores, labelled with the N it ran) and the argument set the driver passes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["ms_per_step"] * d["value"] - 1000.0) < 1e-6 * 1000.0
    # the line names the size it ran, not the GPU arm's
    assert d["config"]["N"] == 4096 and "2^12" in d["metric"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_arguments():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--gpus", "2", "--steps", "7", "--warmup", "3", "--workload", "newton_bounded"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert (a.gpus, a.steps, a.warmup, a.workload, a.impl, a.N) == (2, 7, 3, "newton_bounded", "gb300", 20)
    cfg = bench.config(a)
    assert cfg["workload"] == "orbit_raising_newton_krylov_bounded_thrust" and cfg["N"] == 1 << 20
    assert cfg["barrier"]["form"] == "primal"
    assert "bounded thrust" in bench.metric_name(a)
