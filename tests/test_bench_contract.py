"""bench.py's reference arm (the CPU oracle timed as it stands) prints one JSON
line with the keys the measurement contract names; runs on CPU in seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-samples", "2", "--P", "3", "--Q", "3", "--M", "16"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_every_workload_and_option_parses():
    """The argument parser accepts every workload and its options (CPU, no run)."""
    sys.path.insert(0, ROOT)
    import bench

    argv = sys.argv
    try:
        for extra in (["--workload", "kl", "--kl-n", "64", "--kl-S", "8", "--kl-chunk", "8"],
                      ["--workload", "uneven"], ["--workload", "serving"],
                      ["--workload", "ce", "--ce-S", "4", "--ce-batch", "2", "--ce-L", "7", "--ce-scale", "1",
                       "--ce-solve-S", "2"],
                      ["--workload", "estimator", "--est-S", "16"],
                      ["--workload", "convergence", "--conv-S", "4", "--conv-cycles", "5", "--conv-kmax", "4"]):
            sys.argv = ["bench.py"] + extra
            assert bench.parse().workload == extra[1]
    finally:
        sys.argv = argv
