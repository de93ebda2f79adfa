"""bench.py's entry points exist and its reference arm runs on one rank
(the GPU arm is exercised by the GPU runs of bench.py itself)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_flags_resolve_to_functions():
    import bench
    for name in ("stability_map", "accuracy", "cpu_baseline", "batched_vs_loop", "run_reference",
                 "measured_traffic", "workload_config", "max_over_ranks", "job_mlups", "time_steps"):
        assert callable(getattr(bench, name)), name


def test_reference_arm_one_rank():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
