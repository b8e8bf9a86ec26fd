"""The benchmark line's contract, checked on the CPU through the reference
arm (the oracle on the host cores), which shares the config object and the key
layout with the GPU arm."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _line("--impl", "reference", "--steps", "1", "--warmup", "1", "--oracle-rows", "65536",
              "--workload", "tall")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "TFLOP/s"
    cfg = d["config"]
    assert cfg["m"] == 1 << 23 and cfg["n"] == 128 and cfg["sampled_rows"] == 65536
    assert cfg["precision"] == "fp64" and cfg["parallelism"] == "single"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "65536" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_and_gpu_arms_share_the_config():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)

    class A:
        workload, variant, precision, inverse_depth, graph = "wide512", "fused", "ozaki", 0, False

    cfg = bench.workload_config(A, 1)
    assert cfg["m"] == 1 << 21 and cfg["n"] == 512 and cfg["variant"] == "plain"  # fusion is FP64-only
    assert bench.stage_work(1 << 20, 128, "fp64", True)["qform1"] == 2 * (1 << 20) * 128 * 129


def test_reference_arm_batch_workload():
    d = _line("--impl", "reference", "--steps", "1", "--warmup", "0", "--oracle-rows", "4", "--workload", "batch")
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "TFLOP/s"
    cfg = d["config"]
    assert cfg["m"] == 4096 and cfg["n"] == 32 and cfg["count"] == 1024 and cfg["sampled_problems"] == 4
    assert cfg["variant"] == "grouped" and cfg["precision"] == "fp64"
    assert d["cpu_baseline"]["kind"] == "oracle" and "4 of the 1024 problems" in d["cpu_baseline"]["sample"]


def test_small_inputs_are_timed_with_l2_flushed():
    """Inputs that fit in L2 (129 MB) would stay there between timed steps: the
    config (shared by both arms) says that a larger buffer is rewritten between
    steps; inputs larger than L2 say that none is."""
    small = _line("--impl", "reference", "--steps", "1", "--warmup", "1", "--workload", "small")
    assert "rewritten between steps" in small["config"]["l2"]
    tall = _line("--impl", "reference", "--steps", "1", "--warmup", "1", "--oracle-rows", "65536",
                 "--workload", "tall")
    assert "no flush" in tall["config"]["l2"] and "> 129 MB" in tall["config"]["l2"]
