"""bench.py's host side on the CPU: the module parses and imports, and the
reference arm (the oracle) prints one JSON line with the contract's keys on
the small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_imports_and_counts():
    sys.path.insert(0, ROOT)
    import bench
    assert set(bench.WORKLOADS) >= {"full", "small", "large"}
    assert bench.STAGES == list(bench.KERNELS_PER_STAGE)
    assert sum(bench.KERNELS_PER_STAGE.values()) == 31
    assert bench.workload_name("full") == "queen_residual_step_n300000_sh3_1352x1014_v20"


def test_reference_arm_prints_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small", "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
