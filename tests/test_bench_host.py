"""bench.py's host side on the CPU: the module parses and imports, the
reference arm (the oracle) prints one JSON line with the contract's keys on
the small workload, and the learned-skip sequence summary of hand records."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_imports_and_counts():
    sys.path.insert(0, ROOT)
    import bench
    assert set(bench.WORKLOADS) >= {"full", "small", "large"}
    assert bench.STAGES == list(bench.KERNELS_PER_STAGE)
    # fused decode+projection, 17 binning, forward + tile order, 4 loss, adjoint, gather, projection
    # adjoint, 2 decode adjoint, 2 Adam
    assert sum(bench.KERNELS_PER_STAGE.values()) == 28
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


def test_sequence_summary_of_hand_records():
    """The skip-frame summary: frames after the MLP's training frames only,
    s/frame of both arms, the PSNR differences against same-state plain
    training, fallbacks, and the static-set recall and precision of the
    skipped set and of the plain arm's zero gates."""
    from paper_2412_04469_gb300.sequence import FrameRecord, SequenceConfig, summarize
    cfg = SequenceConfig(frames=14, train_frames=10)
    plain = [FrameRecord(t=t, seconds=1.0 + 0.01 * t, psnr=30.0, gate0_recall=0.9 + 0.01 * (t > 10),
                         gate0_precision=0.8) for t in range(1, 14)]
    learned = [FrameRecord(t=t, seconds=1.0 if t <= 10 else 0.5, psnr=30.0 - 0.1 * (t == 12), psnr_plain=30.0,
                           psnr_train=31.0, psnr_plain_train=31.0 + 0.02 * (t == 13), fallback=t == 13,
                           skipped=0.25 * (t > 10), static_recall=0.6 if t > 10 else float("nan"),
                           static_precision=0.99 if t > 10 else float("nan")) for t in range(1, 14)]
    s = summarize(cfg, plain, learned)
    assert s["s_per_frame_plain_skip_frames"] == pytest.approx(1.12)           # frames 11, 12, 13
    assert s["s_per_frame_learned_skip_frames"] == pytest.approx(0.5)
    assert s["min_dpsnr_skip_frames"] == pytest.approx(-0.1) and s["min_dpsnr_train_skip_frames"] == pytest.approx(-0.02)
    assert s["fallbacks"] == 1 and s["mean_skipped"] == pytest.approx(0.25)
    assert s["static_recall"] == pytest.approx(0.6) and s["static_precision"] == pytest.approx(0.99)
    assert s["plain_gate0_recall"] == pytest.approx(0.91) and s["plain_gate0_precision"] == pytest.approx(0.8)


def test_reference_arm_times_fewer_whole_iterations_when_the_budget_is_short():
    """With a budget that cannot hold the K + W requested whole iterations,
    the reference arm times fewer of them (3 warm-up steps, at least 3 timed)
    and says so; the timed steps fit inside the run's own wall time."""
    import time
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small", "--steps", "500", "--warmup", "20", "--ref-budget", "0.01"],
                         capture_output=True, text=True, timeout=600, check=True)
    wall = time.perf_counter() - t0
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["steps"] == 3 and line["warmup"] == 3
    assert line["steps_requested"] == 500 and line["warmup_requested"] == 20 and "note" in line
    assert line["steps"] * line["ms_per_step"] * 1e-3 <= wall
    assert line["value"] == pytest.approx(1e3 / line["ms_per_step"], rel=1e-3)


def test_measured_traffic_is_reported_only_for_its_workload_and_sources(monkeypatch):
    import hashlib
    import os
    import bench
    srcs = bench.NCU_TRAFFIC["render_bwd"]["sources"]
    h = hashlib.sha256()
    for f in srcs:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    rec = {"workload": "full", "bytes": 123.0, "sources": srcs, "sha256": h.hexdigest()}
    monkeypatch.setitem(bench.NCU_TRAFFIC, "render_bwd", rec)
    assert bench.ncu_traffic("render_bwd", "full") == 123.0
    assert bench.ncu_traffic("render_bwd", "large") is None              # another workload
    assert bench.ncu_traffic("gather", "full") is None                   # no capture
    monkeypatch.setitem(bench.NCU_TRAFFIC, "render_bwd", dict(rec, sha256="0" * 64))
    assert bench.ncu_traffic("render_bwd", "full") is None               # the sources changed since
