"""Host logic of bench.py, without a GPU: the reference arm's JSON line (it
runs the oracle on the host cores), the clock-record parsing that decides
whether a run is rejected, the ALU work count of the RD line, and the oracle
sample helpers of the other workloads."""
import json
import os
import subprocess
import sys
import tempfile
import types

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("64 frames 1920x1080")


def test_defaults_meet_the_timing_rules():
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours" and a.workload == "frames"


def clock_summary(rows):
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    os.write(fd, "\n".join(rows).encode())
    os.close(fd)
    return s.summary()      # also removes the file


def test_clock_summary_reports_throttle_reasons():
    idle = "0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1890, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x20, Not Active, Active, Not Active, Not Active"
    s = clock_summary([idle, busy, busy, busy])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == [] and s["samples"] == 4
    s = clock_summary([busy, capped, capped, hot])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1890.0          # median of the loaded samples; the idle one is left out
    assert clock_summary([])["reasons"] == ["unavailable"]


def test_rd_ops_per_region_closed_form():
    # forward: per size 2 passes x 32 vectors x (32 / N) blocks x A(N) adds, A = 22, 60, 152 (T^);
    # per q the inverse of every size in int64 (two operations per add)
    fwd = 2 * 32 * (4 * 22 + 2 * 60 + 1 * 152)
    assert bench.rd_ops_per_region("hat", 3) == fwd * 7 == 161280


def test_oracle_sample_helpers():
    from paper_2207_11638_gb300 import synth, workload as wl
    args = types.SimpleNamespace(no_cpu_baseline=False, cpu_seconds=0.0)
    regs = synth.residual_regions_32(2, seed=4)
    b = bench.rd_baseline(args, regs, (8, 16, 32), "test regions")
    assert b["kind"] == "oracle" and b["value"] > 0 and "regions of test regions" in b["sample"]
    assert b["single_core"]["sample"].startswith("1 regions")
    args.no_cpu_baseline = True
    assert bench.rd_baseline(args, regs, (8,), "x") is None
    img = np.random.default_rng(1).integers(0, 256, (64, 96)).astype(np.uint8)
    gpx, k, secs = bench.oracle_images_sample([img, img], 0.0, wl.PASSES)
    assert k == 1 and gpx > 0


def test_nvml_summary_reports_reasons_and_load():
    s = object.__new__(bench.NvmlSampler)
    s.interval = 0.002
    s.rows = [(345.0, 2070.0, 120.0, 0x1), (2070.0, 2070.0, 900.0, 0x0), (1890.0, 2070.0, 1400.0, 0x4),
              (2070.0, 2070.0, 1000.0, 0x0)]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["samples_under_load"] == 3 and out["reasons"] == ["sw_power_cap"]
    s.rows.append((1500.0, 2070.0, 1300.0, 0x40 | 0x8))
    assert s.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    s.rows = []
    assert s.summary()["reasons"] == ["unavailable"]


def test_all_core_oracle_baseline_states_its_cores():
    frames = np.random.default_rng(2).integers(-255, 256, (3, 32, 48)).astype(np.int16)
    gpx, n, secs = bench.oracle_pool_sample(frames, 0.0, 2)
    assert gpx > 0 and n == 2
    cpu = bench.frames_cpu_baseline(frames, 0.0)
    assert cpu["cores"] == cpu["nproc"] == bench.host_cores() >= 1
    assert cpu["single_core"]["cores"] == 1 and cpu["single_core"]["value"] > 0 and cpu["value"] > 0


def test_all_core_rd_baseline_states_its_cores():
    from paper_2207_11638_gb300 import synth
    regions = synth.residual_regions_32(3, seed=4)
    gpx, n, secs = bench.oracle_rd_pool_sample(regions, (8, 16), 0.0, 2, per_task=1)
    assert gpx > 0 and n == 2
    cpu = bench.rd_baseline(types.SimpleNamespace(no_cpu_baseline=False, cpu_seconds=0.0), regions, (8, 16), "3 regions")
    assert cpu["cores"] == cpu["nproc"] == bench.host_cores() >= 1
    assert cpu["single_core"]["cores"] == 1 and cpu["single_core"]["value"] > 0 and cpu["value"] > 0


def test_all_core_images_baseline():
    imgs = [np.random.default_rng(k).integers(0, 256, (32 + 8 * k, 48)).astype(np.uint8) for k in range(3)]
    gpx, n, secs = bench.oracle_images_pool_sample(imgs, 0.0, 2)
    assert gpx > 0 and n == 2
