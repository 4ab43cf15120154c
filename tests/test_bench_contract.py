"""The benchmark's bookkeeping on the CPU: the roofline arithmetic of the raster kernels and of the whole
step (the per-pair and per-Gaussian counts of the hot-path measurement plan), the scaling of the
committed DRAM-traffic record to a launch of the bench's size, and the reference arm's JSON line (the FP64
oracle on one full projection per step, here on a small cloud so that it runs in seconds)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_kernel_roofline_arithmetic():
    peaks = {"fp32_per_s": 40e12, "sfu_per_s": 6.7e12}
    # 1e9 pairs of the backward at 46 FP32 + 2 SFU each, in 2 ms: FP32-bound
    r = bench.kernel_roofline("raster_bwd", 1e9, 2.0, peaks)
    assert r["pipe"] == "fp32" and r["kernel"] == "k_raster_bwd"
    assert r["achieved"] == pytest.approx(46e9 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(46e9 / 2e-3 / 40e12)
    assert r["roofline_ms"] == pytest.approx(46e9 / 40e12 * 1e3)
    # with a slow SFU the SFU term binds
    r2 = bench.kernel_roofline("raster_fwd", 1e9, 1.0, {"fp32_per_s": 40e12, "sfu_per_s": 1e12})
    assert r2["pipe"] == "sfu" and r2["frac"] == pytest.approx(2e9 / 1e-3 / 1e12)


def test_step_work_counts():
    pairs, B, N, R, npix = 1e9, 16, 100_000, 3, 65536
    fp32, sfu, nbytes = bench.step_work(pairs, B, N, R, npix)
    assert fp32 == pytest.approx(pairs * (18 + 46) + B * N * 850 + N * 64 * 42 * R)
    assert sfu == pytest.approx(pairs * 4)
    assert nbytes == B * (2 * N * (11 + 12 * R) * 4 + 2 * npix * 4)


def test_traffic_record_scales_with_projections():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for k in ("k_raster_fwd", "k_raster_bwd"):
        base = bench.traffic_for(k, rec[k]["projections"], rec[k]["tile"], rec[k]["bwd_lanes"])
        if base is None:  # the kernel source changed since the capture: the bench reports null too
            continue
        assert base == pytest.approx(rec[k]["bytes_per_launch"])
        assert bench.traffic_for(k, 8 * rec[k]["projections"], rec[k]["tile"], rec[k]["bwd_lanes"]) == \
            pytest.approx(8 * base)
        assert bench.traffic_for(k, 128, rec[k]["tile"] * 2, rec[k]["bwd_lanes"]) is None


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "300"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["steps"] == 1 and line["warmup"] == 0
    assert line["unit"] == "projections/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
