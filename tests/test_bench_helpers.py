"""Host-side helpers of bench.py: the roofline classification of a kernel and
the DRAM-traffic record, which is reported only for the kernel sources it was
measured on."""
import json

import pytest

import bench


def test_roofline_picks_the_bound_reached_first():
    # 1 GB moved and 1 GFLOP in 1 ms (1000 GB/s): HBM time 0.15 ms against 0.012 ms of FP32 -> HBM-bound
    r = bench.kernel_roofline("face_jvp_f32", 1, 1.0, 1e9, 1e9, 6800.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1000.0) and r["frac"] == pytest.approx(1000.0 / 6800.0)
    # FP64 kernel with many flops: ALU-bound against the FP64 peak
    r = bench.kernel_roofline("vol_res_f64", 2, 2.0, 1e6, 2e9, 6800.0)
    assert r["bound"] == "alu" and r["alu"] == "fp64" and r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["achieved"] == pytest.approx(1.0)
    # double-float kernels against the FP32 rate / 15
    r = bench.kernel_roofline("vol_res_df", 1, 1.0, 1e6, 1e9, 6800.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS / 15)


def test_traffic_record_matches_only_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    assert set(rec) >= {"csrc_hash", "kernels", "command"}
    if rec["csrc_hash"] == bench._csrc_hash():
        k = next(iter(rec["kernels"]))
        assert bench._traffic_for(k) == pytest.approx(rec["kernels"][k])
    monkeypatch.setattr(bench, "_csrc_hash", lambda: "0" * 16)
    assert bench._traffic_for(next(iter(rec["kernels"]))) is None
