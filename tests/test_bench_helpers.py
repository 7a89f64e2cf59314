"""Host-side helpers of bench.py: the roofline classification of a kernel and
the DRAM-traffic record, which is reported only for the kernel sources it was
measured on."""
import json

import pytest

import bench


PEAKS = {"fp64": 1.2, "fp32": 77.0, "df": 77.0 / 15}


def test_roofline_picks_the_bound_reached_first():
    # 1 GB moved and 1 GFLOP in 1 ms (1000 GB/s): HBM time 0.15 ms against 0.013 ms of FP32 -> HBM-bound
    r = bench.kernel_roofline("face_jvp_f32", 1, 1.0, 1e9, 1e9, 6800.0, PEAKS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1000.0) and r["frac"] == pytest.approx(1000.0 / 6800.0)
    # FP64 kernel with many flops: ALU-bound against the FP64 peak
    r = bench.kernel_roofline("vol_res_f64", 2, 2.0, 1e6, 2e9, 6800.0, PEAKS)
    assert r["bound"] == "alu" and r["alu"] == "fp64" and r["peak"] == pytest.approx(1.2)
    assert r["achieved"] == pytest.approx(1.0)
    # double-float kernels against the FP32 rate / 15
    r = bench.kernel_roofline("vol_res_df", 1, 1.0, 1e6, 1e9, 6800.0, PEAKS)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(77.0 / 15)


def test_survey_roofline_charges_the_operator_bytes():
    """The survey's bytes: 3 N s per JVP evaluation, 2 N s per residual, charged
    to each launch of a kernel of that operator."""
    N = 1_000_000
    r = bench.survey_roofline("face_jvp_f32", 10, 2.0, N, 6800.0)      # 0.2 ms a launch
    assert r["operator"] == "jvp" and r["bytes_per_launch"] == 3 * N * 4
    assert r["achieved"] == pytest.approx(3 * N * 4 / 0.2e-3 / 1e9)
    r = bench.survey_roofline("vol_res_df", 1, 1.0, N, 6800.0)
    assert r["operator"] == "residual" and r["bytes_per_launch"] == 2 * N * 8
    assert bench.survey_roofline("arnoldi_dot", 1, 1.0, N, 6800.0)["frac"] is None
    r = bench.survey_roofline("arnoldi_update", 2, 1.0, N, 6800.0, nbytes=2 * 8 * 3 * N)   # 0.5 ms a launch
    assert r["bytes_per_launch"] == 8 * 3 * N and r["achieved"] == pytest.approx(8 * 3 * N / 0.5e-3 / 1e9)
    assert bench._operator_of("trace_f32") == ("jvp", 4) and bench._operator_of("trace_f64") == ("residual", 8)
    assert bench._operator_of("fused_jvp_f32") == ("jvp", 4) and bench._operator_of("ctrace_f32") == ("jvp", 4)
    # both compact face kernels of the FP32 JVP charge the JVP's bytes
    assert bench._operator_of("cface_jvp_f32") == ("jvp", 4) and bench._operator_of("cface_vt_jvp_f32") == ("jvp", 4)


def test_double_float_instruction_count_matches_dfma():
    """The 15 FP32 instructions a double-float FMA is charged (the divisor of the
    double-float ALU peak) are the operations dfma in dfloat.cuh performs."""
    import re
    src = open(bench.os.path.join(bench.ROOT, "paper_1910_03693_gb300", "csrc", "dfloat.cuh")).read()
    body = lambda name: src[src.index(name):].split("\n}\n", 1)[0]
    ops = lambda txt: len(re.findall(r"__f(?:add|sub|mul|maf)_rn\(", txt))
    n = ops(body("__device__ __forceinline__ dfloat dfma(")) + ops(body("__device__ __forceinline__ void two_sum(")) \
        + ops(body("__device__ __forceinline__ void fast_two_sum("))
    assert n == bench.DF_FP32_INSTRUCTIONS_PER_FMA


def test_traffic_record_matches_only_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    assert set(rec) >= {"csrc_hash", "kernels", "command"}
    if rec["csrc_hash"] == bench._csrc_hash():
        k = next(iter(rec["kernels"]))
        assert bench._traffic_for(k) == pytest.approx(rec["kernels"][k])
    monkeypatch.setattr(bench, "_csrc_hash", lambda: "0" * 16)
    assert bench._traffic_for(next(iter(rec["kernels"]))) is None
