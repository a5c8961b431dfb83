"""bench.py's roofline and error arithmetic, on the CPU.

The bench line's fractions are only as good as the counts behind them: the
GEMM's useful FLOP are 2 B rows K over the distinct rows of Eq. 2.12 (the
executed ones eight products over rows - 1 operator rows and the padded K of
the split path), its algorithmic bytes the operator and input planes read once
and G written once; the transform's operation count is the double-float FFT
of length M/4 plus its pre- and post-processing.  These tests recompute them
from the sizes by hand and check the derived fields (achieved, frac, bytes).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}


def test_split_gemm_roofline_counts():
    B, rows, K, Kp, ms = 256, 8193, 8193, 8224, 0.168
    r = bench.gemm_roofline(B, rows, K, Kp, "split_fp16", ms, PEAKS, "test", {}, "w")
    useful = 2.0 * B * rows * K
    executed = 8 * 2.0 * B * (rows - 1) * Kp
    nbytes = 3 * (rows - 1) * Kp * 2 + 7 * B * Kp * 2 + B * rows * 8
    assert r["flops_per_launch"] == useful and r["executed_flops_per_launch"] == executed
    assert r["algorithmic_bytes_per_launch"] == nbytes
    assert np.isclose(r["achieved"], useful / (ms / 1e3) / 1e12)
    assert np.isclose(r["frac"], r["achieved"] / 2000.0) and r["bound"] == "tensor"
    assert np.isclose(r["executed_frac"], executed / (ms / 1e3) / 1e12 / 2000.0)
    assert np.isclose(r["hbm_frac"], nbytes / (ms / 1e3) / 1e9 / 6000.0)
    assert r["traffic"] is None


def test_simt_gemm_roofline_uses_the_alu_peak():
    r = bench.gemm_roofline(4096, 1025, 1025, 1056, "f32", 0.2, PEAKS, "test", {("abel_gemm", "f32", "w"): 7}, "w")
    assert r["bound"] == "alu" and np.isclose(r["peak"], 152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["executed_flops_per_launch"] == 2.0 * 4096 * 1025 * 1056 and r["traffic"] == 7


def test_transform_operation_counts():
    M, N = 16384, 4096
    H = M // 4
    lg = 12
    # the FFT: (H/2) lg radix-2 butterflies of 6 add + 4 mul; double-float add 8, mul 4 FP32 ops
    fft_adds, fft_muls = 6 * (H // 2) * lg, 4 * (H // 2) * lg
    sine = bench.dst_fp32_ops(M, N)
    assert sine == 8 * (fft_adds + 14 * H) + 4 * (fft_muls + 8 * H + 2 * N)
    assert bench.dst_fp32_ops(M, N, fp64=True) == fft_adds + 14 * H + fft_muls + 8 * H + 2 * N
    even = bench.fft_fp32_ops(M, N)
    L = M // 2
    assert even == 8 * (fft_adds + 3.5 * L + 8 * H + H + N) + 4 * (fft_muls + 2.5 * L + 4 * H + N)


def test_transform_roofline_bounds():
    B, M, N, rows, ms = 256, 16384, 4096, 8193, 0.03
    r = bench.fft_roofline(B, M, N, rows, "split_fp16", ms, PEAKS, "test", {}, "w", sine=True)
    assert r["bound"] == "alu" and np.isclose(r["ops_per_launch"], bench.dst_fp32_ops(M, N) * B)
    assert np.isclose(r["frac"], r["achieved"] / bench.ALU_PEAK_TOPS["f32"])
    assert r["bytes_per_launch"] == B * rows * 8 + B * N * 4
    f = bench.fft_roofline(4096, 2048, 512, 1025, "f32", 0.0166, PEAKS, "test", {}, "w", sine=True)
    assert f["bound"] == "hbm" and f["unit"] == "GB/s"
    assert f["bytes_per_launch"] == 4096 * 1025 * 4 + 4096 * 512 * 4
    assert np.isclose(f["frac"], f["bytes_per_launch"] / 0.0166e-3 / 1e9 / 6000.0)


def test_relative_error_is_per_function_then_max():
    ref = np.array([[1.0, -2.0, 0.5], [10.0, 0.0, 0.0]])
    c = ref + np.array([[0.0, 2e-6, 0.0], [0.0, 0.0, 3e-5]])
    assert np.isclose(bench.relerr(c, ref), max(2e-6 / 2.0, 3e-5 / 10.0))


def test_sample_rows_cover_every_tile_edge():
    idx = bench.sample_rows(300, 128, 5, 1)
    for t0 in range(0, 300, 128):
        assert t0 in idx and min(300, t0 + 128) - 1 in idx
    assert len(idx) == 6 + 5 and len(set(idx.tolist())) == len(idx)
