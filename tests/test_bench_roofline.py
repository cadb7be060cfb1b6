"""The bench's whole-step roofline (pure host arithmetic, no GPU): each launch record costs the
slower of flops / peak of its arithmetic and bytes / HBM rate; the must-move byte counts."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_path_roofline_sums_the_slower_side_of_each_record():
    import bench
    peaks = {"hbm_gbs": 1000.0, "bf16_tflops": 600.0, "src": "test"}  # tensor 3xTF32: 100 TFLOP/s
    trace = [
        {"kind": "gemm_tc", "flops": 1e12, "bytes": 1e9},   # 10 ms of tensor flops vs 1 ms of bytes
        {"kind": "fwd_class", "flops": 1e6, "bytes": 2e9},  # 2 ms of bytes
        {"kind": "gemm", "flops": bench.FP32_SIMT_PEAK_TFLOPS * 1e9, "bytes": 0.0},  # 1 ms at the FP32 rate
    ]
    info = {"n_dof": 1000, "nnz_lu": 1e6, "sum_cb": 2e6}
    r = bench.path_roofline(trace, 2, False, peaks, info, elem_bytes=1e6, nsolve=3, nrhs=1, ms_step=26.0)
    assert r["t_roof_ms"] == pytest.approx((10.0 + 2.0 + 1.0) / 2)
    assert r["frac"] == pytest.approx(6.5 / 26.0)
    # B_min: elements 4 times, factors written once and read 3 times (4 B each), vectors 8 B x (2 + 12) x n
    assert r["b_min_GB"] == pytest.approx((4e6 + 4.0 * 1e6 * 4 + 8.0 * 1000 * 14) / 1e9)
    assert r["b_sched_GB"] == pytest.approx(r["b_min_GB"] + 2 * 4.0 * 2e6 / 1e9)
    # FP64 fronts: the DFMA rate and 8-byte factors
    r64 = bench.path_roofline(trace[2:], 1, True, peaks, info, 1e6, 3, 1, 10.0)
    assert r64["t_roof_ms"] == pytest.approx(1e3 * bench.FP32_SIMT_PEAK_TFLOPS / bench.FP64_DFMA_TFLOPS / 1e3)
