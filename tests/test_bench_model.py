"""The benchmark's FP64 operation model and peak lookup (no GPU)."""
import json
import os

from conftest import ROOT


def test_fp64_ops_per_launch_counts_the_kernel_arithmetic():
    import bench

    n, nnz = 2_097_152, 14_581_760  # level 0 of the 3D 7-point 128^3 workload
    # post-smoothing z = x + d (b - A x) with r.z: one FMA per entry, then b - s, d *, + x, r.z per row
    assert bench.fp64_ops_per_launch("relax_post", 0, n, nnz, "fp64") == nnz + 3 * n == 20_873_216
    # coarse levels carry no dot product
    assert bench.fp64_ops_per_launch("relax_post", 1, 100, 900, "fp64") == 900 + 2 * 100
    assert bench.fp64_ops_per_launch("relax_pre_residual", 0, n, nnz, "fp64") == nnz + n
    assert bench.fp64_ops_per_launch("pcg_Ap_dot", 0, n, nnz, "fp32") == nnz + n  # the outer loop stays FP64
    assert bench.fp64_ops_per_launch("pcg_vector", 0, n, nnz, "fp64") == 4 * n
    # FP32 cycles put no relaxation work on the FP64 pipe
    assert bench.fp64_ops_per_launch("relax_post", 0, n, nnz, "fp32") is None


def test_measured_peak_reads_the_driver_file():
    import bench

    peak, source = bench.measured_peak()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert source == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, source) == (6800.0, "fallback")


def test_ncu_traffic_summary_parses():
    import bench

    t = bench.ncu_traffic()
    rows, nnz, b = t["relax_post_L0"]
    assert (rows, nnz) == (2_097_152, 14_581_760) and b > 0
