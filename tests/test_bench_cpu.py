"""Roofline arithmetic of bench.py (host logic, no GPU): the top class, the
closer roof, the fraction, the traffic taken from the measured DRAM ratio of
the same kernel, and the per-class rates."""
import numpy as np

import bench


def test_alu_bound_class_and_its_traffic():
    # cell solves on the FP32 pipes: 4 launches of 30 ms, 240 GB and 3.2 TFLOP per step in all
    kt_ms = np.array([120.0, 20.0, 80.0])
    kt_n = np.array([4, 700, 1500])
    kt_b = np.array([240e9, 10e9, 400e9])
    kt_f = np.array([3.2e12, 0.2e12, 1.0e12])
    roof = bench.roofline(kt_ms, kt_n, kt_b, kt_f, 260.0, 1, True, False, "layered2000x4000")
    assert roof["kernel"] == "cell_chain" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["achieved"] - 3.2e12 / 0.120 / 1e12) < 1e-3 * roof["achieved"]
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-3 * roof["frac"]
    ratio = bench.DRAM_PER_ALGO[("cell_chain", "layered2000x4000", "simt")][0]
    assert roof["traffic"] == round(ratio * 240e9 / 4)
    assert "frac_tensor_3xtf32" not in roof["classes"]["cell_chain"]  # not on the tensor cores
    assert abs(roof["share_of_step"] - 120.0 / 260.0) < 1e-3
    c = roof["classes"]["batched_fes_gemm"]
    assert abs(c["gb_s"] - 400e9 / 0.080 / 1e9) < 0.1 and c["launches_per_step"] == 1500


def test_hbm_bound_class_without_a_capture():
    kt_ms = np.array([1.0, 0.5, 10.0])
    kt_n = np.array([1, 1, 100])
    kt_b = np.array([1e9, 1e8, 60e9])     # 6 TB/s
    kt_f = np.array([1e10, 1e9, 1e11])    # 10 TFLOP/s
    roof = bench.roofline(kt_ms, kt_n, kt_b, kt_f, 12.0, 1, True, True, "smooth1024")
    assert roof["kernel"] == "batched_fes_gemm" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["traffic"] is None  # no DRAM capture of this kernel on this workload
    assert "frac_tensor_3xtf32" in roof["classes"]["cell_chain"]


def test_traffic_sources_name_no_files():
    for ratio, src in bench.DRAM_PER_ALGO.values():
        assert 0.5 < ratio < 2.0
        assert "/" not in src and ".md" not in src
