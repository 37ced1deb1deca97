"""Host-side arithmetic of bench.py's roofline objects: the per-kernel table
of the trace, the algorithmic work per launch of each product kernel, and
the achieved / peak fractions (no GPU involved)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_table_orders_and_normalises():
    trace = {"a": (10, 30.0), "b": (4, 10.0), "c": (1, 60.0)}
    kt = bench.kernel_table(trace, 2)
    assert list(kt) == ["c", "a", "b"]
    assert kt["a"]["launches_per_step"] == 5 and kt["a"]["ms_per_step"] == 15.0
    assert kt["a"]["ms_per_launch"] == 3.0
    assert abs(sum(v["share_of_traced"] for v in kt.values()) - 1.0) < 1e-12


def _work():
    # two dense leaves (one mirrored pair: only the upper one is evaluated)
    # and made-up matrix sizes
    mi = {"u_entries": 1000, "lr_entries": 2500, "dense_entries": 800, "mean_rank": 2.0, "aca_entries": 3000}
    ti = {"n_adm": 10, "n_clusters": 15}
    leaves = np.array([[0, 20, 20, 40], [20, 40, 0, 20]], dtype=np.int64)
    return bench.algorithmic_work(mi, ti, leaves, 40)


def test_algorithmic_work_counts():
    w = _work()
    # FP64 product: 2 flops per stored entry
    assert w["row_kernel.f64"] == ("alu", 2.0 * (800 + 1000), "flop")
    assert w["col_kernel.f64"] == ("alu", 2.0 * 1500, "flop")
    # FP32 row kernel: 4 B per entry + 4 B per gathered x / t value + 8 B per y
    K = 2.0 * 10
    assert w["row_kernel.f32"][1] == 4.0 * 1800 + 4.0 * (40 + K) + 8.0 * 40
    # entry evaluations: one per upper dense entry, 49 pairs each
    assert w["nearfield_kernel"][1] == 20 * 20 * bench.PAIRS_PER_ENTRY * bench.FF_FLOPS_PER_PAIR
    assert w["nearfield_kernel.f64"][1] == 20 * 20 * bench.PAIRS_PER_ENTRY * bench.FLOPS_PER_PAIR
    assert w["aca_kernel"][1] == 3000 * bench.PAIRS_PER_ENTRY * bench.FF_FLOPS_PER_PAIR


def test_roofline_entry_fractions():
    w = _work()
    peaks = {"hbm_gbs": 6000.0}
    kt = {"ms_per_launch": 2.0, "launches_per_step": 3.0}
    r = bench.roofline_entry("row_kernel.f32", kt, w["row_kernel.f32"], peaks, "measured")
    assert r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(w["row_kernel.f32"][1] / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    r = bench.roofline_entry("row_kernel.f64", kt, w["row_kernel.f64"], peaks, "measured")
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS
    # traffic only for the workload and kernel source of the recorded capture
    assert r["traffic"] is None
    r = bench.roofline_entry("row_kernel.f64", kt, w["row_kernel.f64"], dict(peaks, workload="precision"), "m")
    tr = bench.TRAFFIC["row_kernel.f64"]
    same_source = bench._file_sha(tr["source"]) == tr["sha256"]
    assert r["traffic"] == (tr["bytes_per_launch"] if same_source else None)
    r = bench.roofline_entry("aca_kernel", kt, w["aca_kernel"], peaks, "measured")
    assert r["peak"] == bench.FP32_PEAK_TFLOPS
    assert r["kernel_evaluations_per_s"] == pytest.approx(3000 * bench.PAIRS_PER_ENTRY / 2e-3)


def test_measured_alu_peaks_are_the_denominators():
    w = _work()
    peaks = {"hbm_gbs": 6000.0, "fp64_tflops": 1.0, "fp32_tflops": 70.0}
    kt = {"ms_per_launch": 2.0, "launches_per_step": 1.0}
    r = bench.roofline_entry("row_kernel.f64", kt, w["row_kernel.f64"], peaks, "measured")
    assert r["peak"] == 1.0 and "measured" in r["peak_source"]
    assert r["frac"] == pytest.approx(2.0 * 1800 / 2e-3 / 1e12)
    r = bench.roofline_entry("nearfield_kernel", kt, w["nearfield_kernel"], peaks, "measured")
    assert r["peak"] == 70.0


def test_multi_rhs_product_bytes():
    w = _work()
    K = 2.0 * 10
    # 16 right-hand sides: X / t rows as BF16 pairs (64 B), output rows into the FP32 Krylov block (64 B)
    assert w["row_mrhs_kernel.f32"] == ("hbm", 4.0 * 1800 + 64.0 * (40 + K) + 64.0 * 40, "byte")
    assert w["row_mrhs_kernel.bf16"][1] == 4.0 * 800 + 2.0 * 1000 + 64.0 * (40 + K) + 64.0 * 40
    assert w["col_bcp_kernel.f32"][1] == 4.0 * 1500 + 64.0 * (40 + K)
    assert w["col_bcp_kernel.bf16"][1] == 2.0 * 1500 + 64.0 * (40 + K)


def test_multi_rhs_product_bytes_with_bf16_tails():
    # FP32 factors with BF16 tails: 400 of the 1000 U entries and 600 of the
    # 1500 W entries are trailing terms (2 bytes); 8 of the 20 terms of t
    mi = {"u_entries": 1000, "lr_entries": 2500, "dense_entries": 800, "mean_rank": 2.0, "aca_entries": 3000,
          "u_tail_entries": 400, "lr_tail_entries": 1000, "factor_tail_terms": 8}
    ti = {"n_adm": 10, "n_clusters": 15}
    leaves = np.array([[0, 20, 20, 40], [20, 40, 0, 20]], dtype=np.int64)
    w = bench.algorithmic_work(mi, ti, leaves, 40)
    K = 2.0 * 10
    assert w["row_mrhs_kernel.f32"][1] == 4.0 * (800 + 600) + 2.0 * 400 + 64.0 * (40 + K) + 64.0 * 40
    assert w["col_bcp_kernel.f32"][1] == 4.0 * 900 + 64.0 * (40 + K - 8)
    assert w["col_bcp_kernel.bf16"][1] == 2.0 * 600 + 64.0 * (40 + 8)


def test_dominant_kernel_is_the_longest_with_known_work():
    mi = {"u_entries": 1000, "lr_entries": 2500, "dense_entries": 800, "mean_rank": 2.0, "aca_entries": 3000}
    ti = {"n_adm": 10, "n_clusters": 15}
    leaves = np.array([[0, 20, 20, 40], [20, 40, 0, 20]], dtype=np.int64)
    trace = {"batch_dots": (100, 500.0), "row_mrhs_kernel.f32": (10, 300.0), "aca_kernel": (1, 100.0)}
    dom, others, kernels = bench.rooflines(trace, 1, mi, ti, leaves, 40, {"hbm_gbs": 6000.0}, "measured")
    assert dom["kernel"] == "row_mrhs_kernel.f32"
    assert set(others) == {"aca_kernel"}
    assert list(kernels) == ["batch_dots", "row_mrhs_kernel.f32", "aca_kernel"]


def test_cpu_oracle_sample_estimate_runs_on_a_small_mesh():
    import meshgen
    V, T = meshgen.icosphere(3)
    W = dict(leaf_size=32, eta=1.5, ss_order=8, aca_eps=1e-6, aca_kmax=64)
    est, wall, sample, parts = bench.cpu_oracle_step("test_level3", V, T, W, 2, 10, dense_sample=50)
    assert est > 0 and wall > 0
    assert abs(est - (parts["tree_s"] + parts["nearfield_s"] + parts["aca_s"] + parts["solve_s"])) < 1e-9 * est
    assert "2 systems x 10 Arnoldi steps" in sample
