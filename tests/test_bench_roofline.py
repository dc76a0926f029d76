"""Host logic of bench.py's roofline object (CPU): which kernel is reported,
and the arithmetic of achieved / peak / frac from a synthetic solve record."""
import math

import bench

PEAKS = {"hbm_gbs": 6794.5, "bf16_tflops_sustained": 1719.1, "sm_max_mhz": 2070.0}
N, N_TETS = 21024, 10368


def _last(far_ms=65.0, tc_ms=40.0, mv_ms=50.0, pc_ms=23.7):
    return {
        "k_far_tt_ms": far_ms,
        "k_tc_n": 80, "k_tc_ms": tc_ms, "k_tc_bytes": 1.49e11, "k_tc_flops": 3.7e13,
        "k_matvec_n": 93, "k_matvec_ms": mv_ms,
        "k_precond_ms": pc_ms, "k_precond_bytes": 95 * 1.18e9, "k_precond_n": 95,
    }


def test_dominant_kernel_is_the_largest_device_time():
    dom, allr = bench.roofline(_last(), N, PEAKS, 1, N_TETS)
    assert set(allr) == {"k_far_tt", "k_tc_update", "k_matvec"}
    assert dom["kernel"] == "k_matvec"               # 50 + 23.7 ms > 65 ms > 40 ms
    assert math.isclose(dom["total_ms"], 73.7)
    dom2, _ = bench.roofline(_last(far_ms=90.0), N, PEAKS, 1, N_TETS)
    assert dom2["kernel"] == "k_far_tt"


def test_matvec_bytes_and_fraction():
    _, allr = bench.roofline(_last(), N, PEAKS, 1, N_TETS)
    m = allr["k_matvec"]
    ld = (N + 3) // 4 * 4
    per_z = N * ld * 8 + N * 2 * 8 * 2            # FP32 Z and the two complex vectors
    assert m["algorithmic_bytes_per_z_product"] == per_z
    ach = (93 * per_z + 95 * 1.18e9) / (73.7e-3) / 1e9
    assert math.isclose(m["achieved"], ach, rel_tol=1e-12)
    assert math.isclose(m["frac"], ach / 6794.5, rel_tol=1e-12)
    assert m["bound"] == "hbm" and m["unit"] == "GB/s"
    assert m["traffic"] == bench.MATVEC_Z_TRAFFIC   # captured on this workload only
    _, other = bench.roofline(_last(), 8910, PEAKS, 1, 4374)
    assert other["k_matvec"]["traffic"] is None


def test_far_kernel_against_the_issue_rate():
    _, allr = bench.roofline(_last(), N, PEAKS, 1, N_TETS)
    f = allr["k_far_tt"]
    vals = 16.0 * N_TETS * N_TETS
    peak = 152 * 4 * 2070e6 / 1e9                   # G warp instructions / s
    assert f["bound"] == "alu" and math.isclose(f["peak"], peak)
    winst, flops, _ = bench.FAR_COUNTS["normal"]
    assert math.isclose(f["achieved"], winst * vals / 65e-3 / 1e9, rel_tol=1e-12)
    assert 0.0 < f["frac"] < 1.0
    assert math.isclose(f["fp32_tflops"], flops * vals / 65e-3 / 1e12, rel_tol=1e-12)


def test_far_kernel_counts_left_out_for_another_split(monkeypatch):
    monkeypatch.setattr(bench, "FAR_SPLIT_CHOSEN", 1.75)
    _, allr = bench.roofline(_last(), N, PEAKS, 1, N_TETS)
    assert "k_far_tt" not in allr


def test_products_take_the_binding_roof():
    _, allr = bench.roofline(_last(), N, PEAKS, 1, N_TETS)
    t = allr["k_tc_update"]
    t_hbm = 1.49e11 / 6794.5e9
    t_tc = 3.7e13 / 1719.1e12
    assert t["bound"] == ("tensor" if t_tc > t_hbm else "hbm")
    # a flop-heavier record binds on the tensor rate
    last = _last()
    last["k_tc_flops"] = 3.0e14
    _, allr2 = bench.roofline(last, N, PEAKS, 1, N_TETS)
    t2 = allr2["k_tc_update"]
    assert t2["bound"] == "tensor" and t2["unit"] == "TFLOP/s"
    assert math.isclose(t2["frac"], 3.0e14 / 40e-3 / 1e12 / 1719.1, rel_tol=1e-12)


def test_matvec_bytes_follow_the_precision_of_the_products():
    """FP16 / BF16 Z: the GMRES products read 4 bytes per complex entry, FP32 8, FP64 16."""
    import bench
    got = {}
    for prec in (0, 1, 2, 3):
        _, allr = bench.roofline(_last(), N, PEAKS, prec, N_TETS)
        got[prec] = allr["k_matvec"]["algorithmic_bytes_per_z_product"]
    ld = (N + 3) // 4 * 4
    assert got[1] - got[2] == N * ld * 4 and got[2] == got[3] and got[0] - got[1] > N * ld * 8 - 1
