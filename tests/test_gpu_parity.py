"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (each derived from the arithmetic of its path):
  FP64 Faddeeva           |rel| <= 1e-13      (Weideman N=40 error ~3e-14)
  FP32 Faddeeva           |rel| <= 2e-6       (N=20 expansion in FP32)
  FP64 g_p                |rel| <= 1e-11      (Ewald truncation, rounding)
  FP32 g_p                |abs| <= 2e-6 max|g|
  FP64 Z, b               max|dZ| <= 1e-9 max|Z|
  FP32 Z                  max|dZ| <= 2e-5 max|Z|
  FP64 solve              |dA|, |dR|, |dT| <= 1e-8; coefficients rel 1e-7
  FP32 + FP64 refinement  |dA| <= 1e-4 and FP64 relative residual <= 1e-6 (the stated bar)
"""
import numpy as np
import pytest
from scipy.special import wofz

import cellgen
import golden_data
from oracle import solve_cell
from oracle.fill import Problem, assemble
from oracle.greens import PeriodicGreen
from oracle.topology import build_topology

pytestmark = pytest.mark.gpu

vie = pytest.importorskip("paper_1809_05334_gb300.vie")


@pytest.fixture(scope="module")
def solver64():
    s = vie.Solver(precision=vie.VIE_FP64, tol=1e-10)
    yield s
    s.close()


@pytest.fixture(scope="module")
def solver32():
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    yield s
    s.close()


_ORACLE = {}


def oracle_run(name, cell, lam, th, ph):
    key = (name, lam, th, ph)
    if key not in _ORACLE:
        _ORACLE[key] = solve_cell(cell, lam, th, ph, keep_matrix=True)
    return _ORACLE[key]


CASES = [("slab_3x3x1", 500.0, 0.0, 0.0), ("slab_4x3x2_jit", 470.0, 0.5, 0.3),
         ("plasmonic_tiny", 520.0, 0.35, 0.2), ("plasmonic_tiny", 560.0, 0.6, 0.0)]


# --------------------------------------------------------------------------- special functions
def test_faddeeva_fp64_and_fp32(solver64):
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.uniform(0, 8, 3000) + 1j * rng.uniform(-8, 8, 3000),
                        rng.uniform(0, 1e-3, 200) + 1j * rng.uniform(-3, 3, 200),
                        rng.uniform(0, 30, 200) + 0j, np.array([0.0 + 0j, 1e-12 + 0j])])
    ref = wofz(1j * u)
    g64 = solver64.erfcx(u, vie.VIE_FP64)
    g32 = solver64.erfcx(u, vie.VIE_FP32)
    assert np.max(np.abs(g64 - ref) / np.abs(ref)) < 1e-13
    assert np.max(np.abs(g32 - ref) / np.abs(ref)) < 2e-6


@pytest.mark.parametrize("a,b,lam,th,ph", [(200.0, 200.0, 500.0, 0.0, 0.0), (180.0, 150.0, 430.0, 0.6, 0.3),
                                           (400.0, 400.0, 650.0, 0.9, 1.1), (60.0, 54.0, 520.0, 0.35, 0.2),
                                           (200.0, 200.0, 500.0, 0.5, 0.0), (400.0, 400.0, 650.0, 0.9, 0.0),
                                           (300.0, 240.0, 420.0, 1.2, 0.0)])
def test_periodic_green_vs_oracle(solver64, a, b, lam, th, ph):
    cell = cellgen.slab_cell(2, 2, 1, a, b, 20.0, (2.0, 0.1))
    solver64.set_mesh(cell)
    rng = np.random.default_rng(3)
    d = np.stack([rng.uniform(-a, a, 400) * 0.999, rng.uniform(-b, b, 400) * 0.999, rng.uniform(-80, 80, 400)], 1)
    d[:10, 2] = 0.0
    d[10:20] *= 0.01
    k0 = 2 * np.pi / lam
    ref = PeriodicGreen(k0, k0 * np.sin(th) * np.cos(ph), k0 * np.sin(th) * np.sin(ph), a, b)(d)
    g64 = solver64.green(d, lam, th, ph, vie.VIE_FP64)
    g32 = solver64.green(d, lam, th, ph, vie.VIE_FP32)
    assert np.max(np.abs(g64 - ref) / np.abs(ref)) < 1e-11
    assert np.max(np.abs(g32 - ref)) < 2e-6 * np.max(np.abs(ref)) + 0.0
    assert np.max(np.abs(g32 - ref) / np.abs(ref)) < 5e-4


# --------------------------------------------------------------------------- matrix fill
@pytest.mark.parametrize("name,lam,th,ph", CASES)
def test_fill_fp64_matches_oracle(solver64, name, lam, th, ph):
    cell = cellgen.small_cells()[name]
    n = solver64.set_mesh(cell)
    ref = oracle_run(name, cell, lam, th, ph)
    assert n == ref["topo"]["n"]
    eps = cell.eps(lam)
    Z, b = solver64.fill_matrix(lam, th, ph, eps)
    scale = np.max(np.abs(ref["Z"]))
    err = np.abs(Z - ref["Z"])
    assert np.max(err) < 1e-9 * scale, (np.max(err) / scale, np.unravel_index(np.argmax(err), err.shape))
    assert np.max(np.abs(b - ref["b"])) < 1e-12 * np.max(np.abs(ref["b"]))


@pytest.mark.parametrize("name,lam,th,ph", CASES)
def test_fill_fp32_matches_oracle(solver32, name, lam, th, ph):
    cell = cellgen.small_cells()[name]
    solver32.set_mesh(cell)
    ref = oracle_run(name, cell, lam, th, ph)
    Z = solver32.fill_matrix_prec(lam, th, ph, cell.eps(lam))
    scale = np.max(np.abs(ref["Z"]))
    assert np.max(np.abs(Z - ref["Z"])) < 2e-5 * scale


# --------------------------------------------------------------------------- solve
@pytest.mark.parametrize("name,lam,th,ph", CASES)
def test_solve_fp64_matches_oracle(solver64, name, lam, th, ph):
    cell = cellgen.small_cells()[name]
    solver64.set_mesh(cell)
    ref = oracle_run(name, cell, lam, th, ph)
    out = solver64.solve(lam, th, ph, cell.eps(lam), coeffs=True)
    assert out["status"] == 0
    assert np.all(out["rel_residual"] <= 1e-10)
    assert np.max(np.abs(out["A"] - ref["A"])) < 1e-8
    assert np.max(np.abs(out["R"] - ref["R"])) < 1e-8
    assert np.max(np.abs(out["T"] - ref["T"])) < 1e-8
    x = out["x"]
    assert np.linalg.norm(x - ref["x"]) < 1e-7 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("name,lam,th,ph", CASES)
def test_solve_mixed_meets_bar(solver32, name, lam, th, ph):
    cell = cellgen.small_cells()[name]
    solver32.set_mesh(cell)
    ref = oracle_run(name, cell, lam, th, ph)
    out = solver32.solve(lam, th, ph, cell.eps(lam), coeffs=True)
    assert out["status"] == 0
    assert np.all(out["rel_residual"] <= 1e-6)
    assert np.max(np.abs(out["A"] - ref["A"])) <= 1e-4
    # residual of the returned unknowns against the oracle's FP64 matrix: the
    # refinement converges on the FP32-stored Z, whose entries differ from the
    # FP64 ones by <= 2e-5 max|Z| (test_fill_fp32), so this residual is bounded
    # by that difference, not by the 1e-6 solver tolerance
    r = ref["b"] - ref["Z"] @ out["x"]
    assert np.all(np.linalg.norm(r, axis=0) <= 1e-3 * np.linalg.norm(ref["b"], axis=0))
    # the reported residual is the FP64 residual against the stored FP32 Z (the
    # device forms Z x at double length from FP32 arithmetic): numpy in FP64 on
    # a fresh fill of the same matrix gives the same number, up to the
    # fill-to-fill spread of Z (its FP32 contributions are summed by atomics in
    # no fixed order), measured here on two more fills
    zs = solver32.fill_matrix_prec(lam, th, ph, cell.eps(lam))
    z2 = solver32.fill_matrix_prec(lam, th, ph, cell.eps(lam))
    bn = np.linalg.norm(ref["b"], axis=0)
    rel = np.linalg.norm(ref["b"] - zs @ out["x"], axis=0) / bn
    spread = np.linalg.norm((zs - z2) @ out["x"], axis=0) / bn
    assert np.all(np.abs(rel - out["rel_residual"]) <= 4 * spread + 1e-11), (rel, out["rel_residual"], spread)


def test_preconditioner_does_not_change_solution(solver64):
    cell = cellgen.small_cells()["plasmonic_tiny"]
    solver64.set_mesh(cell)
    lam = 480.0
    a = solver64.solve(lam, 0.2, 0.1, cell.eps(lam), coeffs=True)
    solver64.set_options(use_precond=0)
    try:
        b = solver64.solve(lam, 0.2, 0.1, cell.eps(lam), coeffs=True)
    finally:
        solver64.set_options(use_precond=1)
    # Eq. (8): relative difference of the current coefficients; both solves stop
    # at relative residual 1e-10, so they agree to ~cond(Z) x 1e-10; the paper
    # reports < 12% per unknown at its own, looser, tolerance (golden fixture;
    # checked here on the coefficients above 1e-3 of the largest)
    rel = np.linalg.norm(a["x"] - b["x"]) / np.linalg.norm(b["x"])
    assert rel < 1e-5
    per_unknown = np.abs(a["x"] - b["x"]) / np.maximum(np.abs(b["x"]), 1e-300)
    big = np.abs(b["x"]) > 1e-3 * np.max(np.abs(b["x"]))
    assert np.all(per_unknown[big] < golden_data.load("paper_eq8_preconditioner.txt")["eq8_relative_error_max"])
    assert a["iterations"][0] <= b["iterations"][0]


def test_config_slab_full_size(solver64, solver32):
    """The homogeneous-slab workload (432 tets, 936 unknowns) at both precisions."""
    cell = cellgen.config_slab()
    ref = oracle_run("config_slab", cell, 500.0, 0.0, 0.0)
    for s, tolA in ((solver64, 1e-8), (solver32, 1e-4)):
        assert s.set_mesh(cell) == 936
        out = s.solve(500.0, 0.0, 0.0, cell.eps(500.0))
        assert out["status"] == 0
        assert np.max(np.abs(out["A"] - ref["A"])) <= tolA
        assert abs(out["R"][0] - ref["R"][0]) <= 10 * tolA


# --------------------------------------------------------------------------- error paths
def test_rayleigh_anomaly_is_reported(solver64):
    cell = cellgen.slab_cell(2, 2, 1, 400.0, 400.0, 20.0, (2.0, 0.1))
    solver64.set_mesh(cell)
    with pytest.raises(vie.VIEError) as e:
        solver64.solve(400.0, 0.0, 0.0, cell.eps(400.0))
    assert e.value.code == -4


def test_bad_mesh_is_rejected(solver64):
    cell = cellgen.slab_cell(2, 2, 1, 100.0, 100.0, 20.0, (2.0, 0.1))
    bad = cellgen.Cell(verts=cell.verts, tets=cell.tets[:, [0, 2, 1, 3]].copy(), tet_domain=cell.tet_domain,
                       n_domains=1, period_a=100.0, period_b=100.0, active_domain=0, domain_names=cell.domain_names)
    with pytest.raises(vie.VIEError) as e:
        solver64.set_mesh(bad)
    assert e.value.code == -6
