"""GPU tests of the autotuner (vie_tune, vie_options.autotune).

The tuner times candidate Ewald split multipliers of the FP32 fill and launch
shapes of the GMRES products on the caller's mesh and keeps the fastest.  The
split only moves work between the two Ewald series, so a solve after tuning
must still meet the parity bar against the FP64 oracle (|dA| <= 1e-4, FP64
residual <= 1e-6) and agree with the untuned solve to the spread of two FP32
fills (|dA| <= 1e-5).
"""
import numpy as np
import pytest

import cellgen
from oracle import solve_cell

pytestmark = pytest.mark.gpu

vie = pytest.importorskip("paper_1809_05334_gb300.vie")

CASES = [(520.0, 0.0, 0.0), (560.0, 0.6, 0.0), (520.0, 0.35, 0.2)]


@pytest.fixture(scope="module")
def cell():
    return cellgen.small_cells()["plasmonic_tiny"]


@pytest.mark.parametrize("lam,th,ph", CASES)
def test_tune_report_and_parity(cell, lam, th, ph):
    ref = solve_cell(cell, lam, th, ph)
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(cell)
        base = s.solve(lam, th, ph, cell.eps(lam))
        rep = s.tune(lam, th, ph, cell.eps(lam))
        assert rep["incidence_class"] == (0 if th == 0.0 else 1)
        assert len(rep["split"]) == 3 and len(rep["mv_grid"]) == 3
        timed = [(t, c) for t, c in zip(rep["fill_ms"], rep["split"]) if t > 0]
        assert timed, rep
        assert rep["split_chosen"] == min(timed)[1]
        assert rep["mv_chosen"] == rep["mv_grid"][int(np.argmin(rep["mv_ms"]))]
        assert all(t > 0 for t in rep["mv_ms"])
        out = s.solve(lam, th, ph, cell.eps(lam))
    finally:
        s.close()
    assert out["status"] == 0 and np.all(out["rel_residual"] <= 1e-6)
    assert np.max(np.abs(out["A"] - ref["A"])) <= 1e-4
    assert np.max(np.abs(out["A"] - base["A"])) <= 1e-5


def test_pivot_width_tuned_once_per_mesh():
    """A mesh with a domain block wider than 1024 unknowns: the first tuning
    times the inversion at both widths and keeps the faster; the next class's
    tuning reuses it; solves meet the bar with it."""
    mini = cellgen.small_cells()["plasmonic_mini"]
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(mini)
        r0 = s.tune(500.0, 0.0, 0.0, mini.eps(500.0))
        assert r0["pivot"] == [512, 1024] and all(t > 0 for t in r0["factor_ms"])
        assert r0["pivot_chosen"] == r0["pivot"][int(np.argmin(r0["factor_ms"]))]
        r1 = s.tune(500.0, 0.4, 0.0, mini.eps(500.0))
        assert r1["pivot"] == [] and r1["pivot_chosen"] == r0["pivot_chosen"]
        ref = solve_cell(mini, 500.0, 0.4, 0.0)
        out = s.solve(500.0, 0.4, 0.0, mini.eps(500.0))
    finally:
        s.close()
    assert out["status"] == 0 and np.max(np.abs(out["A"] - ref["A"])) <= 1e-4


def test_autotune_batch_equals_alone(cell):
    lams = [480.0, 520.0, 560.0, 600.0]
    ths = [0.0, 0.3, 0.0, 0.6]
    phs = [0.0] * 4
    eps = [cell.eps(l) for l in lams]
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6, autotune=True)
    try:
        s.set_mesh(cell)
        batch, used = s.solve_batch(lams, ths, phs, eps, max_slots=2)
        alone = [s.solve(l, t, p, e) for l, t, p, e in zip(lams, ths, phs, eps)]
    finally:
        s.close()
    for b, a in zip(batch, alone):
        assert b["status"] == 0 and a["status"] == 0
        assert np.max(np.abs(b["A"] - a["A"])) <= 1e-5
