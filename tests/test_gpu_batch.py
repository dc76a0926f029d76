"""Batched sweeps (vie_solve_batch): every request's result in the batch equals
its result alone.

The fill accumulates Z with atomics, so two fills of the same request agree to
rounding, not bit for bit; each solve stops at its relative residual.  The
bars below follow from that: FP64 solves stop at 1e-10 (|dA| <= 1e-9), FP32
solves at 1e-6 after FP64 refinement on an FP32 Z that differs between runs
by rounding of its ~1e-7 relative entries (|dA| <= 1e-5, unknowns within
1e-4 relative).
"""
import numpy as np
import pytest

import cellgen

pytestmark = pytest.mark.gpu

vie = pytest.importorskip("paper_1809_05334_gb300.vie")

SWEEP = [(420.0, 0.0), (480.0, 0.35), (540.0, 0.7), (600.0, 0.2), (660.0, 1.0), (720.0, 0.5), (760.0, 1.3)]


@pytest.mark.parametrize("precision,tol,bar_a,bar_x", [(vie.VIE_FP64, 1e-10, 1e-9, 1e-8),
                                                       (vie.VIE_FP32, 1e-6, 1e-5, 1e-4)])
def test_batch_equals_single(precision, tol, bar_a, bar_x):
    cell = cellgen.small_cells()["plasmonic_tiny"]
    s = vie.Solver(precision=precision, tol=tol)
    try:
        s.set_mesh(cell)
        lams = [l for l, _ in SWEEP]
        ths = [t for _, t in SWEEP]
        phs = [0.3 * i for i in range(len(SWEEP))]
        eps = [cell.eps(l) for l in lams]
        alone = [s.solve(l, t, p, e, coeffs=True) for l, t, p, e in zip(lams, ths, phs, eps)]
        batch, used = s.solve_batch(lams, ths, phs, eps, max_slots=3, coeffs=True)
        assert used == 3
        for a, b in zip(alone, batch):
            assert b["status"] == 0 and a["status"] == 0
            assert np.all(b["rel_residual"] <= tol)
            assert np.max(np.abs(a["A"] - b["A"])) <= bar_a
            assert np.max(np.abs(a["R"] - b["R"])) <= bar_a
            assert np.max(np.abs(a["T"] - b["T"])) <= bar_a
            assert np.linalg.norm(a["x"] - b["x"]) <= bar_x * np.linalg.norm(a["x"])
        # a second batch reuses the slots (and their buffers)
        again, used2 = s.solve_batch(lams[:2], ths[:2], phs[:2], eps[:2], max_slots=3)
        assert used2 == 2
        for a, b in zip(alone[:2], again):
            assert np.max(np.abs(a["A"] - b["A"])) <= bar_a
    finally:
        s.close()


def test_batch_single_slot_and_statuses():
    """One slot runs the requests in order; a request at a Rayleigh anomaly gets
    its own error status without failing the others."""
    cell = cellgen.slab_cell(2, 2, 1, 400.0, 400.0, 20.0, (2.0, 0.1))
    s = vie.Solver(precision=vie.VIE_FP64, tol=1e-10)
    try:
        s.set_mesh(cell)
        lams = [500.0, 400.0, 600.0]
        out, used = s.solve_batch(lams, [0.0] * 3, [0.0] * 3, [cell.eps(l) for l in lams], max_slots=1)
        assert used == 1
        assert [o["status"] for o in out] == [0, -4, 0]
        ref = s.solve(600.0, 0.0, 0.0, cell.eps(600.0))
        assert np.max(np.abs(out[2]["A"] - ref["A"])) <= 1e-9
    finally:
        s.close()
