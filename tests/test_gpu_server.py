"""Solve server (vie_server_*): continuous batching with HBM-footprint admission.

Each result in the mix equals the same request solved alone (vie_solve on a
plain context).  The fill accumulates Z with atomics, so repeated fills agree
to rounding; FP32 solves stop at relative residual 1e-6 after FP64
refinement, hence |dA| <= 1e-5 (see test_gpu_batch.py for the reasoning).
"""
import numpy as np
import pytest

import cellgen

pytestmark = pytest.mark.gpu

vie = pytest.importorskip("paper_1809_05334_gb300.vie")


def _mix():
    cells = cellgen.small_cells()
    out = []
    for name, lam, th, ph in [("plasmonic_tiny", 450.0, 0.3, 0.1), ("slab_3x3x1", 520.0, 0.0, 0.0),
                              ("slab_4x3x2_jit", 610.0, 0.9, 0.4), ("plasmonic_tiny", 700.0, 1.2, 0.0),
                              ("plasmonic_mini", 560.0, 0.5, 0.2), ("slab_3x3x1", 430.0, 0.6, 0.3)]:
        c = cells[name]
        out.append((c, lam, th, ph, c.eps(lam)))
    return out


def _alone(mix):
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    try:
        res = []
        for c, lam, th, ph, eps in mix:
            s.set_mesh(c)
            res.append(s.solve(lam, th, ph, eps))
        return res
    finally:
        s.close()


def test_server_mix_equals_alone():
    mix = _mix()
    alone = _alone(mix)
    srv = vie.Server(n_slots=3)
    try:
        tickets = [srv.submit(c, lam, th, ph, eps)[0] for c, lam, th, ph, eps in mix]
        out = [srv.poll(t, wait_ms=-1) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert st["submitted"] == len(mix) and st["completed"] == len(mix)
    assert st["max_running"] >= 2            # requests overlapped on the device
    for a, b in zip(alone, out):
        assert b["status"] == 0
        assert np.all(b["rel_residual"] <= 1e-6)
        assert np.max(np.abs(a["A"] - b["A"])) <= 1e-5
        assert np.max(np.abs(a["R"] - b["R"])) <= 1e-5
        assert b["t_latency_ms"] >= b["t_queue_ms"] >= 0.0


def test_server_budget_admission_and_rejection():
    """A budget that holds one request at a time serialises the slots; a request
    larger than the whole budget is rejected at submission."""
    cells = cellgen.small_cells()
    c = cells["plasmonic_tiny"]
    probe = vie.Server(n_slots=1)
    try:
        _, fp = probe.submit(c, 500.0, 0.0, 0.0, c.eps(500.0))
    finally:
        probe.close()
    srv = vie.Server(n_slots=3, hbm_budget_bytes=int(1.5 * fp))
    try:
        reqs = [(500.0, 0.0), (560.0, 0.4), (620.0, 0.8), (680.0, 0.2)]
        tickets = [srv.submit(c, lam, th, 0.0, c.eps(lam))[0] for lam, th in reqs]
        big = cellgen.config_sweep_geometry()       # ~8.9k unknowns: > 1 GB
        with pytest.raises(vie.VIEError) as e:
            srv.submit(big, 500.0, 0.0, 0.0, big.eps(500.0))
        assert e.value.code == -2
        out = [srv.poll(t, wait_ms=-1) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert st["max_running"] == 1
    assert st["rejected"] == 1
    assert st["peak_reserved_bytes"] <= st["budget_bytes"]
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(c)
        for (lam, th), o in zip(reqs, out):
            ref = s.solve(lam, th, 0.0, c.eps(lam))
            assert o["status"] == 0
            assert np.max(np.abs(ref["A"] - o["A"])) <= 1e-5
    finally:
        s.close()


def test_server_poll_pending_and_unknown_ticket():
    c = cellgen.small_cells()["slab_3x3x1"]
    srv = vie.Server(n_slots=1)
    try:
        t, _ = srv.submit(c, 500.0, 0.0, 0.0, c.eps(500.0))
        r = srv.poll(t, wait_ms=0)
        if r is None:
            r = srv.poll(t, wait_ms=-1)
        assert r["status"] == 0
        with pytest.raises(vie.VIEError):
            srv.poll(t, wait_ms=0)          # a ticket is forgotten once its result is read
    finally:
        srv.close()


def test_server_cancel_queued_and_running():
    """vie_server_cancel: with one slot, a request queued behind a running one
    never runs and polls as VIE_CANCELLED; the running one, cancelled while it
    runs, stops at its next check (VIE_CANCELLED) unless it finished first;
    a finished request keeps its result; an unknown ticket is an error."""
    import time
    big = cellgen.config_sweep_geometry()
    small = cellgen.small_cells()["slab_3x3x1"]
    srv = vie.Server(n_slots=1, precision=vie.VIE_FP32, tol=1e-6)
    try:
        t_run, _ = srv.submit(big, 500.0, 0.2, 0.0, big.eps(500.0))
        t_queued, _ = srv.submit(small, 520.0, 0.0, 0.0, small.eps(520.0))
        t_done, _ = srv.submit(small, 520.0, 0.0, 0.0, small.eps(520.0))
        for _ in range(2000):                       # wait until the first request runs
            if srv.stats()["running"] == 1:
                break
            time.sleep(0.005)
        srv.cancel(t_queued)
        srv.cancel(t_run)
        r_run = srv.poll(t_run, wait_ms=-1)
        r_queued = srv.poll(t_queued, wait_ms=-1)
        r_done = srv.poll(t_done, wait_ms=-1)
        assert r_queued["status"] == vie.VIE_CANCELLED
        assert r_run["status"] in (vie.VIE_CANCELLED, 0)
        assert r_done["status"] == 0
        with pytest.raises(vie.VIEError):
            srv.cancel(123456789)
        st = srv.stats()
        assert st["cancelled"] >= 1 and st["queued"] == 0 and st["running"] == 0
    finally:
        srv.close()


def test_bounded_device_wait_reports_timeout_and_device_stays_usable():
    """The failure path of the bounded device waits: a wait on a barrier that
    nobody arrives on runs out after its poll limit and comes back as
    VIE_DEVICE_TIMEOUT (no fault, no hang); the same wait with its arrival
    completes; a solve afterwards still works."""
    assert vie.check_device_wait(0, arrive=False, polls=1000) == -5
    assert vie.check_device_wait(0, arrive=True, polls=1000) == 0
    cell = cellgen.small_cells()["slab_3x3x1"]
    s = vie.Solver(precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(cell)
        out = s.solve(500.0, 0.0, 0.0, cell.eps(500.0))
    finally:
        s.close()
    assert out["status"] == 0
