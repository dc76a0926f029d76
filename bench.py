"""Benchmark: (lambda, theta) solves per second of the preconditioned periodic VIE.

Workload (one step = one full solve at one incidence, TE and TM together):
the plasmonic unit cell, period 200 nm, Ag sphere r = 20 nm centred in a
100 nm active layer over a 40 nm buffer (three material domains, ~21k SWG
unknowns), lambda = 500 nm, normal incidence.  A step runs the whole path:
Ewald-summed fill of Z (Eq. (2)-(4)), inversion of the domain blocks
(Eq. (6)), preconditioned GMRES with FP64 residual refinement, absorption
(Eq. (7)), reflectance and transmittance.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64] [--impl reference]

N > 1 runs under torch.distributed.run: every rank solves the same workload on
its own GPU (independent solves, replicas only), timing is the max over ranks.
--impl reference times the FP64 CPU oracle (the plain restatement of the
method, dense LU) on a reduced-density sample of the same cell.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(lambda,theta) solves/s"
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}   # vie_precision
UNIT = "solves/s"
LAM, THETA, PHI = 500.0, 0.0, 0.0
WORKLOADS = {
    "plasmonic": ("config_plasmonic",
                  "plasmonic cell 200 nm period, Ag sphere r=20 nm (smooth mapped-cube mesh, 384 tets) in 100 nm "
                  "active over 40 nm buffer, 10368 tets, 21024 unknowns, lambda=500 nm, theta=0, TE+TM"),
    # the same cell with the grid nodes near the sphere snapped onto it (faceted particle surface)
    "plasmonic_snap": ("config_plasmonic_snap",
                       "plasmonic cell 200 nm period, Ag sphere r=20 nm (snapped grid) in 100 nm active over "
                       "40 nm buffer, 10368 tets, 21024 unknowns, lambda=500 nm, theta=0, TE+TM"),
    # a finer particle mesh
    "plasmonic_fine": ("config_plasmonic_fine",
                       "plasmonic cell 200 nm period, Ag sphere r=20 nm (mapped cube, 750 tets) in 100 nm active "
                       "over 40 nm buffer, 17550 tets, 35550 unknowns, lambda=500 nm, theta=0, TE+TM"),
    # the same geometry at the sweep density (~9.9k unknowns): a smaller case for profiling
    "sweep_cell": ("config_sweep_geometry",
                   "plasmonic cell 200 nm period at sweep density (4860 tets, 9882 unknowns), lambda=500 nm, "
                   "theta=0, TE+TM"),
}


SWEEP_WORKLOAD = ("batched sweep on the plasmonic geometry at sweep density (9882 unknowns): lambda 400-800 nm "
                  "in 5 nm steps (81 values, dispersive Drude/Cauchy eps) with theta cycling 0-80 deg in 10 deg "
                  "steps, TE+TM per solve")


def sweep_requests(k):
    """The first k (lambda, theta) points of the sweep: lambda_i = 400 + 5 (i mod 81) nm,
    theta_i = 10 deg x (i mod 9), phi = 0."""
    lams = [400.0 + 5.0 * (i % 81) for i in range(k)]
    ths = [np.deg2rad(10.0 * (i % 9)) for i in range(k)]
    return lams, ths


def _cell(name):
    import cellgen
    return getattr(cellgen, WORKLOADS[name][0])()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local



def _max_dA(a, b):
    return float(np.max(np.abs(np.asarray(a["A"]) - np.asarray(b["A"]))))


def _timed_solves(solver, eps, steps, stream, torch, warm=True):
    """`steps` solves of the bench incidence on `stream`, bracketed by CUDA events
    (after one warm-up solve if warm); returns (ms per solve, the last result)."""
    sp = stream.cuda_stream
    if warm:
        solver.solve(LAM, THETA, PHI, eps, stream=sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        out = solver.solve(LAM, THETA, PHI, eps, stream=sp)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def leg_precision(vie, torch, local, cell, eps, prec, steps, stream, mixed, tol=1e-6, warm=True):
    """The same workload at another precision of the path (FP64: the plain FP64
    GPU path; FP16 / BF16: 16-bit Z in the GMRES products): solves/s, and the
    largest absorption difference from the mixed-precision (FP32) results."""
    s = vie.Solver(device=local, precision=prec, tol=tol, timing=True)
    try:
        s.set_mesh(cell)
        ms, out = _timed_solves(s, eps, steps, stream, torch, warm=warm)
    finally:
        s.close()
    return {"value": 1e3 / ms, "unit": UNIT, "steps": steps, "warmed_up": warm, "ms_per_solve": ms, "tol": tol,
            "kernels_ms": {"far_tt": out["k_far_tt_ms"], "fill": out["k_fill_ms"], "factor": out["k_factor_ms"],
                           "matvec_total": out["k_matvec_ms"], "matvec_n": out["k_matvec_n"],
                           "precond_total": out["k_precond_ms"]},
            "phases_ms": {k: out["t_" + k + "_ms"] for k in ("fill", "factor", "solve", "post")},
            "iterations": out["iterations"], "refinements": out["refinements"],
            "rel_residual": [float(v) for v in out["rel_residual"]], "status": out["status"],
            "absorbed_active": [float(v) for v in out["A"][:, cell.active_domain]],
            "max_abs_dA_vs_fp32_mixed": _max_dA(out, mixed)}


def leg_preconditioner(vie, local, cell, eps, stream, with_pre):
    """Fig. 2 on the bench workload: GMRES iterations with the Eq. (6)
    preconditioner (the timed solves) and without it (capped at 1000
    iterations, reported as not converged if it does not reach the tolerance)."""
    s = vie.Solver(device=local, precision=vie.VIE_FP32, tol=1e-6, use_precond=False, max_iter=1000)
    try:
        s.set_mesh(cell)
        t0 = time.perf_counter()
        out = s.solve(LAM, THETA, PHI, eps, stream=stream.cuda_stream)
        dt = time.perf_counter() - t0
    finally:
        s.close()
    return {"with_eq6": {"iterations": with_pre["iterations"], "refinements": with_pre["refinements"],
                         "rel_residual": [float(v) for v in with_pre["rel_residual"]], "status": with_pre["status"]},
            "without": {"iterations": out["iterations"], "refinements": out["refinements"],
                        "rel_residual": [float(v) for v in out["rel_residual"]],
                        "status": vie.STATUS.get(out["status"], out["status"]), "max_iter": 1000,
                        "wall_s": dt}}


def leg_sweep(vie, torch, local, k, slots):
    """The first k (lambda, theta) points of the 81-point sweep through
    vie_solve_batch (slots in flight) in FP32 and in FP16: solves/s, and the
    largest absorption difference between the two."""
    cell = _cell("sweep_cell")
    lams, ths = sweep_requests(k)
    eps = [cell.eps(l) for l in lams]
    phs = [0.0] * k
    out = {"workload": SWEEP_WORKLOAD + " (first %d points)" % k, "n_unknowns": None}
    res = {}
    for name in ("fp32", "fp16"):
        s = vie.Solver(device=local, precision=PRECISIONS[name], tol=1e-6, autotune=True)
        try:
            out["n_unknowns"] = s.set_mesh(cell)
            # warm-up; its normal and oblique requests autotune the schedule (untimed)
            s.solve_batch(lams[:slots], ths[:slots], phs[:slots], eps[:slots], max_slots=slots)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r, used = s.solve_batch(lams, ths, phs, eps, max_slots=slots)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        finally:
            s.close()
        res[name] = r
        out[name] = {"value": k / dt, "unit": UNIT, "slots": used,
                     "iterations_mean": float(np.mean([sum(o["iterations"]) / 2 for o in r])),
                     "max_rel_residual": float(max(np.max(o["rel_residual"]) for o in r)),
                     "non_ok_status": [o["status"] for o in r if o["status"] != 0]}
    out["fp16_over_fp32"] = out["fp16"]["value"] / out["fp32"]["value"]
    out["max_abs_dA_fp16_vs_fp32"] = max(_max_dA(a, b) for a, b in zip(res["fp16"], res["fp32"]))
    return out


def leg_serve(vie, torch, local, k, slots):
    """k requests of the serving stream through the solve server, submitted at
    their Poisson arrival times (several in flight): solves/s and p50/p99
    latency from submission to completion, queueing included."""
    reqs = serve_requests(k)
    srv = vie.Server(device=local, n_slots=slots, precision=vie.VIE_FP32, tol=1e-6)
    try:
        import cellgen
        warm = cellgen.small_cells()["plasmonic_tiny"]
        t, _ = srv.submit(warm, 500.0, 0.0, 0.0, warm.eps(500.0))
        srv.poll(t, wait_ms=-1)
        torch.cuda.synchronize()
        tickets = []
        t0 = time.perf_counter()
        for at, cell, lam, th in reqs:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            tk, _ = srv.submit(cell, lam, th, 0.0, cell.eps(lam))
            tickets.append(tk)
        out = [srv.poll(tk, wait_ms=-1) for tk in tickets]
        elapsed = time.perf_counter() - t0
        st = srv.stats()
    finally:
        srv.close()
    lat = [o["t_latency_ms"] for o in out]
    ns = [o["n"] for o in out]
    return {"workload": SERVE_WORKLOAD + " (first %d requests)" % k, "slots": slots, "value": len(out) / elapsed,
            "unit": UNIT, "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "unknowns_min_median_max": [int(min(ns)), int(np.median(ns)), int(max(ns))],
            "max_running": st["max_running"], "non_ok_status": [o["status"] for o in out if o["status"] != 0],
            "max_rel_residual": float(max(np.max(o["rel_residual"]) for o in out))}


LARGE_WORKLOAD = ("large cell: period 400 nm, 2 x 2 Ag spheres r = 35 nm in a 120 nm active layer over a 40 nm "
                  "Ag back grating (40 nm ridges), 44550 tets, 90450 unknowns (FP32 Z 65 GB)")


def leg_large(vie, torch, local, prec, stream, lam=600.0, theta=0.0, pivot=1024):
    """One solve of the large cell (mixed precision only: an FP64 Z would not
    leave room for the block inverses): set-up time, solve time and phases,
    iterations, FP64 residual, and the GMRES products' HBM rate at this size.
    pivot: the block inversion's outer pivot width (0: the library default).
    The cell is not autotuned (that would time four inversions of seconds);
    1024 is the width measured faster on it (factor 3.32 -> 2.97 s at 600 nm,
    the same iterations)."""
    import cellgen
    cell = cellgen.config_large()
    s = vie.Solver(device=local, precision=prec, tol=1e-6, timing=True, precond_pivot=pivot)
    try:
        t0 = time.perf_counter()
        n = s.set_mesh(cell)
        t1 = time.perf_counter()
        ms, out = _timed_solves(s, cell.eps(lam), 1, stream, torch, warm=False)
    finally:
        s.close()
    ld = (n + 3) // 4 * 4
    zb = Z_BYTES[prec]
    mv = out["k_matvec_ms"]
    return {"workload": LARGE_WORKLOAD, "n_unknowns": n, "lambda_nm": lam, "theta_deg": float(np.rad2deg(theta)),
            "precision": {v: k for k, v in PRECISIONS.items()}[prec], "set_mesh_s": t1 - t0, "precond_pivot": pivot or 512,
            "value": 1e3 / ms, "unit": UNIT, "ms_per_solve": ms, "warmed_up": False,
            "phases_ms": {k: out["t_" + k + "_ms"] for k in ("fill", "factor", "solve", "post")},
            "iterations": out["iterations"], "refinements": out["refinements"],
            "rel_residual": [float(v) for v in out["rel_residual"]], "status": out["status"],
            "absorbed_active": [float(v) for v in out["A"][:, cell.active_domain]],
            "z_products_gbs": out["k_matvec_n"] * n * ld * zb / (mv / 1e3) / 1e9 if mv else None}


def run_large(args):
    """The large cell's sweep: lambda 400-800 nm in 20 nm steps at theta = 0 and
    45 deg (the first --steps points; lambda = 400 nm at theta = 0 sits on a
    Rayleigh anomaly of the 400 nm lattice and is moved to 400.01 nm), one
    solve at a time, FP16 products with FP64 refinement."""
    import torch

    import cellgen
    from paper_1809_05334_gb300 import vie
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    prec = PRECISIONS[args.precision]
    cell = cellgen.config_large()
    pts = [(400.0 + 20.0 * i, th) for th in (0.0, np.pi / 4) for i in range(21)][:args.steps]
    pts = [(l + 0.01 if (abs(l - 400.0) < 1e-9 and th == 0.0) else l, th) for l, th in pts]
    s = vie.Solver(device=local, precision=prec, tol=1e-6, precond_pivot=1024)   # as leg_large
    try:
        t0 = time.perf_counter()
        n = s.set_mesh(cell)
        t_mesh = time.perf_counter() - t0
        outs = []
        t0 = time.perf_counter()
        for lam, th in pts:
            outs.append(s.solve(lam, th, 0.0, cell.eps(lam)))
        dt = time.perf_counter() - t0
    finally:
        s.close()
    print(json.dumps({"metric": METRIC, "value": len(pts) / dt, "unit": UNIT, "steps": len(pts),
                      "ms_per_step": dt * 1e3 / len(pts), "higher_is_better": True, "data": "synthetic",
                      "dtype": {"fp32": "c64+f64", "fp16": "c32(fp16)+c64+f64", "bf16": "c32(bf16)+c64+f64"}.get(
                          args.precision, "c128"),
                      "config": {"workload": LARGE_WORKLOAD, "n_unknowns": n, "precision": args.precision},
                      "set_mesh_s": t_mesh,
                      "points": [{"lambda_nm": l, "theta_deg": float(np.rad2deg(t)), "A_active": float(np.mean(o["A"][:, 1])),
                                  "iterations": o["iterations"], "rel_residual": float(np.max(o["rel_residual"])),
                                  "status": o["status"]} for (l, t), o in zip(pts, outs)]}))


def oracle_sample(full_cell):
    """The FP64 oracle timed whole on a bounded sample of the bench geometry (the
    plasmonic cell at 378 tetrahedra), its fill and dense-LU phases timed
    apart, and the throughput it extrapolates to the full workload (fill by
    the tetrahedron-pair ratio, LU by the cube of the unknown ratio)."""
    import cellgen
    from oracle.fill import Problem, assemble
    from oracle.post import absorption
    from oracle.solve import solve_dense
    from oracle.topology import build_topology
    sample = cellgen.config_plasmonic_sample()
    t0 = time.perf_counter()
    topo = build_topology(sample)
    prob = Problem(topo, LAM, THETA, PHI, sample.eps(LAM))
    Z, b = assemble(prob)
    t1 = time.perf_counter()
    x = solve_dense(Z, b)
    t2 = time.perf_counter()
    for p in range(2):
        absorption(prob, x[:, p])
    t3 = time.perf_counter()
    from oracle.topology import build_topology as _bt
    n_full = _bt(full_cell)["n"] if full_cell.n_tets <= 20000 else None
    fill_s, lu_s, post_s = t1 - t0, t2 - t1, t3 - t2
    scale_fill = (full_cell.n_tets / sample.n_tets) ** 2
    scale_lu = (n_full / topo["n"]) ** 3 if n_full else scale_fill ** 1.5
    t_full = fill_s * scale_fill + lu_s * scale_lu + post_s * full_cell.n_tets / sample.n_tets
    return sample, topo["n"], {"fill_s": fill_s, "lu_s": lu_s, "post_s": post_s, "total_s": t3 - t0,
                               "extrapolated_s": t_full, "scale_fill": scale_fill, "scale_lu": scale_lu}


def leg_same_workload(vie, torch, local, sample, stream, steps=5):
    """The GPU path on the oracle's timing sample itself (mixed precision): the
    same-workload comparison with the timed oracle."""
    s = vie.Solver(device=local, precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(sample)
        ms, out = _timed_solves(s, sample.eps(LAM), steps, stream, torch)
    finally:
        s.close()
    return {"value": 1e3 / ms, "unit": UNIT, "ms_per_solve": ms, "steps": steps}


def _leg(res, name, fn, *a, **kw):
    """Run one measured side leg; a failure is recorded, not raised (the main
    line must still print)."""
    t0 = time.perf_counter()
    try:
        res[name] = fn(*a, **kw)
    except Exception as e:   # noqa: BLE001
        res[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    if isinstance(res[name], dict):
        res[name]["leg_wall_s"] = round(time.perf_counter() - t0, 2)


def max_over_ranks(value, device, dist, ws):
    """The largest of a per-rank float over all ranks (the value itself on one rank)."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, steps, ms_max):
    """Whole-job solves/s of ws independent replicas that each ran `steps` solves,
    timed by the slowest rank."""
    return ws * steps / (ms_max / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import cellgen
    from paper_1809_05334_gb300 import vie

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = PRECISIONS[args.precision]
    cell = _cell(args.workload)
    eps = cell.eps(LAM)
    solver = vie.Solver(device=local, precision=prec, tol=1e-6, timing=True)
    n = solver.set_mesh(cell)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # schedule autotuning on this mesh and incidence (set-up, untimed)
    tune = solver.tune(LAM, THETA, PHI, eps, stream=sp)
    global FAR_SPLIT_CHOSEN
    FAR_SPLIT_CHOSEN = tune["split_chosen"]
    for _ in range(args.warmup):
        out = solver.solve(LAM, THETA, PHI, eps, stream=sp)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        ev0.record(stream)
        step_ev[0].record(stream)
        for k in range(args.steps):
            results.append(solver.solve(LAM, THETA, PHI, eps, stream=sp))
            step_ev[k + 1].record(stream)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    lat = [step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps)]
    ms_max = max_over_ranks(ms, dev, dist, ws)
    last = results[-1]

    # end-to-end through the public API with host buffers: every step uploads its
    # request (incidence, permittivities and the per-request tables) from the
    # host and reads the solved unknowns and the results back to the host; the
    # mesh stays resident (set once, like a model's weights)
    barrier()
    coeffs = np.zeros((n, 2), dtype=np.complex128)
    e2e_steps = max(1, min(args.steps, 3))
    h2d = d2h = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r = solver.solve(LAM, THETA, PHI, eps, coeffs=coeffs, stream=sp)
        h2d += r["h2d_bytes"]
        d2h += r["d2h_bytes"]
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev, dist, ws)
    h2d //= e2e_steps
    d2h //= e2e_steps

    value = replica_throughput(ws, args.steps, ms_max)
    peaks = _peaks()
    # FP32 / FP64 FMA peaks measured on this GPU with the library's FMA-loop
    # kernel (the denominators of the CUDA-core fill kernels' FP rates)
    try:
        peaks["fp32_fma_tflops"] = vie.fma_peak(local, vie.VIE_FP32)
        peaks["fp64_fma_tflops"] = vie.fma_peak(local, vie.VIE_FP64)
    except Exception:   # noqa: BLE001
        pass
    # roofline: the kernel with the largest device time in the solve (see roofline())
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "c64+f64", "fp16": "c32(fp16)+c64+f64", "bf16": "c32(bf16)+c64+f64"}.get(args.precision, "c128"),
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "n_unknowns": n, "n_tets": cell.n_tets, "precision": args.precision,
                   "theta_deg": args.theta_deg,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (Z is %.1f GB)" % (n * n * (8 if prec == vie.VIE_FP32 else 16) / 1e9)},
        "autotune": tune,
        "phases_ms": {"fill": last["t_fill_ms"], "factor": last["t_factor_ms"], "solve": last["t_solve_ms"],
                      "post": last["t_post_ms"]},
        "kernels_ms": {"far_tt": last["k_far_tt_ms"], "fill": last["k_fill_ms"], "factor": last["k_factor_ms"],
                       "tc_update_total": last["k_tc_ms"], "tc_update_n": last["k_tc_n"],
                       "matvec_total": last["k_matvec_ms"], "matvec_n": last["k_matvec_n"],
                       "precond_total": last["k_precond_ms"], "precond_n": last["k_precond_n"],
                       "ortho_total": last["k_ortho_ms"]},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "note": "per solve, one solve in flight"},
        "iterations": last["iterations"], "rel_residual": [float(v) for v in last["rel_residual"]],
        "absorbed_active": [float(v) for v in last["A"][:, cell.active_domain]],
        "e2e": {"value": replica_throughput(ws, e2e_steps, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": None,
    }
    res["roofline"], res["rooflines"] = roofline(last, n, peaks, prec, cell.n_tets)
    res["clocks"] = clk.summary()
    res["measured_peaks"] = {k: peaks[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained",
                                                   "fp32_fma_tflops", "fp64_fma_tflops") if k in peaks}
    # kernels launched inside the timed region, counted by the library at each launch site
    res["gpu_launches"] = int(sum(r["n_launches"] for r in results))
    solver.close()
    # measured side legs (after the timed region; they do not enter `value`):
    # the rest of the headline metric, mixed vs FP64 and the other precisions on
    # this workload, the Fig. 2 iteration counts, a batched sweep, a serving
    # stream with requests in flight together, and the timed oracle
    if not args.main_only and prec == vie.VIE_FP32 and ws == 1:
        # the plain FP64 path costs about a minute per solve here (its Ewald
        # series run on the FP64 pipe): one timed solve, no warm-up
        _leg(res, "fp64_gpu_path", leg_precision, vie, torch, local, cell, eps, vie.VIE_FP64, args.fp64_steps,
             stream, last, tol=args.fp64_tol, warm=False)
        if "value" in res["fp64_gpu_path"]:
            res["fp64_gpu_path"]["mixed_over_fp64"] = value / ws / res["fp64_gpu_path"]["value"]
        for name in ("fp16", "bf16"):
            _leg(res, name + "_path", leg_precision, vie, torch, local, cell, eps, PRECISIONS[name], 5, stream, last)
        _leg(res, "preconditioner_fig2", leg_preconditioner, vie, local, cell, eps, stream, last)
        if rank == 0:
            _leg(res, "sweep", leg_sweep, vie, torch, local, args.sweep_points, args.slots)
            _leg(res, "serving", leg_serve, vie, torch, local, args.serve_requests, 4)
            if not args.no_large:
                _leg(res, "large_cell", leg_large, vie, torch, local, vie.VIE_FP16, stream)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        res["cpu_baseline"] = cpu_baseline(args, cell, vie, torch, local, stream, value)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


# Per g_p value of the far tetrahedron-pair kernels (16 values per ordered pair
# of tetrahedra), counted with ncu on the plasmonic geometry at sweep density
# (4860 tets), lambda = 500 nm, at the default Ewald split (the series has the
# same terms per value for every cell of this period, wavelength and incidence
# class): executed warp instructions and FP32 operations (2 FFMA + FADD + FMUL,
# thread level).  Normal incidence: k_far_tt_n (split 1.5); oblique incidence
# at theta = 0.3 rad, phi = 0: k_far_tt_o, the k_y = 0 fold (split 1.0).  With
# another split (the autotuner's choice) the counts do not apply and the
# issue-rate figures are left out.
FAR_COUNTS = {"normal": (13.61, 279.2, 1.5), "oblique": (34.09, 512.2, 1.0)}
FAR_SPLIT_CHOSEN = None   # set by the main leg from its autotune report
SMS, FP32_LANES, SCHEDULERS = 152, 128, 4
MATVEC_Z_TRAFFIC = 3.5527e9   # DRAM read + write per FP32 Z product, 21,024 unknowns (ncu)


Z_BYTES = {0: 16, 1: 8, 2: 4, 3: 4}   # bytes per complex entry of the Z the GMRES products read, per precision


def roofline(last, n, peaks, prec, n_tets):
    """Roofline of the dominant kernel (largest device time in the solve), plus the others.

    k_far_tt (far tetrahedron pairs of the fill): instruction-issue bound ("alu");
    achieved = warp instructions per value (FAR_COUNTS) x 16 n_tets^2 values / event time, against
    152 SMs x 4 schedulers x 1 warp instruction per clock x the maximum SM
    clock; the FP32 rate (FAR_COUNTS) is reported beside it.
    k_tc_update (tensor-core products of the block inversion of Eq. (6), FP16
    operands, FP32 accumulation): K = 512 complex, ~256 flop per byte of the
    updated block (near the ridge); algorithmic bytes = read and write of the updated block +
    one read of the two packed FP16 operand panels, per launch; the roof is
    whichever of HBM and the FP16 tensor rate binds for those bytes and flops.
    k_matvec (GMRES Z products and block-inverse products): HBM-bound; bytes =
    N ld 8 B (FP32 Z) + the two vectors per Z product, one read of every block
    inverse + the vectors per preconditioner application.
    """
    peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    out = {}
    fp32 = prec != 0          # the FP32 fill kernels (every precision but FP64)
    cls = "normal" if THETA == 0.0 else "oblique"
    winst, flops, split0 = FAR_COUNTS[cls]
    counted = (FAR_SPLIT_CHOSEN in (None, split0)) and (THETA == 0.0 or abs(THETA - 0.3) < 1e-6) and PHI == 0.0
    if last.get("k_far_tt_ms") and fp32 and counted:
        # instruction-issue bound (a mix of FP32, integer and load instructions):
        # warp instructions per value x values / event time, against 152 SMs x 4
        # schedulers x 1 warp instruction per clock x the maximum SM clock
        t = last["k_far_tt_ms"] / 1e3
        clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        vals = 16.0 * n_tets * n_tets
        ipeak = SMS * SCHEDULERS * clk / 1e9
        ach = winst * vals / t / 1e9
        fpeak = float(peaks.get("fp32_fma_tflops") or SMS * FP32_LANES * 2 * clk / 1e12)
        out["k_far_tt"] = {"bound": "alu", "kernel": "k_far_tt", "achieved": ach, "peak": ipeak,
                           "unit": "Gwarp-inst/s", "frac": ach / ipeak, "traffic": None,
                           "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction/clock x %.0f MHz"
                                          % (clk / 1e6),
                           "fp32_tflops": flops * vals / t / 1e12,
                           "fp32_frac": flops * vals / t / 1e12 / fpeak,
                           "fp32_peak_tflops": fpeak,
                           "fp32_peak_source": "measured FMA loop (vie_fma_peak)" if peaks.get("fp32_fma_tflops")
                                               else "derived: 152 x 128 lanes x 2 x max clock",
                           "total_ms": last["k_far_tt_ms"], "launches": 1, "gp_values_per_s": vals / t}
    if last.get("k_tc_n"):
        # bound = whichever roof is lower for the algorithmic bytes and flops:
        # HBM at the measured copy bandwidth, or FP16 tensor cores at the
        # measured sustained bf16 rate (FP16 and bf16 have the same nominal rate)
        t = last["k_tc_ms"] / 1e3
        b, f = last["k_tc_bytes"], last.get("k_tc_flops", 0.0)
        tpeak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        t_hbm = b / (peak * 1e9)
        t_tc = f / (tpeak * 1e12)
        if t_tc > t_hbm:
            ach = f / t / 1e12
            out["k_tc_update"] = {"bound": "tensor", "kernel": "k_tc_update", "achieved": ach, "peak": tpeak,
                                  "unit": "TFLOP/s", "frac": ach / tpeak, "traffic": None,
                                  "peak_source": "measured bf16 sustained (FP16 operands)",
                                  "hbm_gbs": b / t / 1e9, "hbm_frac": b / t / 1e9 / peak}
        else:
            ach = b / t / 1e9
            out["k_tc_update"] = {"bound": "hbm", "kernel": "k_tc_update", "achieved": ach, "peak": peak,
                                  "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": src,
                                  "tensor_tflops": f / t / 1e12, "tensor_frac": f / t / 1e12 / tpeak}
        out["k_tc_update"].update({"total_ms": last["k_tc_ms"], "launches": last["k_tc_n"]})
    if last["k_matvec_n"]:
        # the Z products of GMRES and the block-inverse products of the
        # preconditioner applications (the same kernel)
        ld = (n + 3) // 4 * 4
        zb = Z_BYTES[prec]
        bytes_z = last["k_matvec_n"] * (n * ld * zb + n * 2 * (8 if fp32 else 16) * 2)
        tot_ms = last["k_matvec_ms"] + last.get("k_precond_ms", 0.0)
        tot_b = bytes_z + last.get("k_precond_bytes", 0.0)
        ach = tot_b / (tot_ms / 1e3) / 1e9
        # DRAM bytes per Z product from one ncu capture of this workload (its
        # summary is under profiles/); other workloads: not captured
        traffic = MATVEC_Z_TRAFFIC if (n == 21024 and prec == 1) else None
        out["k_matvec"] = {"bound": "hbm", "kernel": "k_matvec", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "traffic": traffic, "traffic_unit": "bytes per Z product",
                           "algorithmic_bytes_per_z_product": n * ld * zb + n * 2 * (8 if fp32 else 16) * 2,
                           "peak_source": src, "total_ms": tot_ms,
                           "launches": last["k_matvec_n"], "precond_applications": last.get("k_precond_n", 0),
                           "z_products_gbs": bytes_z / (last["k_matvec_ms"] / 1e3) / 1e9}
    if not out:
        return None, out
    dom = max(out.values(), key=lambda r: r["total_ms"])
    return dict(dom), out


def run_sweep(args):
    """Batched wavelength x angle sweep through vie_solve_batch (several solve
    slots in flight); a step is one (lambda, theta) solve, TE and TM together."""
    import torch

    from paper_1809_05334_gb300 import vie

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = PRECISIONS[args.precision]
    cell = _cell("sweep_cell")
    solver = vie.Solver(device=local, precision=prec, tol=1e-6, autotune=True)   # tuned in the warm-up
    n = solver.set_mesh(cell)
    steps = args.steps
    lams, ths = sweep_requests(max(steps, args.warmup))
    eps = [cell.eps(l) for l in lams]
    phs = [0.0] * len(lams)
    w = args.warmup
    solver.solve_batch(lams[:w], ths[:w], phs[:w], eps[:w], max_slots=args.slots)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        out, used = solver.solve_batch(lams[:steps], ths[:steps], phs[:steps], eps[:steps], max_slots=args.slots)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    lat = [o["t_fill_ms"] + o["t_factor_ms"] + o["t_solve_ms"] + o["t_post_ms"] for o in out]
    bad = [o["status"] for o in out if o["status"] != 0]
    res = {
        "metric": METRIC, "value": steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": w, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64" if prec == vie.VIE_FP32 else "c128", "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD, "n_unknowns": n, "n_tets": cell.n_tets, "precision": args.precision,
                   "slots": used, "parallelism": "single",
                   "l2": "inputs larger than L2 (each slot's Z is %.2f GB)"
                         % (n * n * (8 if prec == vie.VIE_FP32 else 16) / 1e9)},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "note": "per solve, wall time inside the batch with %d slots in flight" % used},
        "iterations_mean": float(np.mean([sum(o["iterations"]) / 2 for o in out])),
        "max_rel_residual": float(max(np.max(o["rel_residual"]) for o in out)),
        "non_ok_status": bad,
        "absorbed_active_first": [float(v) for v in out[0]["A"][:, cell.active_domain]],
        "gpu_launches": int(sum(o["n_launches"] for o in out)),
        "clocks": clk.summary(),
    }
    solver.close()
    if args.compare_fp64 and prec == vie.VIE_FP32:
        # the plain FP64 GPU path (FP64 Z, FP64 Krylov, tolerance 1e-10) on the
        # first requests of the same sweep, with the same slots: its throughput
        # and the absorption difference of the mixed-precision results
        k = min(args.compare_fp64, steps)
        s64 = vie.Solver(device=local, precision=vie.VIE_FP64, tol=1e-10)
        s64.set_mesh(cell)
        s64.solve_batch(lams[:1], ths[:1], phs[:1], eps[:1], max_slots=1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        o64, used64 = s64.solve_batch(lams[:k], ths[:k], phs[:k], eps[:k], max_slots=args.slots)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        s64.close()
        dA = max(float(np.max(np.abs(a["A"] - b["A"]))) for a, b in zip(out[:k], o64))
        res["fp64_gpu_path"] = {"solves": k, "slots": used64, "value": k / dt, "unit": UNIT,
                                "mixed_over_fp64": (steps / (ms / 1e3)) / (k / dt),
                                "max_abs_dA_mixed_vs_fp64": dA,
                                "fp64_max_rel_residual": float(max(np.max(o["rel_residual"]) for o in o64))}
    print(json.dumps(res))


SERVE_WORKLOAD = ("serving stream: Poisson arrivals (mean 200 req/s) of solves on seeded random cells (square "
                  "period 150-400 nm, 0-4 Ag spheres r 10-40 nm, active and buffer layers 30-150 nm, ~2k-40k "
                  "unknowns), lambda U[400,800] nm, theta U[0,80] deg, TE+TM per solve")


def serve_requests(k, rate=200.0, master_seed=4):
    """The first k requests of the serving stream: (arrival time s, cell, lambda, theta).
    A lambda within 1e-3/a of a Rayleigh anomaly (|gamma_pq| a < 1e-3) is moved
    up in 0.01 nm steps."""
    import cellgen
    rng = np.random.default_rng([master_seed, 1 << 20])
    t = np.cumsum(rng.exponential(1.0 / rate, size=k))
    out = []
    for i in range(k):
        cell, _ = cellgen.serving_cell(i, master_seed)
        r = np.random.default_rng([master_seed, i, 1])
        lam, th = float(r.uniform(400.0, 800.0)), float(r.uniform(0.0, np.deg2rad(80.0)))
        a = cell.period_a
        while True:
            k0 = 2 * np.pi / lam
            p = np.arange(-4, 5)
            kx = k0 * np.sin(th) + 2 * np.pi * p[:, None] / a
            ky = 2 * np.pi * p[None, :] / a
            if np.min(np.abs(np.sqrt((kx ** 2 + ky ** 2 - k0 ** 2).astype(complex)))) * a >= 1e-3:
                break
            lam += 0.01
        out.append((float(t[i]), cell, lam, th))
    return out


def run_serve(args):
    """Serving stream through the solve server (vie_server_*): requests are
    submitted at their Poisson arrival times; value = requests / (last completion
    - first arrival); latency from submission to completion, queueing included."""
    import torch

    from paper_1809_05334_gb300 import vie

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    prec = PRECISIONS[args.precision]
    reqs = serve_requests(args.steps)
    srv = vie.Server(device=local, n_slots=args.slots, precision=prec, tol=1e-6)
    import cellgen
    warm = cellgen.small_cells()["plasmonic_tiny"]
    for _ in range(args.warmup):
        t, _ = srv.submit(warm, 500.0, 0.0, 0.0, warm.eps(500.0))
        srv.poll(t, wait_ms=-1)
    torch.cuda.synchronize()
    tickets = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for at, cell, lam, th in reqs:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            tk, fp = srv.submit(cell, lam, th, 0.0, cell.eps(lam))
            tickets.append((tk, fp, cell))
        out = [srv.poll(tk, wait_ms=-1) for tk, _, _ in tickets]
        elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = [o["t_latency_ms"] for o in out]
    ns = [o["n"] for o in out]
    res = {
        "metric": METRIC, "value": len(out) / elapsed, "unit": UNIT, "n_gpus": 1, "steps": len(out),
        "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / len(out), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if prec == vie.VIE_FP32 else "c128",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "slots": args.slots, "precision": args.precision,
                   "unknowns_min_median_max": [int(min(ns)), int(np.median(ns)), int(max(ns))],
                   "parallelism": "single", "l2": "inputs larger than L2 (Z of 26 MB to 13 GB per request)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "note": "submission to completion, queueing included"},
        "server": {k: st[k] for k in ("max_running", "peak_reserved_bytes", "budget_bytes", "completed")},
        "non_ok_status": [o["status"] for o in out if o["status"] != 0],
        "max_rel_residual": float(max(np.max(o["rel_residual"]) for o in out)),
        "gpu_launches": int(sum(o["n_launches"] for o in out)),
        "timing": "host wall clock (several streams and host threads in flight)",
        "clocks": clk.summary(),
    }
    print(json.dumps(res))


ENH_WORKLOAD = ("enhancement and angular response (Sec. 3, Fig. 4, 6): Ag cubes W = 40 nm centred in a 60 nm "
                "active layer over a 20 nm spacer, square lattice a = 50-80 nm, each cell solved with and without "
                "the particle (same mesh, the cube filled with the active material), synthetic Drude/Cauchy eps")


def run_enhancement(args):
    """Absorption enhancement A_active(with NP) / A_active(without NP) over the
    wavelength for lattice constants a = 50, 60, 70, 80 nm at normal incidence
    (Fig. 4), and the angular response at 500, 600 and 750 nm for theta = 0-80
    deg (Fig. 6): the active layer's absorption normalised to theta = 0, beside
    the Lambertian cos(theta).  Absorption is Eq. (7) over the active material
    only; "without NP" integrates over the cube's volume too (it is active
    material there).  Every solve goes through vie_solve_batch (slots in
    flight); TE and TM are averaged (unpolarised sunlight)."""
    import torch

    import cellgen
    from paper_1809_05334_gb300 import vie
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    lams = [400.0 + 20.0 * i for i in range(21)]
    out = {"metric": "absorption enhancement and angular response", "unit": "ratio", "data": "synthetic",
           "config": {"workload": ENH_WORKLOAD, "lambda_nm": lams, "h_nm": 10.0}, "spectra": {}, "angular": {}}
    t0 = time.perf_counter()
    n_solves = 0
    with_A = {}
    for a in (50.0, 60.0, 70.0, 80.0):
        cw = cellgen.cube_cell(a, 20.0, 60.0, 40.0, 10.0, 10.0, particle=True)
        co = cellgen.cube_cell(a, 20.0, 60.0, 40.0, 10.0, 10.0, particle=False)
        s = vie.Solver(device=local, precision=vie.VIE_FP32, tol=1e-6)
        try:
            s.set_mesh(cw)
            rw, _ = s.solve_batch(lams, [0.0] * len(lams), [0.0] * len(lams), [cw.eps(l) for l in lams],
                                  max_slots=args.slots)
            s.set_mesh(co)
            ro, _ = s.solve_batch(lams, [0.0] * len(lams), [0.0] * len(lams), [co.eps(l) for l in lams],
                                  max_slots=args.slots)
        finally:
            s.close()
        n_solves += 2 * len(lams)
        aw = [float(np.mean(r["A"][:, 1])) for r in rw]
        ao = [float(np.mean(r["A"][:, 1] + r["A"][:, 2])) for r in ro]
        with_A[a] = aw
        enh = [w / o for w, o in zip(aw, ao)]
        out["spectra"]["a=%g" % a] = {"A_with": aw, "A_without": ao, "enhancement": enh,
                                      "max_enhancement": max(enh), "at_lambda_nm": lams[int(np.argmax(enh))],
                                      "status": sorted({r["status"] for r in rw + ro})}
    thetas = [10.0 * i for i in range(9)]
    cw = cellgen.cube_cell(60.0, 20.0, 60.0, 40.0, 10.0, 10.0, particle=True)
    s = vie.Solver(device=local, precision=vie.VIE_FP32, tol=1e-6)
    try:
        s.set_mesh(cw)
        for lam in (500.0, 600.0, 750.0):
            r, _ = s.solve_batch([lam] * len(thetas), [np.deg2rad(t) for t in thetas], [0.0] * len(thetas),
                                 [cw.eps(lam)] * len(thetas), max_slots=args.slots)
            n_solves += len(thetas)
            a = [float(np.mean(x["A"][:, 1])) for x in r]
            out["angular"]["lambda=%g" % lam] = {"theta_deg": thetas, "A": a, "normalised": [v / a[0] for v in a],
                                                  "cos_theta": [float(np.cos(np.deg2rad(t))) for t in thetas]}
    finally:
        s.close()
    dt = time.perf_counter() - t0
    out["solves"] = n_solves
    out["value"] = n_solves / dt
    out["value_unit"] = UNIT
    out["wall_s"] = dt
    print(json.dumps(out))


def cpu_baseline(args, cell, vie, torch, local, stream, gpu_value):
    """The FP64 oracle on the host cores: timed whole on a bounded sample of the
    same geometry (378 tetrahedra), and extrapolated to the full workload; the
    GPU path timed on that same sample gives the same-workload ratio."""
    sample, n_s, t = oracle_sample(cell)
    cores = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    out = {"value": 1.0 / t["extrapolated_s"], "unit": UNIT, "cores": cores, "kind": "oracle, extrapolated",
           "sample": "one oracle solve of the same geometry at %d tets / %d unknowns took %.1f s (fill %.1f s, "
                     "dense LU %.3f s); extrapolated to %d tets by the tetrahedron-pair ratio %.0f (fill) and the "
                     "cube of the unknown ratio %.0f (LU)"
                     % (sample.n_tets, n_s, t["total_s"], t["fill_s"], t["lu_s"], cell.n_tets, t["scale_fill"],
                        t["scale_lu"]),
           "measured": {"value": 1.0 / t["total_s"], "unit": UNIT, "kind": "oracle", "n_tets": sample.n_tets,
                        "n_unknowns": n_s, "seconds": t["total_s"]}}
    try:
        g = leg_same_workload(vie, torch, local, sample, stream)
        out["measured"]["gpu_same_sample"] = g
        out["measured"]["gpu_over_oracle_same_sample"] = g["value"] * t["total_s"]
    except Exception as e:   # noqa: BLE001
        out["measured"]["gpu_same_sample"] = {"error": str(e)}
    return out


def run_reference(args):
    """The FP64 oracle (the plain restatement of the method, dense LU) on the host
    cores: each step is one oracle solve of a bounded sample of the workload (the
    plasmonic geometry at 378 tetrahedra); `ms_per_step` is that measured step,
    `value` the throughput it extrapolates to the full workload."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    full = _cell(args.workload)
    import cellgen
    from oracle import solve_cell
    warm = cellgen.small_cells()["slab_3x3x1"]
    for _ in range(args.warmup):   # untimed: starts the oracle's worker pool (a small cell keeps the run short)
        solve_cell(warm, LAM, THETA, PHI)
    runs = [oracle_sample(full) for _ in range(args.steps)]
    sample, n_s = runs[0][0], runs[0][1]
    step_s = float(np.mean([r[2]["total_s"] for r in runs]))
    ext_s = float(np.mean([r[2]["extrapolated_s"] for r in runs]))
    value = 1.0 / ext_s
    cores = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    t = runs[0][2]
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "value_basis": "each step is one oracle solve of a %d-tet sample (ms_per_step, measured); value is the "
                          "throughput that extrapolates to the %d-tet workload (fill x%.0f, LU x%.0f)"
                          % (sample.n_tets, full.n_tets, t["scale_fill"], t["scale_lu"]),
           "config": {"workload": WORKLOADS[args.workload][1], "sample_tets": sample.n_tets,
                      "sample_unknowns": n_s, "full_tets": full.n_tets},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle, extrapolated",
                            "sample": "each step: one oracle solve of the geometry at %d tets (%.1f s measured); "
                                      "value extrapolated to the %d-tet workload" % (sample.n_tets, step_s, full.n_tets),
                            "measured": {"value": 1.0 / step_s, "unit": UNIT, "kind": "oracle",
                                         "n_tets": sample.n_tets, "n_unknowns": n_s}},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed solves (default 5; 81 with --sweep)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="plasmonic", choices=sorted(WORKLOADS))
    ap.add_argument("--sweep", action="store_true",
                    help="batched wavelength x angle sweep on the sweep-density cell (vie_solve_batch)")
    ap.add_argument("--slots", type=int, default=3, help="solve slots in flight for --sweep / --serve")
    ap.add_argument("--compare-fp64", type=int, default=0, metavar="K",
                    help="with --sweep: also time the FP64 GPU path on the first K requests and compare")
    ap.add_argument("--serve", action="store_true",
                    help="serving stream of random cells through the solve server (vie_server_*)")
    ap.add_argument("--main-only", action="store_true", help="only the timed main leg (no side legs)")
    ap.add_argument("--large", action="store_true",
                    help="the large cell's lambda x theta sweep (~90k unknowns, one solve at a time)")
    ap.add_argument("--no-large", action="store_true", help="leave the large-cell leg out of the default run")
    ap.add_argument("--enhancement", action="store_true",
                    help="absorption enhancement spectra and angular response of the cube cells (Fig. 4, 6)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed solves of the FP64 GPU path leg")
    ap.add_argument("--fp64-tol", type=float, default=1e-8, help="FP64 residual tolerance of the FP64 leg")
    ap.add_argument("--sweep-points", type=int, default=27, help="sweep points of the default run's sweep leg")
    ap.add_argument("--serve-requests", type=int, default=12, help="requests of the default run's serving leg")
    ap.add_argument("--theta-deg", type=float, default=0.0,
                    help="incidence angle of the main workload (default 0: the bench configuration)")
    args = ap.parse_args()
    if args.theta_deg != 0.0:
        global THETA
        THETA = float(np.deg2rad(args.theta_deg))
    if args.steps is None:
        args.steps = 81 if args.sweep else (24 if args.serve else 5)
    if args.impl == "reference":
        run_reference(args)
    elif args.enhancement:
        run_enhancement(args)
    elif args.large:
        run_large(args)
    elif args.sweep:
        run_sweep(args)
    elif args.serve:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
