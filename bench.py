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
UNIT = "solves/s"
LAM, THETA, PHI = 500.0, 0.0, 0.0
WORKLOADS = {
    "plasmonic": ("config_plasmonic",
                  "plasmonic cell 200 nm period, Ag sphere r=20 nm in 100 nm active over 40 nm buffer, "
                  "~21k unknowns, lambda=500 nm, theta=0, TE+TM"),
    # the same cell with the Ag sphere meshed as a mapped cube (smooth particle surface)
    "plasmonic_ball": ("config_plasmonic_ball",
                       "plasmonic cell 200 nm period, Ag sphere r=20 nm (mapped-cube mesh) in 100 nm active over "
                       "40 nm buffer, ~35.6k unknowns, lambda=500 nm, theta=0, TE+TM"),
    # the same geometry at the sweep density (~8.9k unknowns): a smaller case for profiling
    "sweep_cell": ("config_sweep_geometry",
                   "plasmonic cell 200 nm period at sweep density (~8.9k unknowns), lambda=500 nm, theta=0, TE+TM"),
}


SWEEP_WORKLOAD = ("batched sweep on the plasmonic geometry at sweep density (~8.9k unknowns): lambda 400-800 nm "
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
    prec = vie.VIE_FP32 if args.precision == "fp32" else vie.VIE_FP64
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
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
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
    te = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    h2d //= e2e_steps
    d2h //= e2e_steps

    value = ws * args.steps / (ms_max / 1e3)
    peaks = _peaks()
    # roofline: the kernel with the largest device time in the solve (see roofline())
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64" if args.precision == "fp32" else "c128",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "n_unknowns": n, "n_tets": cell.n_tets, "precision": args.precision,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (Z is %.1f GB)" % (n * n * (8 if prec == vie.VIE_FP32 else 16) / 1e9)},
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
        "e2e": {"value": ws * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": None,
    }
    res["roofline"], res["rooflines"] = roofline(last, n, peaks, prec == vie.VIE_FP32, cell.n_tets)
    res["clocks"] = clk.summary()
    # kernels launched inside the timed region, counted by the library at each launch site
    res["gpu_launches"] = int(sum(r["n_launches"] for r in results))
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        res["cpu_baseline"] = cpu_baseline(args)
    solver.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


# Per g_p value of the far tetrahedron-pair kernel (16 values per ordered pair
# of tetrahedra), counted with ncu on the plasmonic 21k workload at 500 nm,
# normal incidence (the Ewald series has the same terms per value for every
# cell of this period, wavelength and incidence): executed FP32 operations
# (2 FFMA + FADD + FMUL, thread level) and executed warp instructions.
FAR_FLOPS_PER_VALUE = 429.5
FAR_WINST_PER_VALUE = 32.44
SMS, FP32_LANES, SCHEDULERS = 152, 128, 4
MATVEC_Z_TRAFFIC = 3.5527e9   # DRAM read + write per FP32 Z product, 21,024 unknowns (ncu)


def roofline(last, n, peaks, fp32, n_tets):
    """Roofline of the dominant kernel (largest device time in the solve), plus the others.

    k_far_tt (far tetrahedron pairs of the fill): instruction-issue bound ("alu");
    achieved = FAR_WINST_PER_VALUE x 16 n_tets^2 values / event time, against
    152 SMs x 4 schedulers x 1 warp instruction per clock x the maximum SM
    clock; the FP32 rate (FAR_FLOPS_PER_VALUE) is reported beside it.
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
    if last.get("k_far_tt_ms") and fp32:
        # instruction-issue bound (a mix of FP32, integer and load instructions):
        # warp instructions per value x values / event time, against 152 SMs x 4
        # schedulers x 1 warp instruction per clock x the maximum SM clock
        t = last["k_far_tt_ms"] / 1e3
        clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        vals = 16.0 * n_tets * n_tets
        ipeak = SMS * SCHEDULERS * clk / 1e9
        ach = FAR_WINST_PER_VALUE * vals / t / 1e9
        fpeak = SMS * FP32_LANES * 2 * clk / 1e12
        out["k_far_tt"] = {"bound": "alu", "kernel": "k_far_tt", "achieved": ach, "peak": ipeak,
                           "unit": "Gwarp-inst/s", "frac": ach / ipeak, "traffic": None,
                           "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction/clock x %.0f MHz"
                                          % (clk / 1e6),
                           "fp32_tflops": FAR_FLOPS_PER_VALUE * vals / t / 1e12,
                           "fp32_frac": FAR_FLOPS_PER_VALUE * vals / t / 1e12 / fpeak,
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
        zb = 8 if fp32 else 16
        bytes_z = last["k_matvec_n"] * (n * ld * zb + n * 2 * (8 if fp32 else 16) * 2)
        tot_ms = last["k_matvec_ms"] + last.get("k_precond_ms", 0.0)
        tot_b = bytes_z + last.get("k_precond_bytes", 0.0)
        ach = tot_b / (tot_ms / 1e3) / 1e9
        # DRAM bytes per Z product from one ncu capture of this workload (its
        # summary is under profiles/); other workloads: not captured
        traffic = MATVEC_Z_TRAFFIC if (n == 21024 and fp32) else None
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
    prec = vie.VIE_FP32 if args.precision == "fp32" else vie.VIE_FP64
    cell = _cell("sweep_cell")
    solver = vie.Solver(device=local, precision=prec, tol=1e-6)
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
    prec = vie.VIE_FP32 if args.precision == "fp32" else vie.VIE_FP64
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


def cpu_baseline(args):
    """The FP64 oracle on a reduced-density sample of the same cell, scaled to the full workload."""
    import cellgen
    from oracle import solve_cell
    sample = cellgen.config_plasmonic_sample()
    full = _cell(args.workload)                          # scaled to the workload being timed
    t0 = time.perf_counter()
    solve_cell(sample, LAM, THETA, PHI)
    dt = time.perf_counter() - t0
    scale = (full.n_tets / sample.n_tets) ** 2          # the fill dominates: pairs of tetrahedra
    cores = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one oracle solve of the same geometry at reduced density (%d tets vs %d) took %.1f s; "
                      "scaled by the tetrahedron-pair ratio %.0f" % (sample.n_tets, full.n_tets, dt, scale)}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    import cellgen
    from oracle import solve_cell
    sample = cellgen.config_plasmonic_sample()
    full = _cell(args.workload)                          # scaled to the workload being timed
    scale = (full.n_tets / sample.n_tets) ** 2
    for _ in range(args.warmup):
        solve_cell(sample, LAM, THETA, PHI)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solve_cell(sample, LAM, THETA, PHI)
    dt = (time.perf_counter() - t0) / args.steps
    value = 1.0 / (dt * scale)
    cores = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * scale * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": WORKLOADS["plasmonic"][1], "sample_tets": sample.n_tets, "full_tets": full.n_tets},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "each step: one oracle solve of the geometry at %d tets; value scaled by "
                                      "the tetrahedron-pair ratio %.0f to the %d-tet workload"
                                      % (sample.n_tets, scale, full.n_tets)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed solves (default 5; 81 with --sweep)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="plasmonic", choices=sorted(WORKLOADS))
    ap.add_argument("--sweep", action="store_true",
                    help="batched wavelength x angle sweep on the sweep-density cell (vie_solve_batch)")
    ap.add_argument("--slots", type=int, default=3, help="solve slots in flight for --sweep / --serve")
    ap.add_argument("--compare-fp64", type=int, default=0, metavar="K",
                    help="with --sweep: also time the FP64 GPU path on the first K requests and compare")
    ap.add_argument("--serve", action="store_true",
                    help="serving stream of random cells through the solve server (vie_server_*)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 81 if args.sweep else (24 if args.serve else 5)
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.serve:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
