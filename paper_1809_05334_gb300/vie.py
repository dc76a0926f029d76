"""ctypes binding of libvie.so (include/vie.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts numpy arrays to pointers and C structs back to Python values.  There
is no fallback: if the library is missing or no GPU is present, the calls
raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvie.so")
MAX_DOMAINS = 8

VIE_FP64, VIE_FP32, VIE_FP16, VIE_BF16 = 0, 1, 2, 3
VIE_PENDING = 2
VIE_CANCELLED = -7
STATUS = {0: "VIE_OK", 1: "VIE_NOT_CONVERGED", 2: "VIE_PENDING", -1: "VIE_EINVAL", -2: "VIE_ENOMEM", -3: "VIE_ECUDA",
          -4: "VIE_RAYLEIGH_ANOMALY", -5: "VIE_DEVICE_TIMEOUT", -6: "VIE_BAD_MESH", -7: "VIE_CANCELLED",
          -8: "VIE_BREAKDOWN"}

# every symbol include/vie.h declares
EXPORTS = ["vie_default_options", "vie_create", "vie_set_options", "vie_set_mesh", "vie_num_unknowns",
           "vie_solve", "vie_fill_matrix", "vie_fill_matrix_prec", "vie_erfcx", "vie_green",
           "vie_status_str", "vie_last_error", "vie_destroy", "vie_green_noalloc", "vie_solve_batch",
           "vie_server_create", "vie_server_submit", "vie_server_poll", "vie_server_get_stats",
           "vie_server_destroy", "vie_server_cancel", "vie_domain_block", "vie_fma_peak",
           "vie_check_device_wait", "vie_tune"]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("use_precond", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("timing", ctypes.c_int32), ("precond_block_max", ctypes.c_int32), ("precond_pivot", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("incidence_class", ctypes.c_int32), ("n_split", ctypes.c_int32), ("split", ctypes.c_double * 4),
                ("fill_ms", ctypes.c_double * 4), ("split_chosen", ctypes.c_double), ("n_mv", ctypes.c_int32),
                ("mv_grid", ctypes.c_int32 * 4), ("mv_ms", ctypes.c_double * 4), ("mv_chosen", ctypes.c_int32),
                ("n_pivot", ctypes.c_int32), ("pivot", ctypes.c_int32 * 2), ("factor_ms", ctypes.c_double * 2),
                ("pivot_chosen", ctypes.c_int32), ("tune_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("lambda_nm", ctypes.c_double), ("theta", ctypes.c_double), ("phi", ctypes.c_double),
                ("eps", ctypes.c_double * (2 * MAX_DOMAINS)), ("coeffs_out", ctypes.c_void_p),
                ("coeffs_on_device", ctypes.c_int32), ("density_on_device", ctypes.c_int32),
                ("density_out", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_unknowns", ctypes.c_int32), ("iterations", ctypes.c_int32 * 2),
                ("refinements", ctypes.c_int32), ("rel_residual", ctypes.c_double * 2),
                ("absorbed", (ctypes.c_double * MAX_DOMAINS) * 2), ("reflectance", ctypes.c_double * 2),
                ("transmittance", ctypes.c_double * 2), ("t_fill_ms", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double), ("t_post_ms", ctypes.c_double),
                ("k_far_tt_ms", ctypes.c_double), ("k_fill_ms", ctypes.c_double), ("k_factor_ms", ctypes.c_double),
                ("k_matvec_ms", ctypes.c_double), ("k_matvec_n", ctypes.c_int32), ("n_near_pairs", ctypes.c_int32),
                ("far_pair_evals", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("k_tc_ms", ctypes.c_double), ("k_tc_bytes", ctypes.c_double), ("k_tc_n", ctypes.c_int32),
                ("n_launches", ctypes.c_int32), ("t_queue_ms", ctypes.c_double),
                ("t_latency_ms", ctypes.c_double), ("k_precond_ms", ctypes.c_double),
                ("k_precond_bytes", ctypes.c_double), ("k_precond_n", ctypes.c_int32),
                ("reserved3", ctypes.c_int32), ("k_tc_flops", ctypes.c_double),
                ("k_ortho_ms", ctypes.c_double)]


class Mesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int32), ("tets", ctypes.c_void_p),
                ("n_tets", ctypes.c_int32), ("tet_domain", ctypes.c_void_p), ("n_domains", ctypes.c_int32),
                ("active_domain", ctypes.c_int32), ("period_a", ctypes.c_double), ("period_b", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "rejected", "queued", "running",
                                              "max_running", "budget_bytes", "reserved_bytes",
                                              "peak_reserved_bytes", "cancelled")]


_LIB = None


def load():
    """Load libvie.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError("libvie.so not built: run `python -m paper_1809_05334_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.vie_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.vie_default_options.restype = None
    lib.vie_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(Options)]
    lib.vie_set_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.vie_set_mesh.argtypes = [P, P, I, P, I, P, I, D, D, I]
    lib.vie_num_unknowns.argtypes = [P]
    lib.vie_num_unknowns.restype = I
    lib.vie_solve.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(Result), P]
    lib.vie_fill_matrix.argtypes = [P, ctypes.POINTER(Request), P, P, P]
    lib.vie_fill_matrix_prec.argtypes = [P, ctypes.POINTER(Request), P, P]
    lib.vie_erfcx.argtypes = [P, P, P, I, I]
    lib.vie_green.argtypes = [P, ctypes.POINTER(Request), P, P, I, I]
    lib.vie_status_str.argtypes = [ctypes.c_int]
    lib.vie_status_str.restype = ctypes.c_char_p
    lib.vie_last_error.argtypes = [P]
    lib.vie_last_error.restype = ctypes.c_char_p
    lib.vie_destroy.argtypes = [P]
    lib.vie_destroy.restype = None
    lib.vie_green_noalloc.argtypes = [D, D, D, D, D, D, P, P, I, I, P]
    lib.vie_solve_batch.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(Result), I, I,
                                    ctypes.POINTER(I), P]
    lib.vie_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(Options), I, ctypes.c_int64]
    lib.vie_server_submit.argtypes = [P, ctypes.POINTER(Mesh), ctypes.POINTER(Request),
                                      ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64)]
    lib.vie_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Result), I]
    lib.vie_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.vie_server_destroy.argtypes = [P]
    lib.vie_server_destroy.restype = None
    lib.vie_server_cancel.argtypes = [P, ctypes.c_uint64]
    lib.vie_domain_block.argtypes = [P, ctypes.POINTER(Request), I, ctypes.POINTER(I), P, P, P, P]
    lib.vie_fma_peak.argtypes = [ctypes.c_int, I, ctypes.POINTER(D)]
    lib.vie_check_device_wait.argtypes = [ctypes.c_int, I, I]
    lib.vie_tune.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(TuneReport), P]
    _LIB = lib
    return lib


def fma_peak(device=0, precision=VIE_FP32):
    """Measured FP32 / FP64 FMA peak of the device in TFLOP/s (vie_fma_peak)."""
    lib = load()
    out = ctypes.c_double(0.0)
    rc = lib.vie_fma_peak(int(device), int(precision), ctypes.byref(out))
    if rc != 0:
        raise VIEError(rc, "vie_fma_peak failed")
    return float(out.value)


def check_device_wait(device=0, arrive=False, polls=1000):
    """Status of one bounded device wait on a barrier that gets its arrival or
    never does (vie_check_device_wait): 0 (VIE_OK) or -5 (VIE_DEVICE_TIMEOUT)."""
    return int(load().vie_check_device_wait(int(device), int(bool(arrive)), int(polls)))


class VIEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Solver:
    """One library context on one GPU (vie_create ... vie_destroy)."""

    def __init__(self, device=0, precision=VIE_FP32, use_precond=True, restart=100, max_iter=1000,
                 tol=1e-6, inner_tol=0.0, timing=False, precond_block_max=0, autotune=False, precond_pivot=0):
        self.lib = load()
        self.opt = Options()
        self.lib.vie_default_options(ctypes.byref(self.opt))
        self.opt.precision, self.opt.use_precond = int(precision), int(bool(use_precond))
        self.opt.restart, self.opt.max_iter = int(restart), int(max_iter)
        self.opt.tol, self.opt.inner_tol = float(tol), float(inner_tol)
        self.opt.timing = int(bool(timing))
        self.opt.precond_block_max = int(precond_block_max)
        self.opt.autotune = int(bool(autotune))
        self.opt.precond_pivot = int(precond_pivot)
        self.ctx = ctypes.c_void_p()
        rc = self.lib.vie_create(ctypes.byref(self.ctx), int(device), ctypes.byref(self.opt))
        if rc != 0:
            raise VIEError(rc, "vie_create failed (is a CUDA GPU present?)")
        self.n_domains = 0
        self.n_tets = 0

    def _check(self, rc, allow_positive=False):
        if rc < 0 or (rc > 0 and not allow_positive):
            raise VIEError(rc, self.lib.vie_last_error(self.ctx).decode())
        return rc

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.opt, k, v)
        self._check(self.lib.vie_set_options(self.ctx, ctypes.byref(self.opt)))

    def set_mesh(self, cell):
        self._verts = np.ascontiguousarray(cell.verts, dtype=np.float64)
        self._tets = np.ascontiguousarray(cell.tets, dtype=np.int32)
        self._dom = np.ascontiguousarray(cell.tet_domain, dtype=np.int32)
        self.n_domains = int(cell.n_domains)
        self.n_tets = len(self._tets)
        self._check(self.lib.vie_set_mesh(self.ctx, _ptr(self._verts), len(self._verts), _ptr(self._tets),
                                          len(self._tets), _ptr(self._dom), self.n_domains,
                                          float(cell.period_a), float(cell.period_b), int(cell.active_domain)))
        return self.num_unknowns()

    def num_unknowns(self):
        return int(self.lib.vie_num_unknowns(self.ctx))

    def request(self, lam, theta=0.0, phi=0.0, eps=()):
        r = Request()
        r.lambda_nm, r.theta, r.phi = float(lam), float(theta), float(phi)
        for d, e in enumerate(np.asarray(eps, dtype=np.complex128)):
            r.eps[2 * d], r.eps[2 * d + 1] = e.real, e.imag
        return r

    def solve(self, lam, theta=0.0, phi=0.0, eps=(), coeffs=False, stream=None, density=False):
        """Solve at one incidence; returns a dict of absorbed fractions, R, T, residuals, timings
        (and, with density=True, the per-tetrahedron absorbed fractions [2, n_tets] as "density")."""
        req = self.request(lam, theta, phi, eps)
        out = None
        if coeffs is not False and coeffs is not None:
            if isinstance(coeffs, np.ndarray):
                out = coeffs
            else:
                out = np.zeros((self.num_unknowns(), 2), dtype=np.complex128)
            req.coeffs_out = out.ctypes.data
        dens = None
        if density:
            dens = np.zeros((2, self.n_tets), dtype=np.float64)
            req.density_out = dens.ctypes.data
        res = Result()
        rc = self.lib.vie_solve(self.ctx, ctypes.byref(req), ctypes.byref(res),
                                ctypes.c_void_p(stream) if stream else None)
        self._check(rc, allow_positive=True)
        r = self._result(res, rc, out)
        if density:
            r["density"] = dens
        return r

    def _result(self, res, rc, out=None):
        nd = self.n_domains
        return dict(status=rc, n=res.n_unknowns, iterations=list(res.iterations), refinements=res.refinements,
                    rel_residual=np.array(res.rel_residual[:]),
                    A=np.array([[res.absorbed[p][d] for d in range(nd)] for p in range(2)]),
                    R=np.array(res.reflectance[:]), T=np.array(res.transmittance[:]),
                    t_fill_ms=res.t_fill_ms, t_factor_ms=res.t_factor_ms, t_solve_ms=res.t_solve_ms,
                    t_post_ms=res.t_post_ms, k_far_tt_ms=res.k_far_tt_ms, k_fill_ms=res.k_fill_ms,
                    k_factor_ms=res.k_factor_ms, k_matvec_ms=res.k_matvec_ms, k_matvec_n=res.k_matvec_n,
                    n_near_pairs=res.n_near_pairs, far_pair_evals=res.far_pair_evals,
                    h2d_bytes=res.h2d_bytes, d2h_bytes=res.d2h_bytes, k_tc_ms=res.k_tc_ms,
                    k_tc_bytes=res.k_tc_bytes, k_tc_n=res.k_tc_n, n_launches=res.n_launches,
                    t_queue_ms=res.t_queue_ms, t_latency_ms=res.t_latency_ms, k_precond_ms=res.k_precond_ms,
                    k_precond_bytes=res.k_precond_bytes, k_precond_n=res.k_precond_n, k_tc_flops=res.k_tc_flops,
                    k_ortho_ms=res.k_ortho_ms, x=out)

    def tune(self, lam, theta=0.0, phi=0.0, eps=(), stream=None):
        """Autotune the schedule for this mesh and incidence class (vie_tune); returns
        the report as a dict: candidate split multipliers with their fill times,
        candidate product launch shapes with their times, and the choices."""
        req = self.request(lam, theta, phi, eps)
        rep = TuneReport()
        self._check(self.lib.vie_tune(self.ctx, ctypes.byref(req), ctypes.byref(rep),
                                      ctypes.c_void_p(stream) if stream else None))
        return dict(incidence_class=rep.incidence_class, split=list(rep.split[:rep.n_split]),
                    fill_ms=list(rep.fill_ms[:rep.n_split]), split_chosen=rep.split_chosen,
                    mv_grid=list(rep.mv_grid[:rep.n_mv]), mv_ms=list(rep.mv_ms[:rep.n_mv]),
                    mv_chosen=rep.mv_chosen, pivot=list(rep.pivot[:rep.n_pivot]),
                    factor_ms=list(rep.factor_ms[:rep.n_pivot]), pivot_chosen=rep.pivot_chosen, tune_ms=rep.tune_ms)

    def solve_batch(self, lams, thetas, phis, eps_list, max_slots=2, coeffs=False, stream=None):
        """Independent solves of one mesh (vie_solve_batch): lams/thetas/phis/eps_list
        have one entry per request; returns (list of result dicts, slots used).
        A request whose status is negative gets its dict with that status; the
        call raises only for errors of the batch itself."""
        n = len(lams)
        reqs = (Request * n)()
        outs = []
        for i in range(n):
            reqs[i] = self.request(lams[i], thetas[i], phis[i], eps_list[i])
            out = None
            if coeffs:
                out = np.zeros((self.num_unknowns(), 2), dtype=np.complex128)
                reqs[i].coeffs_out = out.ctypes.data
            outs.append(out)
        res = (Result * n)()
        used = ctypes.c_int32(0)
        rc = self.lib.vie_solve_batch(self.ctx, reqs, res, n, int(max_slots), ctypes.byref(used),
                                      ctypes.c_void_p(stream) if stream else None)
        if rc < 0 and not any(res[i].status == rc for i in range(n)):
            self._check(rc)
        return [self._result(res[i], res[i].status, outs[i]) for i in range(n)], int(used.value)

    def solve_device(self, lam, theta, phi, eps, coeffs_dev_ptr, stream=None):
        """Solve writing the unknowns to a caller-owned device buffer [N][2] complex128."""
        req = self.request(lam, theta, phi, eps)
        req.coeffs_out = int(coeffs_dev_ptr)
        req.coeffs_on_device = 1
        res = Result()
        rc = self.lib.vie_solve(self.ctx, ctypes.byref(req), ctypes.byref(res),
                                ctypes.c_void_p(stream) if stream else None)
        self._check(rc, allow_positive=True)
        return res

    def fill_matrix(self, lam, theta=0.0, phi=0.0, eps=()):
        """FP64 Z [N,N] and b [N,2] in canonical unknown order (parity entry point)."""
        n = self.num_unknowns()
        Z = np.zeros((n, n), dtype=np.complex128)
        b = np.zeros((n, 2), dtype=np.complex128)
        req = self.request(lam, theta, phi, eps)
        self._check(self.lib.vie_fill_matrix(self.ctx, ctypes.byref(req), _ptr(Z), _ptr(b), None))
        return Z, b

    def fill_matrix_prec(self, lam, theta=0.0, phi=0.0, eps=()):
        n = self.num_unknowns()
        Z = np.zeros((n, n), dtype=np.complex128)
        req = self.request(lam, theta, phi, eps)
        self._check(self.lib.vie_fill_matrix_prec(self.ctx, ctypes.byref(req), _ptr(Z), None))
        return Z

    def block_size(self, lam, theta=0.0, phi=0.0, eps=(), block=0):
        """Size of domain block `block` of Eq. (5) for this request (no fill)."""
        req = self.request(lam, theta, phi, eps)
        n = ctypes.c_int32(0)
        self._check(self.lib.vie_domain_block(self.ctx, ctypes.byref(req), int(block), ctypes.byref(n),
                                              None, None, None, None))
        return int(n.value)

    def domain_block(self, lam, theta=0.0, phi=0.0, eps=(), block=0):
        """(unknowns [n], Z_dd [n,n], computed inverse [n,n]) of domain block `block`
        of Eq. (5)-(6), as vie_solve inverts it (vie_domain_block)."""
        req = self.request(lam, theta, phi, eps)
        n = ctypes.c_int32(0)
        self._check(self.lib.vie_domain_block(self.ctx, ctypes.byref(req), int(block), ctypes.byref(n),
                                              None, None, None, None))
        idx = np.zeros(n.value, dtype=np.int32)
        Z = np.zeros((n.value, n.value), dtype=np.complex128)
        M = np.zeros((n.value, n.value), dtype=np.complex128)
        self._check(self.lib.vie_domain_block(self.ctx, ctypes.byref(req), int(block), ctypes.byref(n),
                                              _ptr(idx), _ptr(Z), _ptr(M), None))
        return idx, Z, M

    def erfcx(self, u, precision=VIE_FP64):
        u = np.ascontiguousarray(u, dtype=np.complex128)
        out = np.zeros_like(u)
        self._check(self.lib.vie_erfcx(self.ctx, _ptr(u), _ptr(out), u.size, int(precision)))
        return out

    def green(self, d, lam, theta=0.0, phi=0.0, precision=VIE_FP64):
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(len(d), dtype=np.complex128)
        req = self.request(lam, theta, phi, [1.0] * max(self.n_domains, 1))
        self._check(self.lib.vie_green(self.ctx, ctypes.byref(req), _ptr(d), _ptr(out), len(d), int(precision)))
        return out

    def close(self):
        if self.ctx:
            self.lib.vie_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Solve server (vie_server_*): continuous batching of independent solves,
    each request with its own mesh, in n_slots concurrent slots admitted by
    HBM footprint."""

    def __init__(self, device=0, n_slots=3, hbm_budget_bytes=0, precision=VIE_FP32, use_precond=True,
                 restart=100, max_iter=1000, tol=1e-6, inner_tol=0.0):
        self.lib = load()
        opt = Options()
        self.lib.vie_default_options(ctypes.byref(opt))
        opt.precision, opt.use_precond = int(precision), int(bool(use_precond))
        opt.restart, opt.max_iter, opt.tol, opt.inner_tol = int(restart), int(max_iter), float(tol), float(inner_tol)
        self.s = ctypes.c_void_p()
        rc = self.lib.vie_server_create(ctypes.byref(self.s), int(device), ctypes.byref(opt), int(n_slots),
                                        int(hbm_budget_bytes))
        if rc != 0:
            raise VIEError(rc, "vie_server_create failed")
        self._n_dom = {}

    def submit(self, cell, lam, theta=0.0, phi=0.0, eps=()):
        """Queue one solve; returns (ticket, footprint bytes).  Raises VIEError
        (VIE_ENOMEM) when the request can never fit in the HBM budget."""
        v = np.ascontiguousarray(cell.verts, dtype=np.float64)
        t = np.ascontiguousarray(cell.tets, dtype=np.int32)
        d = np.ascontiguousarray(cell.tet_domain, dtype=np.int32)
        m = Mesh(verts=v.ctypes.data, n_verts=len(v), tets=t.ctypes.data, n_tets=len(t), tet_domain=d.ctypes.data,
                 n_domains=int(cell.n_domains), active_domain=int(cell.active_domain),
                 period_a=float(cell.period_a), period_b=float(cell.period_b))
        r = Request()
        r.lambda_nm, r.theta, r.phi = float(lam), float(theta), float(phi)
        for k, e in enumerate(np.asarray(eps, dtype=np.complex128)):
            r.eps[2 * k], r.eps[2 * k + 1] = e.real, e.imag
        ticket = ctypes.c_uint64(0)
        fp = ctypes.c_int64(0)
        rc = self.lib.vie_server_submit(self.s, ctypes.byref(m), ctypes.byref(r), ctypes.byref(ticket),
                                        ctypes.byref(fp))
        if rc != 0:
            raise VIEError(rc, "vie_server_submit failed (footprint %d bytes)" % fp.value)
        self._n_dom[ticket.value] = int(cell.n_domains)
        return int(ticket.value), int(fp.value)

    def poll(self, ticket, wait_ms=-1):
        """The result dict of a finished request, or None if it is still pending."""
        res = Result()
        rc = self.lib.vie_server_poll(self.s, ctypes.c_uint64(ticket), ctypes.byref(res), int(wait_ms))
        if rc == VIE_PENDING:
            return None
        if rc != 0:
            raise VIEError(rc, "vie_server_poll failed")
        nd = self._n_dom.pop(ticket)
        return dict(status=res.status, n=res.n_unknowns, iterations=list(res.iterations),
                    rel_residual=np.array(res.rel_residual[:]),
                    A=np.array([[res.absorbed[p][k] for k in range(nd)] for p in range(2)]),
                    R=np.array(res.reflectance[:]), T=np.array(res.transmittance[:]),
                    t_fill_ms=res.t_fill_ms, t_factor_ms=res.t_factor_ms, t_solve_ms=res.t_solve_ms,
                    t_post_ms=res.t_post_ms, t_queue_ms=res.t_queue_ms, t_latency_ms=res.t_latency_ms,
                    n_launches=res.n_launches)

    def cancel(self, ticket):
        """Cancel a queued or running request (vie_server_cancel); it then polls
        with status VIE_CANCELLED unless it had already finished."""
        rc = self.lib.vie_server_cancel(self.s, ctypes.c_uint64(ticket))
        if rc != 0:
            raise VIEError(rc, "vie_server_cancel failed")

    def stats(self):
        st = ServerStats()
        self.lib.vie_server_get_stats(self.s, ctypes.byref(st))
        return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}

    def close(self):
        if self.s:
            self.lib.vie_server_destroy(self.s)
            self.s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
