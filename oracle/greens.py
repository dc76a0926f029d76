"""2D periodic Green's function, Eq. (3)-(4) (oracle, test infrastructure).

Time convention exp(j w t), free-space kernel g(R) = exp(-j k R)/(4 pi R)
(Sec. 2.1).  The periodic kernel of Eq. (3), with the Bloch phase of the
incident direction, is

    g_p(d) = sum_{m,n} g(|d + R_mn|) exp(j k_par . R_mn),   R_mn = (m a, n b, 0),

so that g_p(d + R) = exp(-j k_par . R) g_p(d).  Sec. 2.2 evaluates it by Ewald's
method: a spatial series (images, complementary error functions) plus a
spectral series (Floquet modes, by Poisson summation).  With splitting
parameter E, b = k/(2E) and gamma_pq = sqrt(|k_t,pq|^2 - k^2) (Re >= 0,
+j sqrt(k^2 - |k_t|^2) for propagating modes), k_t,pq = k_par + 2 pi (p/a, q/b):

  spatial  = sum_mn exp(j k_par.R_mn) exp(b^2 - R^2 E^2)
             [erfcx(R E - j b) + erfcx(R E + j b)] / (8 pi R),  R = |d + R_mn|
  spectral = 1/(4ab) sum_pq exp(-j k_t.rho) / gamma
             [exp(gamma z) erfc(gamma/2E + zE) + exp(-gamma z) erfc(gamma/2E - zE)]

(erfcx(u) = exp(u^2) erfc(u) = w(j u), w the Faddeeva function.)  The oracle
evaluates w with scipy.special.wofz.  Two plain lattice sums pin it: the pure
Floquet series (1/2ab) sum exp(-j k_t.rho - gamma|z|)/gamma for z != 0, and a
smoothly windowed image sum.
"""
import numpy as np
from scipy.special import erfcx as erfcx_real
from scipy.special import wofz

X_CUT = 6.6   # exp(-X_CUT^2) ~ 1e-19: truncation of both Ewald series
PARALLEL_MIN = 40_000
_POOL = None


def _workers():
    import os
    return int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))


def _pool():
    """Process pool started with 'spawn' (safe next to a CUDA context)."""
    global _POOL
    if _POOL is None:
        import concurrent.futures
        import multiprocessing
        _POOL = concurrent.futures.ProcessPoolExecutor(
            max_workers=_workers(), mp_context=multiprocessing.get_context("spawn"))
    return _POOL


def _eval_chunk(args):
    green, d, sub = args
    return green._eval(d, sub)


def _parallel_eval(green, d, subtract):
    n = d.shape[0]
    k = min(n, 4 * _workers())
    bounds = np.linspace(0, n, k + 1).astype(int)
    jobs = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        if hi <= lo:
            continue
        sub = None
        if subtract is not None:
            sub = subtract[lo:hi] if subtract.shape[0] == n else subtract
        jobs.append((green, d[lo:hi], sub))
    return np.concatenate(list(_pool().map(_eval_chunk, jobs)), axis=0)


def erfcx(u):
    return wofz(1j * np.asarray(u, dtype=np.complex128))


class PeriodicGreen:
    """Ewald evaluation of g_p for one (k, k_par, a, b)."""

    def __init__(self, k0, kx, ky, a, b, E=None, H=3.0):
        self.k0, self.kx, self.ky, self.a, self.b = float(k0), float(kx), float(ky), float(a), float(b)
        # splitting parameter: sqrt(pi/(ab)), raised to k/(2H) at high frequency
        # (Kustepeli & Martin's rule) to bound the exp(b^2) growth
        self.E = float(E) if E is not None else max(np.sqrt(np.pi / (a * b)), k0 / (2.0 * H))
        E = self.E
        # spatial images: any image whose nearest possible distance
        # (|m|-1)a, (|n|-1)b for in-cell differences |dx|<a, |dy|<b) is inside the cut
        mmax = int(np.ceil(X_CUT / (E * a))) + 2
        nmax = int(np.ceil(X_CUT / (E * b))) + 2
        imgs = []
        for m in range(-mmax, mmax + 1):
            for n in range(-nmax, nmax + 1):
                dmin = np.hypot(max(abs(m) - 1, 0) * a, max(abs(n) - 1, 0) * b)
                if dmin * E <= X_CUT:
                    imgs.append((m, n))
        self.images = np.array(imgs, dtype=np.int64)
        # spectral modes: exp(-gamma^2 / 4E^2) below the cut
        pmax = int(np.ceil((2.0 * E * X_CUT + abs(kx)) * a / (2 * np.pi))) + 1
        qmax = int(np.ceil((2.0 * E * X_CUT + abs(ky)) * b / (2 * np.pi))) + 1
        modes = []
        for p in range(-pmax, pmax + 1):
            for q in range(-qmax, qmax + 1):
                ktx = kx + 2 * np.pi * p / a
                kty = ky + 2 * np.pi * q / b
                if np.hypot(ktx, kty) <= 2.0 * E * X_CUT + k0:
                    modes.append((p, q, ktx, kty))
        self.modes = np.array(modes, dtype=np.float64)
        kt2 = self.modes[:, 2] ** 2 + self.modes[:, 3] ** 2
        self.gamma = gamma_branch(kt2, k0)

    # ------------------------------------------------------------------
    def spatial_terms(self, d, m, n):
        """One image term exp(j k_par.R) exp(b^2-R^2E^2)[erfcx(RE-jb)+erfcx(RE+jb)]/(8 pi R)."""
        E, k = self.E, self.k0
        bb = k / (2 * E)
        Rx = d[..., 0] + m * self.a
        Ry = d[..., 1] + n * self.b
        R = np.sqrt(Rx * Rx + Ry * Ry + d[..., 2] ** 2)
        ph = np.exp(1j * (self.kx * m * self.a + self.ky * n * self.b))
        # real k: erfcx(RE - jb) = conj(erfcx(RE + jb)), so the bracket is 2 Re erfcx(RE + jb);
        # terms with R E beyond the cut are below exp(-X_CUT^2) and are skipped
        # R = 0 (coincident points) is singular: such a term must be replaced by
        # its regular part (subtract mask); NaN marks it if it is not
        val = np.zeros(R.shape, dtype=np.float64)
        live = (R * E <= X_CUT + 0.5) & (R > 0)
        if np.any(live):
            Rl = R[live]
            val[live] = np.exp(bb * bb - (Rl * E) ** 2) * np.real(erfcx(Rl * E + 1j * bb)) / (4 * np.pi * Rl)
        val[R == 0] = np.nan
        return ph * val, R, ph

    def spatial_regular(self, d, m, n):
        """Image term minus its static part exp(j k_par.R)/(4 pi R); finite at R -> 0."""
        E, k = self.E, self.k0
        bb = k / (2 * E)
        Rx = d[..., 0] + m * self.a
        Ry = d[..., 1] + n * self.b
        R = np.sqrt(Rx * Rx + Ry * Ry + d[..., 2] ** 2)
        ph = np.exp(1j * (self.kx * m * self.a + self.ky * n * self.b))
        out = np.empty(R.shape, dtype=np.complex128)
        small = R * E < 1e-7
        Rs = np.where(small, 1.0, R)
        full = np.exp(bb * bb - (Rs * E) ** 2) * np.real(erfcx(Rs * E + 1j * bb)) / (4 * np.pi * Rs)
        out[:] = full - 1.0 / (4 * np.pi * Rs)
        # limit R -> 0: (E/4pi) [2 b erfi(b) - (2/sqrt(pi)) exp(b^2)] for real b
        lim = (E / (4 * np.pi)) * (2 * bb * _erfi(bb) - 2.0 / np.sqrt(np.pi) * np.exp(bb * bb))
        out[small] = lim
        return ph * out

    def spectral(self, d):
        E = self.E
        rx, ry, z = d[..., 0], d[..., 1], np.abs(d[..., 2])
        acc = np.zeros(np.shape(rx), dtype=np.complex128)
        for (p, q, ktx, kty), g in zip(self.modes, self.gamma):
            if g.imag == 0.0:          # evanescent mode: real arguments
                gr = g.real
                pre = np.exp(-gr * gr / (4 * E * E) - (z * E) ** 2)
                t1 = pre * erfcx_real(gr / (2 * E) + z * E)
                u = gr / (2 * E) - z * E
                t2 = np.where(u >= 0, pre * erfcx_real(np.abs(u)), 2 * np.exp(-gr * z) - pre * erfcx_real(np.abs(u)))
            else:
                pre = np.exp(-g * g / (4 * E * E) - (z * E) ** 2)
                t1 = pre * erfcx(g / (2 * E) + z * E)
                u = g / (2 * E) - z * E
                t2 = np.where(np.real(u) >= 0, pre * erfcx(u), 2 * np.exp(-g * z) - pre * erfcx(-u))
            acc += np.exp(-1j * (ktx * rx + kty * ry)) * (t1 + t2) / g
        return acc / (4 * self.a * self.b)

    def __call__(self, d, subtract=None):
        """g_p(d) for in-cell difference vectors d[..., 3] (|dx| < a, |dy| < b).

        subtract: optional boolean mask [..., n_images] (broadcastable against
        d[..., 0]) over the image table; for flagged images the static part
        exp(j k_par.R)/(4 pi R) is removed.  Large inputs are split over a
        process pool along the first axis (same arithmetic per element).
        """
        d = np.asarray(d, dtype=np.float64)
        if d.ndim >= 2 and d.shape[0] >= 2 and d[..., 0].size >= PARALLEL_MIN and _workers() > 1:
            return _parallel_eval(self, d, subtract)
        return self._eval(d, subtract)

    def _eval(self, d, subtract=None):
        acc = self.spectral(d)
        for idx, (m, n) in enumerate(self.images):
            full, _, _ = self.spatial_terms(d, m, n)
            if subtract is not None:
                sub = np.broadcast_to(subtract[..., idx], full.shape)
                if np.any(sub):   # flagged entries: the regular part only
                    full[sub] = self.spatial_regular(d[sub], m, n)
            acc += full
        return acc

    def image_index(self, m, n):
        hit = np.nonzero((self.images[:, 0] == m) & (self.images[:, 1] == n))[0]
        return int(hit[0])


def gamma_branch(kt2, k0):
    """sqrt(|k_t|^2 - k^2) with Re >= 0 and +j sqrt(k^2-|k_t|^2) when propagating."""
    g2 = np.asarray(kt2, dtype=np.float64) - k0 * k0
    return np.where(g2 >= 0, np.sqrt(np.maximum(g2, 0.0)) + 0j, 1j * np.sqrt(np.maximum(-g2, 0.0)))


def _erfi(x):
    from scipy.special import erfi
    return erfi(x)


# ----------------------------------------------------------------------
# plain lattice sums used as pins
# ----------------------------------------------------------------------
def spectral_direct(d, k0, kx, ky, a, b, pq_max=60):
    """(1/2ab) sum_pq exp(-j k_t.rho - gamma |z|)/gamma: the Floquet series (z != 0)."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    acc = np.zeros(d.shape[0], dtype=np.complex128)
    for p in range(-pq_max, pq_max + 1):
        for q in range(-pq_max, pq_max + 1):
            ktx = kx + 2 * np.pi * p / a
            kty = ky + 2 * np.pi * q / b
            g = gamma_branch(ktx * ktx + kty * kty, k0)
            acc += np.exp(-1j * (ktx * d[:, 0] + kty * d[:, 1]) - g * np.abs(d[:, 2])) / g
    return acc / (2 * a * b)


def windowed_direct(d, k0, kx, ky, a, b, A, c=0.5):
    """Image sum of Eq. (3) with the smooth window chi(|R_mn|/A) (super-algebraic convergence)."""
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    M = int(np.ceil(A / a)) + 1
    Nn = int(np.ceil(A / b)) + 1
    m, n = np.meshgrid(np.arange(-M, M + 1), np.arange(-Nn, Nn + 1), indexing="ij")
    m, n = m.ravel(), n.ravel()
    Rl = np.hypot(m * a, n * b)
    t = Rl / A
    u = np.clip((t - c) / (1 - c), 0.0, 1.0)
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        chi = np.where(u <= 0, 1.0, np.where(u >= 1, 0.0, np.exp(2 * np.exp(-1 / np.maximum(u, 1e-300)) / (u - 1))))
    keep = chi > 0
    m, n, chi = m[keep], n[keep], chi[keep]
    out = np.zeros(d.shape[0], dtype=np.complex128)
    for i in range(d.shape[0]):
        x = d[i, 0] + m * a
        y = d[i, 1] + n * b
        R = np.sqrt(x * x + y * y + d[i, 2] ** 2)
        out[i] = np.sum(chi * np.exp(-1j * k0 * R) / (4 * np.pi * R) * np.exp(1j * (kx * m * a + ky * n * b)))
    return out
