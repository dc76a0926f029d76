"""Textbook closed forms used to pin the oracle (test helpers, not part of the method).

* Transfer-matrix (characteristic-matrix) reflectance / transmittance of a
  planar layer stack in vacuum, TE and TM (Born & Wolf).
* Mie absorption cross-section of a homogeneous sphere (Bohren & Huffman).
* The standing-wave field inside a homogeneous slab at normal incidence and
  its absorption per depth interval (the same boundary-value problem: E and
  dE/dz continuous at both faces).
Permittivities use the physics sign (Im > 0 lossy), time convention exp(-i w t).
"""
import numpy as np
from scipy.special import spherical_jn, spherical_yn


def tmm_rt(eps_layers, d_layers, lam, theta, pol):
    """R, T, A of layers (listed from the illuminated side) between vacuum half-spaces."""
    k0 = 2 * np.pi / lam
    kx = k0 * np.sin(theta)

    def kz_of(eps):
        kz = np.sqrt(complex(eps) * k0 * k0 - kx * kx)
        return kz if kz.imag >= 0 else -kz

    def q_of(eps):
        kz = kz_of(eps)
        return kz if pol == "TE" else kz / complex(eps)

    M = np.eye(2, dtype=np.complex128)
    for eps, d in zip(eps_layers, d_layers):
        q = q_of(eps)
        dl = kz_of(eps) * d
        Mj = np.array([[np.cos(dl), -1j * np.sin(dl) / q], [-1j * q * np.sin(dl), np.cos(dl)]])
        M = M @ Mj
    q0 = qs = q_of(1.0)
    den = q0 * M[0, 0] + q0 * qs * M[0, 1] + M[1, 0] + qs * M[1, 1]
    r = (q0 * M[0, 0] + q0 * qs * M[0, 1] - M[1, 0] - qs * M[1, 1]) / den
    t = 2 * q0 / den
    R = abs(r) ** 2
    T = abs(t) ** 2 * (qs.real / q0.real)
    return R, T, 1.0 - R - T


def slab_layer_absorption(eps, d, lam, z_edges, n=4000):
    """Absorbed fraction of the incident power in each depth interval
    [z_edges[i], z_edges[i+1]] of a slab 0 < z < d (permittivity eps, physics
    sign) in vacuum, lit at normal incidence from z > d with unit amplitude:
    k0 Im(eps) int |E(z)|^2 dz, E = P exp(-i k1 z) + Q exp(i k1 z) inside
    (k1 = k0 sqrt(eps)).  r, P, Q, t from continuity of E and dE/dz at z = 0
    and z = d.  Returns (per-interval fractions, R, T)."""
    k0 = 2 * np.pi / lam
    n1 = np.sqrt(complex(eps))
    k1 = k0 * (n1 if n1.imag >= 0 else -n1)
    e0, e1 = np.exp(1j * k0 * d), np.exp(1j * k1 * d)
    M = np.array([[0, 1, 1, -1],
                  [0, k1, -k1, -k0],
                  [-e0, 1 / e1, e1, 0],
                  [k0 * e0, k1 / e1, -k1 * e1, 0]], dtype=np.complex128)
    rhs = np.array([0, 0, 1 / e0, k0 / e0], dtype=np.complex128)
    r, P, Q, t = np.linalg.solve(M, rhs)
    out = []
    for z0, z1 in zip(z_edges[:-1], z_edges[1:]):
        z = np.linspace(z0, z1, n + 1)
        f = np.abs(P * np.exp(-1j * k1 * z) + Q * np.exp(1j * k1 * z)) ** 2
        out.append(k0 * complex(eps).imag * np.trapezoid(f, z))
    return np.array(out), abs(r) ** 2, abs(t) ** 2


def mie_cabs(radius, eps, lam, nmax=None):
    """Absorption cross-section of a sphere in vacuum (Bohren & Huffman Mie series)."""
    k = 2 * np.pi / lam
    m = np.sqrt(complex(eps))
    x = k * radius
    mx = m * x
    nmax = nmax or int(x + 4 * x ** (1 / 3) + 4)
    n = np.arange(1, nmax + 1)

    def psi(z, nn):   # Riccati-Bessel z j_n(z) for complex z via upward recurrence on j_n
        return z * _sph_jn_complex(nn, z)

    def dpsi(z, nn):
        return z * _sph_jn_complex(nn - 1, z) - nn * _sph_jn_complex(nn, z)

    jx = spherical_jn(n, x)
    yx = spherical_yn(n, x)
    psix = x * jx
    dpsix = x * spherical_jn(n - 1, x) - n * jx
    xix = x * (jx + 1j * yx)
    dxix = x * (spherical_jn(n - 1, x) + 1j * spherical_yn(n - 1, x)) - n * (jx + 1j * yx)
    pm = psi(mx, n)
    dpm = dpsi(mx, n)
    an = (m * pm * dpsix - psix * dpm) / (m * pm * dxix - xix * dpm)
    bn = (pm * dpsix - m * psix * dpm) / (pm * dxix - m * xix * dpm)
    cext = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * np.real(an + bn))
    csca = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (abs(an) ** 2 + abs(bn) ** 2))
    return cext - csca


def _sph_jn_complex(n, z):
    """Spherical Bessel j_n(z), complex z, by series (adequate for |z| < ~5)."""
    n = np.atleast_1d(n)
    out = np.zeros(n.shape, dtype=np.complex128)
    from math import factorial
    for idx, nn in enumerate(n):
        nn = int(nn)
        if nn < 0:   # j_{-1}(z) = cos(z)/z
            out[idx] = np.cos(z) / z
            continue
        s = 0j
        term_scale = z ** nn / np.prod(np.arange(1, 2 * nn + 2, 2, dtype=np.float64))
        for kk in range(60):
            s += (-(z * z) / 2) ** kk / (factorial(kk) * np.prod(np.arange(2 * nn + 3, 2 * nn + 2 * kk + 2, 2, dtype=np.float64)))
        out[idx] = term_scale * s
    return out
