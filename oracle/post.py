"""Absorption (Eq. (7)), reflectance/transmittance and Eq. (8) for the oracle.

Eq. (7) gives A = w int Im(eps) |E|^2 dv over the active material.  Read with
the time-average factor and the incident power it is normalised by: the
fraction of the incident power absorbed in domain d of one cell is

    A_d = k0 int_d |Im eps_r| |E|^2 dV / (|E0|^2 a b cos(theta)),

from P_abs = (w eps0/2) int |Im eps_r||E|^2 and P_inc = |E0|^2 a b cos(theta)/(2 eta0),
with w eps0 eta0 = k0.  E = d/eps_r is linear in each tetrahedron, so the
integral of |E|^2 is exact with the tetrahedron's second moments.  The same
integrand per tetrahedron is the absorption profile (Fig. 5); its layer sums on
a slab are pinned against the slab's closed-form standing wave.

R and T (not in the paper; they close the energy balance R + T + sum A_d = 1)
come from the Floquet expansion of the scattered field of J = j w kappa D: for
a propagating order with wavevector k = (k_t, +-k_z), the plane-wave amplitude
above (+) / below (-) the cell is

    E_pq = -j k0^2/(2 a b k_z) (I - k^ k^) . int kappa d exp(j k . r) dV,

and R = sum |E+_pq|^2 k_z,pq / k_z,00, T = sum |E-_pq + delta_pq,00 p|^2 k_z,pq / k_z,00.
"""
import numpy as np

from . import quadrature as qr


def _tet_fields(prob, x):
    """Per-tet coefficients beta[t, i] of d(r) = sum_i beta_i (r - v_i)."""
    topo = prob.topo
    wS = np.exp(-1j * (topo["shift"] @ prob.kpar))
    coef = topo["sign"] * topo["area"] / (3.0 * topo["vol"][:, None])
    return x[topo["basis"]] * wS * coef


def absorption(prob, x):
    """A_d per domain for one coefficient vector x [N]."""
    topo = prob.topo
    P = topo["tet_verts"]
    vol = topo["vol"]
    cent = P.mean(axis=1)
    wv = P - cent[:, None, :]
    sq = np.sum(wv * wv, axis=(1, 2))
    G = vol[:, None, None] * (sq[:, None, None] / 20.0 + np.einsum("tid,tjd->tij", wv, wv))
    eps_t = prob.eps[topo["domain"]]
    beta = _tet_fields(prob, x) / eps_t[:, None]
    e2 = np.real(np.einsum("ti,tij,tj->t", beta, G, np.conj(beta)))
    dens = prob.k0 * np.abs(np.imag(eps_t)) * e2 / (topo["a"] * topo["b"] * np.cos(prob.theta))
    return np.bincount(topo["domain"], weights=dens, minlength=topo["n_domains"]), dens


def reflect_transmit(prob, x, pol_index):
    topo = prob.topo
    P = topo["tet_verts"]
    vol = topo["vol"]
    b5, w5 = qr.tet_deg5()
    X = qr.map_points(b5, P)
    W = vol[:, None] * w5
    beta = _tet_fields(prob, x) * prob.kappa[topo["domain"]][:, None]
    # d(x_q) kappa = sum_i beta_i (x_q - v_i)
    dq = np.einsum("ti,tqd->tqd", beta, X) - np.einsum("ti,tid->td", beta, P)[:, None, :]
    a, b, k0 = topo["a"], topo["b"], prob.k0
    kz00 = k0 * np.cos(prob.theta)
    pv = prob.pol_vectors()[pol_index]
    R = T = 0.0
    pm = int(np.ceil(2 * k0 * a / (2 * np.pi))) + 1
    qm = int(np.ceil(2 * k0 * b / (2 * np.pi))) + 1
    for p in range(-pm, pm + 1):
        for q in range(-qm, qm + 1):
            kt = prob.kpar[:2] + 2 * np.pi * np.array([p / a, q / b])
            kz2 = k0 * k0 - kt @ kt
            if kz2 <= 0:
                continue
            kz = np.sqrt(kz2)
            for sgn in (+1, -1):
                kv = np.array([kt[0], kt[1], sgn * kz])
                ph = np.exp(1j * (X @ kv)) * W
                Jt = np.einsum("tq,tqd->d", ph, dq)
                kh = kv / k0
                Et = -1j * k0 * k0 / (2 * a * b * kz) * (Jt - kh * (kh @ Jt))
                if sgn < 0 and p == 0 and q == 0:
                    Et = Et + pv
                pw = np.real(np.vdot(Et, Et)) * kz / kz00
                if sgn > 0:
                    R += pw
                else:
                    T += pw
    return R, T


def relative_error(x_pre, x_nopre):
    """Eq. (8): ||J_pre - J_nopre||_2 / ||J_nopre||_2."""
    return np.linalg.norm(x_pre - x_nopre) / np.linalg.norm(x_nopre)
