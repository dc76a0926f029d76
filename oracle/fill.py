"""Galerkin impedance matrix and right-hand side of the SWG VIE, Eq. (1)-(2) (oracle).

Reading of Eq. (1)-(2) (the printed equations are garbled; see Sec. 2.1): the
unknown is the flux density D = sum_n D_n f_n, the total field is
E = D/(eps0 eps_r), the polarisation current is J = j w kappa D with
kappa = (eps_r - 1)/eps_r, and the charge is rho = -div(kappa D), including
surface charge where kappa jumps (and on the body's outer boundary, where the
outside is vacuum, kappa = 0).  Testing E^i = E + j w A + grad Phi with f_m and
multiplying by eps0 (unknowns d_n = D_n/eps0, lengths in nm, k0 = 2 pi/lambda):

  Z_mn = int f_m . f_n / eps_r                                  (local term)
       - k0^2 int int f_m(r) . kappa(r') f_n(r') g_p(r - r')      (vector potential)
       + int int div f_m(r) q_n(r') g_p(r - r')                   (scalar potential)
  b_m  = int f_m . E^i

where q_n = div'(kappa f_n) in the distributional sense: kappa(T) (+-a_n/V) in
each tetrahedron plus (kappa- - kappa+) delta on face n, and div f_m carries
-delta on face m for a half function.  The surface-charge terms therefore enter
with the sign fixed by charge conservation.

The time convention is exp(j w t): a lossy material has Im eps_r < 0, so the
physics-sign permittivities of the inputs are conjugated here.

Discrete problem (shared as a definition with the CUDA path): element pairs
whose centroid distance, for some lattice image (m, n) in {-1,0,1}^2, is below
NEAR_FACTOR x (sum of the element radii) x (1 + NEAR_MARGIN) are *near* in that
image.  Far pairs use the degree-2 product rules.  Near pairs split g_p into
the static part exp(j k_par.R)/(4 pi R) of every near image plus the remainder,
which is integrated with the degree-2 product rules.  The static part of an
image in which the two elements *touch* (share a vertex) is integrated in
closed form over one element at the points of the degree-5 rule of the other,
averaged over the two orders (outer rule on the test element, and outer rule
on the source element); the static part of a near image in which they do not
touch uses the degree-5 x degree-5 product rule.  Both choices are symmetric,
so the discrete operator keeps the reciprocity Z(k_par) = Z(-k_par)^T of the
continuous one for a single material.
"""
import numpy as np

from . import quadrature as qr
from .greens import PeriodicGreen
from .potentials import tet_integrals, tri_integrals
from .topology import KIND_HALF

NEAR_FACTOR = 1.5
# relative margin of the near test: exact ties (common on structured meshes)
# must classify the same way whatever the rounding of the distance
NEAR_MARGIN = 1e-9
# Sign of the surface-charge terms.  Charge conservation fixes it to +1; the
# tests set it to -1 (the sign printed for the kappa-gradient terms of Eq. (2))
# to show that reading fails.
SURFACE_CHARGE_SIGN = 1.0
NEAR_IMAGES = [(m, n) for m in (-1, 0, 1) for n in (-1, 0, 1)]


def surface_charge(kappa_plus, kappa_minus, half):
    """Surface part of q_n = div'(kappa f_n) on face n, per unit normal flux:
    kappa(T-) - kappa(T+), where kappa(T-) = 0 for a half function (the outside
    of the body is vacuum).  Charge conservation fixes the sign; the paper's
    Eq. (2) prints the kappa-gradient terms with the opposite one."""
    return SURFACE_CHARGE_SIGN * (np.where(half, 0.0, kappa_minus) - kappa_plus)


class Problem:
    """One (lambda, theta, phi) incidence on a meshed cell, with per-domain eps (physics sign)."""

    def __init__(self, topo, lam_nm, theta, phi, eps_phys):
        self.topo = topo
        self.lam = float(lam_nm)
        self.k0 = 2.0 * np.pi / self.lam
        self.theta, self.phi = float(theta), float(phi)
        self.kpar = self.k0 * np.sin(theta) * np.array([np.cos(phi), np.sin(phi), 0.0])
        self.eps_phys = np.asarray(eps_phys, dtype=np.complex128)
        self.eps = np.conj(self.eps_phys)              # exp(j w t) convention
        self.kappa = (self.eps - 1.0) / self.eps
        self.green = PeriodicGreen(self.k0, self.kpar[0], self.kpar[1], topo["a"], topo["b"])

    def pol_vectors(self):
        """TE and TM unit polarisations of the incident plane wave."""
        th, ph = self.theta, self.phi
        te = np.array([-np.sin(ph), np.cos(ph), 0.0])
        tm = np.array([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), np.sin(th)])
        return te, tm

    def k_inc(self):
        return np.array([self.kpar[0], self.kpar[1], -self.k0 * np.cos(self.theta)])


# ----------------------------------------------------------------------------
def _elements(topo):
    """Geometry of the test/source elements: tetrahedra and charge-carrying faces."""
    P = topo["tet_verts"]
    cent_t = P.mean(axis=1)
    rad_t = np.max(np.linalg.norm(P - cent_t[:, None], axis=-1), axis=1)
    cf = topo["charge_faces"]
    F = topo["face_verts"][topo["tp"][cf], topo["ip"][cf]]   # [nf,3,3] at the T+ side
    cent_f = F.mean(axis=1)
    rad_f = np.max(np.linalg.norm(F - cent_f[:, None], axis=-1), axis=1) if len(cf) else np.zeros(0)
    area_f = topo["area"][topo["tp"][cf], topo["ip"][cf]]
    return P, cent_t, rad_t, F, cent_f, rad_f, area_f


def _near_images(cx, rx, cy, ry, a, b):
    """Boolean [nx, ny, 9]: image (m,n) brings the pair within the near distance."""
    out = np.zeros((len(cx), len(cy), len(NEAR_IMAGES)), dtype=bool)
    for k, (m, n) in enumerate(NEAR_IMAGES):
        R = np.array([m * a, n * b, 0.0])
        d = np.linalg.norm(cx[:, None, :] - cy[None, :, :] + R, axis=-1)
        out[:, :, k] = d < NEAR_FACTOR * (rx[:, None] + ry[None, :]) * (1.0 + NEAR_MARGIN)
    return out


def _touch(vx, vy, R, a, b):
    """Boolean [p]: element x shares a vertex with the image y - R of element y."""
    tol = 1e-9 * max(a, b)
    d = np.linalg.norm(vx[:, :, None, :] - (vy[:, None, :, :] - R), axis=-1)
    return (d < tol).any(axis=(1, 2))


def _pair_moments(green, X, wX, cX, Y, wY, cY, sub=None, vector=True):
    """Product-rule moments of g_p between point sets X[nx,Qx,3] and Y[ny,Qy,3].

    Returns S = sum w w' g and, if vector, A = sum w w' (x-cX) g,
    B = sum w w' (y-cY) g, C = sum w w' (x-cX).(y-cY) g.
    `sub` ([nx, ny, n_img] over the Green's image table) removes static parts.
    """
    d = X[:, None, :, None, :] - Y[None, :, None, :, :]          # [nx,ny,Qx,Qy,3]
    if sub is not None:
        sub = sub[:, :, None, None, :]
    G = green(d, subtract=sub)
    W = wX[:, None, :, None] * wY[None, :, None, :]
    GW = G * W
    S = GW.sum(axis=(2, 3))
    if not vector:
        return S
    rx = X - cX[:, None, :]
    ry = Y - cY[:, None, :]
    A = np.einsum("ijpq,ipd->ijd", GW, rx)
    B = np.einsum("ijpq,jqd->ijd", GW, ry)
    C = np.einsum("ijpq,ipd,jqd->ij", GW, rx, ry)
    return S, A, B, C


def _sub_mask(green, near):
    """Map near flags over NEAR_IMAGES to the Green's image table."""
    idx = [green.image_index(m, n) for (m, n) in NEAR_IMAGES]
    mask = np.zeros(near.shape[:-1] + (len(green.images),), dtype=bool)
    mask[..., idx] = near
    return mask


def tet_tet_moments(prob, chunk=48):
    """S[nt,nt], A,B[nt,nt,3], C[nt,nt] with the near/far definition of the module."""
    topo, green = prob.topo, prob.green
    P, cent, rad, *_ = _elements(topo)
    vol = topo["vol"]
    nt = len(P)
    b2, w2 = qr.tet_deg2()
    b5, w5 = qr.tet_deg5()
    X2 = qr.map_points(b2, P)
    W2 = vol[:, None] * w2[None, :]
    S = np.zeros((nt, nt), np.complex128)
    A = np.zeros((nt, nt, 3), np.complex128)
    B = np.zeros((nt, nt, 3), np.complex128)
    C = np.zeros((nt, nt), np.complex128)
    near = _near_images(cent, rad, cent, rad, topo["a"], topo["b"])
    # all pairs by the degree-2 product rule; near images with their static part
    # removed (the near pass below recomputes those pairs and adds it back), so
    # that no term is evaluated at coincident points
    for i0 in range(0, nt, chunk):
        sl = slice(i0, min(nt, i0 + chunk))
        s, a_, b_, c_ = _pair_moments(green, X2[sl], W2[sl], cent[sl], X2, W2, cent, sub=_sub_mask(green, near[sl]))
        S[sl], A[sl], B[sl], C[sl] = s, a_, b_, c_
    # near pairs: closed-form static part + remainder
    ti, tj = np.nonzero(near.any(axis=-1))
    X5 = qr.map_points(b5, P)
    W5 = vol[:, None] * w5[None, :]
    for k0 in range(0, len(ti), 16384):
        I, J = ti[k0:k0 + 16384], tj[k0:k0 + 16384]
        nm = near[I, J]                                            # [p,9]
        sub = _sub_mask(green, nm)
        d = X2[I][:, :, None, :] - X2[J][:, None, :, :]
        G = green(d, subtract=sub[:, None, None, :])
        GW = G * W2[I][:, :, None] * W2[J][:, None, :]
        rx = X2[I] - cent[I][:, None]
        ry = X2[J] - cent[J][:, None]
        s = GW.sum(axis=(1, 2))
        a_ = np.einsum("ipq,ipd->id", GW, rx)
        b_ = np.einsum("ipq,iqd->id", GW, ry)
        c_ = np.einsum("ipq,ipd,iqd->i", GW, rx, ry)
        for k, (m, n) in enumerate(NEAR_IMAGES):
            sel = nm[:, k]
            if not sel.any():
                continue
            R = np.array([m * topo["a"], n * topo["b"], 0.0])
            touch = _touch(P[I[sel]], P[J[sel]], R, topo["a"], topo["b"])
            # non-touching near image: degree-5 x degree-5 product rule of the static part
            nt_ = np.nonzero(sel)[0][~touch]
            if len(nt_):
                ph1 = np.exp(1j * (prob.kpar @ R)) / (4 * np.pi)
                xr, yr = X5[I[nt_]], X5[J[nt_]]                       # [p,14,3]
                Rv = np.linalg.norm(xr[:, :, None, :] - yr[:, None, :, :] + R, axis=-1)
                Wp = W5[I[nt_]][:, :, None] * W5[J[nt_]][:, None, :] / Rv
                rx5 = xr - cent[I[nt_]][:, None]
                ry5 = yr - cent[J[nt_]][:, None]
                s[nt_] += ph1 * Wp.sum(axis=(1, 2))
                a_[nt_] += ph1 * np.einsum("ipq,ipd->id", Wp, rx5)
                b_[nt_] += ph1 * np.einsum("ipq,iqd->id", Wp, ry5)
                c_[nt_] += ph1 * np.einsum("ipq,ipd,iqd->i", Wp, rx5, ry5)
            sel = np.nonzero(sel)[0][touch]
            if not len(sel):
                continue
            ph = 0.5 * np.exp(1j * (prob.kpar @ R)) / (4 * np.pi)    # half of each order
            ct, cs = cent[I[sel]], cent[J[sel]]
            # (i) outer over the test tet, closed form over the image source tet T' - R
            r = X5[I[sel]]                                          # [p,14,3]
            w = W5[I[sel]]
            inv, vec = tet_integrals(r, (P[J[sel]] - R)[:, None, :, :])
            f_src = vec + (r - (cs - R)[:, None, :]) * inv[..., None]   # int (r'-c')/R dV'
            rxq = r - ct[:, None, :]
            s[sel] += ph * np.einsum("iq,iq->i", w, inv)
            a_[sel] += ph * np.einsum("iq,iq,iqd->id", w, inv, rxq)
            b_[sel] += ph * np.einsum("iq,iqd->id", w, f_src)
            c_[sel] += ph * np.einsum("iq,iqd,iqd->i", w, rxq, f_src)
            # (ii) outer over the source tet, closed form over the shifted test tet T + R
            r = X5[J[sel]]
            w = W5[J[sel]]
            inv, vec = tet_integrals(r, (P[I[sel]] + R)[:, None, :, :])
            f_tst = vec + (r - (ct + R)[:, None, :]) * inv[..., None]   # int (r-c)/R dV
            ryq = r - cs[:, None, :]
            s[sel] += ph * np.einsum("iq,iq->i", w, inv)
            a_[sel] += ph * np.einsum("iq,iqd->id", w, f_tst)
            b_[sel] += ph * np.einsum("iq,iq,iqd->id", w, inv, ryq)
            c_[sel] += ph * np.einsum("iq,iqd,iqd->i", w, ryq, f_tst)
        S[I, J], A[I, J], B[I, J], C[I, J] = s, a_, b_, c_
    return S, A, B, C


def _scalar_moments(prob, X_el, X_cent, X_rad, X_kind, Y_el, Y_cent, Y_rad, Y_kind, chunk=64):
    """I[x, y] = int_X int_Y g_p for tetrahedra ('tet') or triangles ('tri')."""
    topo, green = prob.topo, prob.green
    rules2 = {"tet": qr.tet_deg2(), "tri": qr.tri_deg2()}
    rules5 = {"tet": qr.tet_deg5(), "tri": qr.tri_deg5()}

    def measure(el, kind):
        if kind == "tet":
            return np.einsum("ij,ij->i", np.cross(el[:, 1] - el[:, 0], el[:, 2] - el[:, 0]), el[:, 3] - el[:, 0]) / 6.0
        return 0.5 * np.linalg.norm(np.cross(el[:, 1] - el[:, 0], el[:, 2] - el[:, 0]), axis=-1)

    mX, mY = measure(X_el, X_kind), measure(Y_el, Y_kind)
    bX, wX = rules2[X_kind]
    bY, wY = rules2[Y_kind]
    X2, WX = qr.map_points(bX, X_el), mX[:, None] * wX
    Y2, WY = qr.map_points(bY, Y_el), mY[:, None] * wY
    nx, ny = len(X_el), len(Y_el)
    out = np.zeros((nx, ny), np.complex128)
    if nx == 0 or ny == 0:
        return out
    near = _near_images(X_cent, X_rad, Y_cent, Y_rad, topo["a"], topo["b"])
    for i0 in range(0, nx, chunk):   # static part of near images removed, as in tet_tet_moments
        sl = slice(i0, min(nx, i0 + chunk))
        out[sl] = _pair_moments(green, X2[sl], WX[sl], X_cent[sl], Y2, WY, Y_cent, sub=_sub_mask(green, near[sl]),
                                vector=False)
    I, J = np.nonzero(near.any(axis=-1))
    b5, w5 = rules5[X_kind]
    X5, W5 = qr.map_points(b5, X_el), mX[:, None] * w5
    c5, v5 = rules5[Y_kind]
    Y5, WY5 = qr.map_points(c5, Y_el), mY[:, None] * v5
    for k0 in range(0, len(I), 16384):
        Ii, Jj = I[k0:k0 + 16384], J[k0:k0 + 16384]
        nm = near[Ii, Jj]
        sub = _sub_mask(green, nm)
        d = X2[Ii][:, :, None, :] - Y2[Jj][:, None, :, :]
        G = green(d, subtract=sub[:, None, None, :])
        s = (G * WX[Ii][:, :, None] * WY[Jj][:, None, :]).sum(axis=(1, 2))
        for k, (m, n) in enumerate(NEAR_IMAGES):
            sel = nm[:, k]
            if not sel.any():
                continue
            R = np.array([m * topo["a"], n * topo["b"], 0.0])
            touch = _touch(X_el[Ii[sel]], Y_el[Jj[sel]], R, topo["a"], topo["b"])
            nt_ = np.nonzero(sel)[0][~touch]
            if len(nt_):   # non-touching: degree-5 x degree-5 product rule of the static part
                ph1 = np.exp(1j * (prob.kpar @ R)) / (4 * np.pi)
                Rv = np.linalg.norm(X5[Ii[nt_]][:, :, None, :] - Y5[Jj[nt_]][:, None, :, :] + R, axis=-1)
                s[nt_] += ph1 * (W5[Ii[nt_]][:, :, None] * WY5[Jj[nt_]][:, None, :] / Rv).sum(axis=(1, 2))
            sel = np.nonzero(sel)[0][touch]
            if not len(sel):
                continue
            ph = 0.5 * np.exp(1j * (prob.kpar @ R)) / (4 * np.pi)
            # (i) outer over X, closed form over the image of Y; (ii) the reverse
            for outer5, Wo, el, kind, shift in ((X5[Ii[sel]], W5[Ii[sel]], Y_el[Jj[sel]] - R, Y_kind, None),
                                               (Y5[Jj[sel]], WY5[Jj[sel]], X_el[Ii[sel]] + R, X_kind, None)):
                if kind == "tet":
                    inv, _ = tet_integrals(outer5, el[:, None])
                else:
                    inv, _ = tri_integrals(outer5, el[:, None])
                s[sel] += ph * np.einsum("iq,iq->i", Wo, inv)
        out[Ii, Jj] = s
    return out


# ----------------------------------------------------------------------------
def assemble(prob, with_rhs=True):
    """Return (Z [N,N], b [N,2] for TE/TM) of Eq. (2) for `prob` (FP64)."""
    topo = prob.topo
    N = topo["n"]
    P, cent, rad, F, cent_f, rad_f, area_f = _elements(topo)
    vol, area = topo["vol"], topo["area"]
    basis, sign, shift = topo["basis"], topo["sign"], topo["shift"]
    dom = topo["domain"]
    eps_t = prob.eps[dom]
    kap_t = prob.kappa[dom]
    wS = np.exp(-1j * (shift @ prob.kpar))            # source weights [nt,4]
    wT = np.exp(+1j * (shift @ prob.kpar))            # test weights
    coef = sign * area / (3.0 * vol[:, None])         # f = coef (r - v_i)
    div = sign * area / vol[:, None]
    wv = P - cent[:, None, :]                         # free vertices rel. centroid [nt,4,3]

    Z = np.zeros((N, N), np.complex128)

    def scatter(rows, cols, vals):
        np.add.at(Z, (rows.ravel(), cols.ravel()), vals.ravel())

    # --- local (Gram) term -------------------------------------------------
    sq = np.sum(wv * wv, axis=(1, 2))                  # sum_k |d_k|^2
    G = vol[:, None, None] * (sq[:, None, None] / 20.0 + np.einsum("tid,tjd->tij", wv, wv))
    val = (wT[:, :, None] * wS[:, None, :] * coef[:, :, None] * coef[:, None, :] * G) / eps_t[:, None, None]
    scatter(np.broadcast_to(basis[:, :, None], val.shape), np.broadcast_to(basis[:, None, :], val.shape), val)

    # --- tet-tet vector and scalar potential ----------------------------------
    S, A, B, C = tet_tet_moments(prob)
    # M_ij = C - w'_j.A - w_i.B + (w_i.w'_j) S for each pair
    M = (C[:, :, None, None]
         - np.einsum("tsd,sjd->tsj", A, wv)[:, :, None, :]
         - np.einsum("tsd,tid->tsi", B, wv)[:, :, :, None]
         + np.einsum("tid,sjd->tsij", wv, wv) * S[:, :, None, None])
    vec = -prob.k0 ** 2 * kap_t[None, :, None, None] * coef[:, None, :, None] * coef[None, :, None, :] * M
    sca = div[:, None, :, None] * (kap_t[:, None] * div)[None, :, None, :] * S[:, :, None, None]
    val = wT[:, None, :, None] * wS[None, :, None, :] * (vec + sca)
    rows = np.broadcast_to(basis[:, None, :, None], val.shape)
    cols = np.broadcast_to(basis[None, :, None, :], val.shape)
    scatter(rows, cols, val)

    # --- surface charge / surface test terms ---------------------------------
    cf = topo["charge_faces"]
    if len(cf):
        kind = topo["kind"][cf]
        kp = prob.kappa[dom[topo["tp"][cf]]]
        km = prob.kappa[dom[np.maximum(topo["tm"][cf], 0)]]
        qs = surface_charge(kp, km, kind == KIND_HALF)    # surface charge of basis n on its face
        ts = np.where(kind == KIND_HALF, -1.0, 0.0)       # surface part of div f_m
        I_tf = _scalar_moments(prob, P, cent, rad, "tet", F, cent_f, rad_f, "tri")
        val = (wT * div)[:, :, None] * (qs[None, :] * I_tf)[:, None, :]
        scatter(np.broadcast_to(basis[:, :, None], val.shape), np.broadcast_to(cf[None, None, :], val.shape), val)
        hf = ts != 0
        if hf.any():
            I_ft = _scalar_moments(prob, F[hf], cent_f[hf], rad_f[hf], "tri", P, cent, rad, "tet")
            val = ts[hf][:, None, None] * I_ft[:, :, None] * (wS * kap_t[:, None] * div)[None, :, :]
            scatter(np.broadcast_to(cf[hf][:, None, None], val.shape), np.broadcast_to(basis[None], val.shape), val)
            I_ff = _scalar_moments(prob, F[hf], cent_f[hf], rad_f[hf], "tri", F, cent_f, rad_f, "tri")
            val = ts[hf][:, None] * qs[None, :] * I_ff
            scatter(np.broadcast_to(cf[hf][:, None], val.shape), np.broadcast_to(cf[None, :], val.shape), val)

    # every singular term was integrated in closed form: a non-finite entry is a bug
    assert np.all(np.isfinite(Z)), "non-finite impedance matrix entry"
    if not with_rhs:
        return Z, None
    return Z, rhs(prob)


def rhs(prob):
    """b_m = int f_m . p E^i with E^i = p exp(-j k_inc . r), |E0| = 1, for TE and TM (Eq. (2))."""
    topo = prob.topo
    P = topo["tet_verts"]
    vol, area = topo["vol"], topo["area"]
    cent = P.mean(axis=1)
    b5, w5 = qr.tet_deg5()
    X = qr.map_points(b5, P)                                   # [nt,14,3]
    W = vol[:, None] * w5
    wT = np.exp(+1j * (topo["shift"] @ prob.kpar))
    coef = topo["sign"] * area / (3.0 * vol[:, None])
    kin = prob.k_inc()
    ph = np.exp(-1j * (X @ kin)) * W                           # [nt,14]
    out = np.zeros((topo["n"], 2), np.complex128)
    for p_i, pv in enumerate(prob.pol_vectors()):
        # int (r - v_i).p e^{-jk.r} = sum_q w ((x_q - c) - (v_i - c)).p e^{..}
        xp = (X - cent[:, None]) @ pv                          # [nt,14]
        vp = (P - cent[:, None]) @ pv                          # [nt,4]
        integ = (ph * xp).sum(axis=1)[:, None] - vp * ph.sum(axis=1)[:, None]
        val = wT * coef * integ
        np.add.at(out[:, p_i], topo["basis"].ravel(), val.ravel())
    return out
