"""Closed-form integrals of 1/R and R over triangles and tetrahedra (oracle).

Used to extract the 1/(4 pi R) singularity of the Green's function for touching
and nearby elements.  The formulas follow from the divergence theorem
(the approach of Wilton, Rao, Glisson et al. for polygonal and polyhedral
sources), derived here:

Triangle F in a plane with unit normal n, observer r, height h = n.(r - r_F),
for each edge i with unit tangent l_i, in-plane outward normal u_i = l_i x n,
signed distance t_i = u_i.(r_i - r) of the edge line from the projection of r,
edge-end coordinates s_i^{+-} along l_i and distances R_i^{+-}, R0_i^2 = t_i^2 + h^2:

  int_F 1/R = sum_i t_i ln[(R_i^+ + s_i^+)/(R_i^- + s_i^-)]
              - |h| sum_i [atan(t_i s_i^+ /(R0_i^2 + |h| R_i^+)) - atan(t_i s_i^- /(R0_i^2 + |h| R_i^-))]
  int_F R   = (1/3) [ h^2 int_F 1/R
                      + (1/2) sum_i t_i (s^+R^+ - s^-R^- + R0_i^2 ln[(R^+ + s^+)/(R^- + s^-)]) ]

(the second from div_2D(u R) = 3R - h^2/R on the plane).  For a tetrahedron T
with outward face normals n_f and signed distances d_f = n_f.(r_f - r):

  int_T 1/R dV'         = (1/2) sum_f d_f int_f 1/R dS'      (div((r'-r)/R) = 2/R)
  int_T (r' - r)/R dV'  = sum_f n_f int_f R dS'              (grad' R = (r'-r)/R)
"""
import numpy as np


def _log_ratio(Rp, sp, Rm, sm, R0sq):
    """ln[(R+ + s+)/(R- + s-)] without cancellation when s < 0 (R + s = R0^2/(R - s))."""
    def lg(R, s):
        return np.where(s >= 0, np.log(np.maximum(R + s, 1e-300)),
                        np.log(np.maximum(R0sq, 1e-300)) - np.log(np.maximum(R - s, 1e-300)))
    return lg(Rp, sp) - lg(Rm, sm)


def tri_integrals(r, tri):
    """Return (int_F 1/R dS', int_F R dS') for observers r[...,3], triangles tri[...,3,3]."""
    r = np.asarray(r, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.float64)
    v0, v1, v2 = tri[..., 0, :], tri[..., 1, :], tri[..., 2, :]
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
    h = np.sum(nrm * (r - v0), axis=-1)
    ah = np.abs(h)
    # orient edges counter-clockwise about nrm
    edges = ((v0, v1), (v1, v2), (v2, v0))
    inv = np.zeros(np.broadcast(h, h).shape)
    acc_log = np.zeros_like(inv)   # sum t_i * ln
    acc_atan = np.zeros_like(inv)
    acc_r = np.zeros_like(inv)     # sum t_i * (s+R+ - s-R- + R0^2 ln)
    scale = np.max(np.linalg.norm(tri - tri.mean(axis=-2, keepdims=True), axis=-1), axis=-1)
    for pa, pb in edges:
        L = pb - pa
        ell = np.linalg.norm(L, axis=-1, keepdims=True)
        lhat = L / ell
        u = np.cross(lhat, nrm)
        t = np.sum(u * (pa - r), axis=-1)
        sm = np.sum(lhat * (pa - r), axis=-1)
        sp = np.sum(lhat * (pb - r), axis=-1)
        Rm = np.linalg.norm(r - pa, axis=-1)
        Rp = np.linalg.norm(r - pb, axis=-1)
        R0sq = t * t + h * h
        on_line = np.abs(t) <= 1e-13 * scale
        lr = np.where(on_line, 0.0, _log_ratio(Rp, sp, Rm, sm, R0sq))
        acc_log += np.where(on_line, 0.0, t * lr)
        with np.errstate(invalid="ignore", divide="ignore"):
            at = (np.arctan2(t * sp, R0sq + ah * Rp) - np.arctan2(t * sm, R0sq + ah * Rm))
        acc_atan += np.where(ah <= 1e-13 * scale, 0.0, np.nan_to_num(at))
        acc_r += np.where(on_line, 0.0, t * (sp * Rp - sm * Rm + R0sq * lr))
    inv_r = acc_log - ah * acc_atan
    int_r = (h * h * inv_r + 0.5 * acc_r) / 3.0
    return inv_r, int_r


def tet_integrals(r, tet):
    """Return (int_T 1/R dV', int_T (r'-r)/R dV') for observers r[...,3], tets tet[...,4,3]."""
    r = np.asarray(r, dtype=np.float64)
    tet = np.asarray(tet, dtype=np.float64)
    cen = tet.mean(axis=-2)
    s_inv = 0.0
    s_vec = 0.0
    for i in range(4):
        idx = [j for j in range(4) if j != i]
        tri = tet[..., idx, :]
        nrm = np.cross(tri[..., 1, :] - tri[..., 0, :], tri[..., 2, :] - tri[..., 0, :])
        nrm = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
        # outward: away from the opposite vertex
        sgn = np.sign(np.sum(nrm * (tri[..., 0, :] - tet[..., i, :]), axis=-1))
        nrm = nrm * sgn[..., None]
        d = np.sum(nrm * (tri[..., 0, :] - r), axis=-1)
        fi, fr = tri_integrals(r, tri)
        s_inv = s_inv + 0.5 * d * fi
        s_vec = s_vec + nrm * fr[..., None]
    del cen
    return s_inv, s_vec
