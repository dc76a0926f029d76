"""SWG basis functions on a periodic tetrahedral unit cell (oracle, test infrastructure).

Schaubert-Wilton-Glisson (SWG) functions expand the flux density D (Sec. 2.1):
one unknown per face n, with f_n = +(a_n / 3V+)(r - v+) on T+ and
f_n = -(a_n / 3V-)(r - v-) on T-, where a_n is the face area and v+- the
vertex of T+- opposite the face.  f_n has unit normal flux across the face,
divergence +-a_n/V+- and a continuous normal component.

Faces on the top/bottom of the body (vacuum outside) carry a half function
(T+ only, flux leaving the body).  Faces on the lateral cell walls x=0/x=a
and y=0/y=b are paired into one Bloch-periodic function (Sec. 2.2): T+ is the
tetrahedron at the x=0 (y=0) wall, T- the one at the x=a (y=b) wall, and the
T- half is the image of that tetrahedron shifted by s = (a,0,0) or (0,b,0).
In the cell it enters the source side with weight exp(-j k_par . s) and the
test side with weight exp(+j k_par . s).

Canonical numbering, shared as a *convention* with the CUDA path so that
coefficient vectors can be compared entry by entry: local face i of a
tetrahedron is the face opposite its vertex i; unknowns are numbered in order
of first appearance when scanning tetrahedra t = 0.. and local faces i = 0..3;
T+ of an interior face is the lower-numbered tetrahedron.
"""
import numpy as np

KIND_INTERIOR, KIND_HALF, KIND_PERIODIC = 0, 1, 2


def _face_local(i):
    return [j for j in range(4) if j != i]


def build_topology(cell):
    """Return a dict describing the SWG space of `cell` (see module docstring)."""
    verts = np.asarray(cell.verts, dtype=np.float64)
    tets = np.asarray(cell.tets, dtype=np.int64)
    nt = tets.shape[0]
    a, b = float(cell.period_a), float(cell.period_b)
    tol = 1e-9 * max(a, b)

    owners = {}   # sorted vertex triple -> list of (t, i)
    for t in range(nt):
        for i in range(4):
            key = tuple(sorted(tets[t, _face_local(i)].tolist()))
            owners.setdefault(key, []).append((t, i))

    # classify single-owner faces
    def wall(key):
        p = verts[list(key)]
        if np.all(np.abs(p[:, 0]) < tol):
            return "x0"
        if np.all(np.abs(p[:, 0] - a) < tol):
            return "xa"
        if np.all(np.abs(p[:, 1]) < tol):
            return "y0"
        if np.all(np.abs(p[:, 1] - b) < tol):
            return "yb"
        return None

    partner = {}
    upper = {}
    for wlo, whi, s in (("x0", "xa", np.array([a, 0.0, 0.0])), ("y0", "yb", np.array([0.0, b, 0.0]))):
        lo = {}
        hi = {}
        for key, own in owners.items():
            if len(own) != 1:
                continue
            w = wall(key)
            if w == wlo:
                lo[_geom_key(verts[list(key)])] = key
            elif w == whi:
                hi[_geom_key(verts[list(key)] - s)] = key
        if set(lo) != set(hi):
            raise ValueError("periodic walls %s/%s do not match" % (wlo, whi))
        for gk, klo in lo.items():
            khi = hi[gk]
            partner[klo] = (khi, s)
            partner[khi] = (klo, s)
            upper[khi] = True

    basis = -np.ones((nt, 4), dtype=np.int64)
    sign = np.zeros((nt, 4), dtype=np.float64)
    shift = np.zeros((nt, 4, 3), dtype=np.float64)
    info = []  # per basis: kind, tp, ip, tm, im, shift
    for t in range(nt):
        for i in range(4):
            if basis[t, i] >= 0:
                continue
            key = tuple(sorted(tets[t, _face_local(i)].tolist()))
            own = owners[key]
            n = len(info)
            if len(own) == 2:
                (tp, ip), (tm, im) = sorted(own)
                info.append((KIND_INTERIOR, tp, ip, tm, im, np.zeros(3)))
                basis[tp, ip], sign[tp, ip] = n, 1.0
                basis[tm, im], sign[tm, im] = n, -1.0
            elif key in partner:
                other, s = partner[key]
                klo, khi = (other, key) if key in upper else (key, other)
                (tp, ip), = owners[klo]
                (tm, im), = owners[khi]
                info.append((KIND_PERIODIC, tp, ip, tm, im, s.copy()))
                basis[tp, ip], sign[tp, ip] = n, 1.0
                basis[tm, im], sign[tm, im] = n, -1.0
                shift[tm, im] = s
            else:
                info.append((KIND_HALF, t, i, -1, -1, np.zeros(3)))
                basis[t, i], sign[t, i] = n, 1.0
    assert (basis >= 0).all()

    nb = len(info)
    kind = np.array([x[0] for x in info], dtype=np.int64)
    tp = np.array([x[1] for x in info], dtype=np.int64)
    ip = np.array([x[2] for x in info], dtype=np.int64)
    tm = np.array([x[3] for x in info], dtype=np.int64)
    im = np.array([x[4] for x in info], dtype=np.int64)
    bshift = np.array([x[5] for x in info], dtype=np.float64).reshape(nb, 3)

    P = verts[tets]                                   # [nt,4,3]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0]) / 6.0
    if np.any(vol <= 0):
        raise ValueError("tetrahedra must be positively oriented")
    face_verts = np.stack([P[:, _face_local(i)] for i in range(4)], axis=1)   # [nt,4,3,3]
    cr = np.cross(face_verts[:, :, 1] - face_verts[:, :, 0], face_verts[:, :, 2] - face_verts[:, :, 0])
    area = 0.5 * np.linalg.norm(cr, axis=-1)          # [nt,4]
    dom = np.asarray(cell.tet_domain, dtype=np.int64)
    charge = (kind == KIND_HALF) | ((kind != KIND_HALF) & (dom[tp] != dom[np.maximum(tm, 0)]))
    return dict(
        n=nb, nt=nt, verts=verts, tets=tets, tet_verts=P, vol=vol, area=area,
        face_verts=face_verts, basis=basis, sign=sign, shift=shift,
        kind=kind, tp=tp, ip=ip, tm=tm, im=im, bshift=bshift,
        domain=dom, n_domains=int(cell.n_domains), a=a, b=b,
        charge_faces=np.nonzero(charge)[0],
    )


def _geom_key(p):
    q = np.round(np.asarray(p, dtype=np.float64), 6) + 0.0
    return tuple(sorted(tuple(r) for r in q.tolist()))
