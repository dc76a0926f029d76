"""Seeded synthetic unit cells for the periodic volume-integral-equation solver.

This module only *generates inputs*: tetrahedral meshes of one a x b unit cell
of a layered thin-film stack (optionally with embedded metal spheres) and the
per-domain relative permittivities at a wavelength.  It holds none of the
method's arithmetic (no basis functions, Green's functions, quadrature or
linear algebra), so both the FP64 CPU oracle and the CUDA path consume it.

Geometry follows the unit cell of the paper (Fig. 1, Sec. 2.3): a periodic
a x b cell, stacked layers of thickness D1, D2, ... and metal particles inside
the active layer.  The particles are spheres (not the paper's W x W x W cubes),
the material models are synthetic Drude / Cauchy fits (the paper's measured
P3HT:PCBM, PEDOT:PSS and Ag data are not available), and the mesh is a
structured Kuhn (6-tetrahedra-per-hexahedron) split of a graded tensor grid,
with seeded node jitter and nodes snapped to sphere surfaces.

Conventions: lengths in nm; permittivities use the physics sign (Im > 0 is
lossy); tetrahedra are positively oriented; periodic lateral faces match under
translation by (a, 0, 0) and (0, b, 0).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "Cell", "grid_1d", "kuhn_mesh", "slab_cell", "layered_cell",
    "eps_ag_drude", "eps_active", "eps_buffer",
    "config_slab", "config_plasmonic", "config_plasmonic_sample", "config_sweep_geometry", "small_cells",
    "ball_cell", "config_plasmonic_snap", "config_plasmonic_fine", "cube_cell", "config_large",
    "config_large_reduced", "paper_cube_cell", "two_layer_cell",
]


@dataclasses.dataclass
class Cell:
    verts: np.ndarray          # [n_verts, 3] float64, nm
    tets: np.ndarray           # [n_tets, 4] int32, positively oriented
    tet_domain: np.ndarray     # [n_tets] int32 in 0..n_domains-1
    n_domains: int
    period_a: float
    period_b: float
    active_domain: int
    domain_names: tuple
    name: str = ""

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def eps(self, lam_nm: float) -> np.ndarray:
        """Per-domain permittivity at lam_nm from the synthetic models."""
        table = {"ag": eps_ag_drude, "active": eps_active, "buffer": eps_buffer}
        out = []
        for nm in self.domain_names:
            if nm in table:
                out.append(complex(table[nm](lam_nm)))
            else:  # a constant permittivity written as "const:re,im"
                re, im = nm.split(":")[1].split(",")
                out.append(complex(float(re), float(im)))
        return np.array(out, dtype=np.complex128)


# ----------------------------------------------------------------------------
# synthetic material models (inputs, physics sign: Im eps > 0 is lossy)
# ----------------------------------------------------------------------------
_HC_EV_NM = 1239.841984  # h*c in eV*nm


def eps_ag_drude(lam_nm):
    """Silver, Drude fit: eps_inf 3.7, hbar*omega_p 9.1 eV, hbar*gamma 0.055 eV."""
    w = _HC_EV_NM / np.asarray(lam_nm, dtype=np.float64)
    return 3.7 - 9.1 ** 2 / (w * (w + 1j * 0.055))


def eps_active(lam_nm):
    """Organic active layer, Cauchy n plus a Gaussian absorption band near 500 nm."""
    lam = np.asarray(lam_nm, dtype=np.float64)
    n = 1.90 + 0.01925 / (lam * 1e-3) ** 2
    k = 0.1515 * np.exp(-((lam - 500.0) / 120.0) ** 2)
    return (n + 1j * k) ** 2


def eps_buffer(lam_nm):
    """Transparent-ish buffer / spacer layer, Cauchy n and constant k."""
    lam = np.asarray(lam_nm, dtype=np.float64)
    n = 1.52 + 0.0073 / (lam * 1e-3) ** 2
    return (n + 1j * 0.0161) ** 2


# ----------------------------------------------------------------------------
# structured meshes
# ----------------------------------------------------------------------------
def grid_1d(lo, hi, breaks=(), fine_zones=(), h_fine=None, h_coarse=10.0):
    """Graded 1D grid on [lo, hi] containing every break point exactly.

    Segments between consecutive break points (zone edges included) are split
    uniformly with spacing <= h_fine inside any fine zone, <= h_coarse outside.
    """
    pts = {float(lo), float(hi)}
    for b in breaks:
        if lo < b < hi:
            pts.add(float(b))
    for z0, z1 in fine_zones:
        for b in (z0, z1):
            if lo < b < hi:
                pts.add(float(b))
    pts = sorted(pts)
    out = [pts[0]]
    for p0, p1 in zip(pts[:-1], pts[1:]):
        mid = 0.5 * (p0 + p1)
        fine = any(z0 <= mid <= z1 for z0, z1 in fine_zones)
        h = h_fine if (fine and h_fine) else h_coarse
        n = max(1, int(math.ceil((p1 - p0) / h - 1e-9)))
        out.extend(np.linspace(p0, p1, n + 1)[1:].tolist())
    return np.array(out, dtype=np.float64)


def kuhn_mesh(xs, ys, zs):
    """Kuhn split of the tensor grid xs x ys x zs into 6 tetrahedra per hexahedron.

    Every hexahedron is cut along its (0,0,0)-(1,1,1) diagonal into the six
    path simplices; the split is translation invariant, so opposite lateral
    faces of the cell carry identical triangulations.
    """
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros(3, dtype=np.int64)
        path = [vid(I, J, K)]
        for ax in perm:
            off[ax] += 1
            path.append(vid(I + off[0], J + off[1], K + off[2]))
        tets.append(np.stack(path, axis=1))
    tets = np.concatenate(tets, axis=0).astype(np.int64)
    # order tets by hexahedron for locality
    order = np.argsort(np.tile(np.arange(I.size), 6), kind="stable")
    tets = tets[order]
    tets = _orient(verts, tets)
    return verts, tets.astype(np.int32)


def _signed_volumes(verts, tets):
    p = verts[tets]
    return np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0


def _orient(verts, tets):
    tets = tets.copy()
    neg = _signed_volumes(verts, tets) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return tets


def layered_cell(period_a, period_b, layers, spheres=(), h_coarse=20.0, h_fine=None,
                 h_z=None, jitter=0.1, seed=0, snap=0.4, name="", active_domain=None,
                 lateral_fine=True, particles="snap", ridges=None):
    """Layered unit cell with optional spheres.

    layers:  list of (thickness_nm, material_name) from bottom (z=0) to top.
    spheres: list of (cx, cy, cz, radius, material_name); each sphere gets its
             own domain, numbered after the layers.
    The grid is graded to spacing h_fine inside the bounding box of each sphere
    (plus half a fine cell), h_coarse elsewhere laterally, h_z (default
    h_coarse) vertically outside fine zones.
    particles: "snap" moves the grid nodes near each sphere surface radially
             onto it; "ball" maps the grid inside a cube of half-width r onto
             the ball and blends a shell of two fine cells out to the
             surrounding grid (a smooth particle surface without slivers or
             steps, conformal with the layers; the box of half-width r + 2
             h_fine must lie inside one layer and inside the cell).
    ridges:  optional (layer_index, [(x0, x1), ...], material_name): a grating
             in that layer, ridges along y occupying x in [x0, x1] (one domain,
             numbered after the spheres); the grid has planes at the ridge walls
             and jitter keeps their nodes on them.
    """
    if particles not in ("snap", "ball"):
        raise ValueError("particles must be 'snap' or 'ball'")
    rng = np.random.default_rng(seed)
    zb = np.concatenate([[0.0], np.cumsum([t for t, _ in layers])])
    fine_x, fine_y, fine_z = [], [], []
    brk_x, brk_y, brk_z = [], [], list(zb[1:-1])
    boxes = []   # "ball" particles: (centre, r, half-width of the blended box)
    for cx, cy, cz, r, _ in spheres:
        if particles == "ball":
            hb = h_fine or h_coarse
            L = r + 2.0 * hb
            if not (L < cx < period_a - L and L < cy < period_b - L):
                raise ValueError("a ball particle's box must lie inside the cell")
            if not any(z0 < cz - L and cz + L < z1 for z0, z1 in zip(zb[:-1], zb[1:])):
                raise ValueError("a ball particle's box must lie inside one layer")
            boxes.append((np.array([cx, cy, cz]), float(r), float(L)))
            fine_x.append((cx - L, cx + L))
            fine_y.append((cy - L, cy + L))
            fine_z.append((cz - L, cz + L))
            brk_x += [cx - L, cx - r, cx + r, cx + L]
            brk_y += [cy - L, cy - r, cy + r, cy + L]
            brk_z += [cz - L, cz - r, cz + r, cz + L]
            continue
        pad = 0.5 * (h_fine or h_coarse)
        fine_x.append((cx - r - pad, cx + r + pad))
        fine_y.append((cy - r - pad, cy + r + pad))
        fine_z.append((cz - r - pad, cz + r + pad))
    walls = sorted({float(x) for x0x1 in (ridges[1] if ridges else ()) for x in x0x1})
    brk_x = list(brk_x) + walls
    xs = grid_1d(0.0, period_a, brk_x, fine_x if (lateral_fine or boxes) else (), h_fine, h_coarse)
    ys = grid_1d(0.0, period_b, brk_y, fine_y if (lateral_fine or boxes) else (), h_fine, h_coarse)
    zs = grid_1d(0.0, zb[-1], brk_z, fine_z, h_fine, h_z or h_coarse)
    verts, tets = kuhn_mesh(xs, ys, zs)
    v0 = verts.copy()
    nxv, nyv, nzv = len(xs), len(ys), len(zs)
    ii, jj, kk = np.meshgrid(np.arange(nxv), np.arange(nyv), np.arange(nzv), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    lateral = (ii == 0) | (ii == nxv - 1) | (jj == 0) | (jj == nyv - 1)
    on_plane = np.isin(np.round(verts[:, 2], 9), np.round(zb, 9))
    # local spacing per node (min of adjacent grid steps)
    def _loc(g, idx):
        d = np.diff(g)
        left = np.where(idx > 0, d[np.clip(idx - 1, 0, len(d) - 1)], np.inf)
        right = np.where(idx < len(g) - 1, d[np.clip(idx, 0, len(d) - 1)], np.inf)
        return np.minimum(left, right)
    hloc = np.minimum(np.minimum(_loc(xs, ii), _loc(ys, jj)), _loc(zs, kk))

    snapped = np.zeros(len(verts), dtype=bool)
    inbox = np.zeros(len(verts), dtype=bool)
    for c, r, L in boxes:
        # inner cube (max-norm <= r) onto the ball of radius r; the shell out to
        # the box blends the ball surface (t = 0) into the grid (t = 1)
        d = verts - c
        sinf = np.abs(d).max(axis=1)
        nrm = np.linalg.norm(d, axis=1)
        sel = sinf <= L * (1.0 + 1e-9)
        unit = np.where(nrm[:, None] > 0, d / np.where(nrm > 0, nrm, 1.0)[:, None], 0.0)
        inner = sel & (sinf <= r * (1.0 + 1e-9))
        verts[inner] = c + unit[inner] * sinf[inner, None]
        shell = sel & ~inner
        t = ((sinf - r) / (L - r))[shell, None]
        verts[shell] = (1.0 - t) * (c + unit[shell] * r) + t * verts[shell]
        inbox |= sel
    for cx, cy, cz, r, _ in (spheres if particles == "snap" else ()):
        d = verts - np.array([cx, cy, cz])
        dist = np.linalg.norm(d, axis=1)
        near = (np.abs(dist - r) < snap * hloc) & ~lateral & ~on_plane & (dist > 0)
        verts[near] = np.array([cx, cy, cz]) + d[near] * (r / dist[near])[:, None]
        snapped |= near
    # seeded jitter: free interior nodes in 3D, interface/top/bottom nodes in-plane
    if jitter > 0:
        free = ~lateral & ~snapped & ~inbox
        dj = rng.uniform(-jitter, jitter, size=verts.shape) * hloc[:, None]
        dj[on_plane, 2] = 0.0
        if walls:   # ridge walls stay planar
            dj[np.isin(np.round(verts[:, 0], 9), np.round(walls, 9)), 0] = 0.0
        # keep jittered nodes clear of sphere surfaces (no accidental straddling)
        cand = verts + dj
        for cx, cy, cz, r, _ in spheres:
            d0 = np.linalg.norm(verts - np.array([cx, cy, cz]), axis=1)
            d1 = np.linalg.norm(cand - np.array([cx, cy, cz]), axis=1)
            free &= ~((d0 - r) * (d1 - r) <= 0) | (np.abs(d0 - r) > 1.5 * hloc)
        verts[free] = cand[free]
    # reject inverted / degenerate tets by undoing moves of their nodes
    vol0 = _signed_volumes(v0, tets)
    for _ in range(20):
        vol = _signed_volumes(verts, tets)
        bad = vol < 0.15 * vol0
        if not bad.any():
            break
        nodes = np.unique(tets[bad])
        nodes = nodes[~inbox[nodes]]   # the ball mapping stays
        if not len(nodes):
            break
        verts[nodes] = v0[nodes]
    vol = _signed_volumes(verts, tets)
    assert (vol > 0).all(), "mesh generation produced an inverted tetrahedron"

    cent = verts[tets].mean(axis=1)
    dom = np.searchsorted(zb, cent[:, 2], side="right") - 1
    dom = np.clip(dom, 0, len(layers) - 1).astype(np.int32)
    names = [m for _, m in layers]
    cent0 = v0[tets].mean(axis=1)
    for s, (cx, cy, cz, r, m) in enumerate(spheres):
        if particles == "ball":   # the tetrahedra of the mapped inner cube
            inside = np.abs(cent0 - np.array([cx, cy, cz])).max(axis=1) < r
        else:
            inside = np.linalg.norm(cent - np.array([cx, cy, cz]), axis=1) < r
        dom[inside] = len(layers) + s
        names.append(m)
    if ridges:
        li, spans, m = ridges
        in_layer = dom == li
        on_ridge = np.zeros(len(dom), dtype=bool)
        for x0, x1 in spans:
            on_ridge |= (cent[:, 0] > x0) & (cent[:, 0] < x1)
        dom[in_layer & on_ridge] = len(names)
        names.append(m)
    if active_domain is None:
        active_domain = names.index("active") if "active" in names else 0
    return Cell(verts=verts, tets=tets.astype(np.int32), tet_domain=dom,
                n_domains=len(names), period_a=float(period_a), period_b=float(period_b),
                active_domain=int(active_domain), domain_names=tuple(names), name=name)


def slab_cell(nx, ny, nz, a=200.0, b=200.0, d=40.0, eps=(4.0, 0.5), jitter=0.0, seed=0):
    """Homogeneous slab of thickness d filling the a x b cell, uniform nx x ny x nz grid."""
    xs = np.linspace(0.0, a, nx + 1)
    ys = np.linspace(0.0, b, ny + 1)
    zs = np.linspace(0.0, d, nz + 1)
    verts, tets = kuhn_mesh(xs, ys, zs)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        h = min(a / nx, b / ny, d / nz)
        interior = ((verts[:, 0] > 1e-9) & (verts[:, 0] < a - 1e-9)
                    & (verts[:, 1] > 1e-9) & (verts[:, 1] < b - 1e-9))
        dj = rng.uniform(-jitter, jitter, size=verts.shape) * h
        planar = (np.abs(verts[:, 2]) < 1e-9) | (np.abs(verts[:, 2] - d) < 1e-9)
        dj[planar, 2] = 0.0
        verts = verts.copy()
        verts[interior] += dj[interior]
        assert (_signed_volumes(verts, tets) > 0).all()
    name = "const:%r,%r" % (float(eps[0]), float(eps[1]))
    return Cell(verts=verts, tets=tets, tet_domain=np.zeros(len(tets), np.int32), n_domains=1,
                period_a=float(a), period_b=float(b), active_domain=0,
                domain_names=(name,), name="slab_%dx%dx%d" % (nx, ny, nz))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def config_slab():
    """Homogeneous absorbing slab: period 200 nm, 40 nm thick, eps 4.0+0.5i, 6x6x2 hexahedra (432 tets)."""
    return slab_cell(6, 6, 2, 200.0, 200.0, 40.0, (4.0, 0.5))


def config_plasmonic(seed=2, h_coarse=30.0, h_fine=10.0, h_z=25.0, particles="ball"):
    """Plasmonic cell: period 200 nm, Ag sphere r=20 nm centred in a 100 nm active
    layer over a 40 nm buffer (three material domains), 10,368 tetrahedra and
    21,024 SWG unknowns.  The sphere is meshed as a mapped cube (384
    tetrahedra, smooth surface, particles="ball", see layered_cell);
    particles="snap" snaps the grid nodes near its surface instead."""
    return layered_cell(200.0, 200.0, [(40.0, "buffer"), (100.0, "active")],
                        spheres=[(100.0, 100.0, 90.0, 20.0, "ag")],
                        h_coarse=h_coarse, h_fine=h_fine, h_z=h_z, jitter=0.1, seed=seed,
                        name="plasmonic_200nm_r20" + ("_ball" if particles == "ball" else "_snap"),
                        particles=particles)


def config_plasmonic_snap(seed=2):
    """The plasmonic cell with the grid nodes near the sphere snapped onto it
    (10,368 tetrahedra, 21,024 unknowns, 1,098 of them in the sphere): a
    faceted particle surface on which the metal's absorption is not reliable."""
    return config_plasmonic(seed=seed, h_coarse=28.0, h_fine=9.5, particles="snap")


def config_plasmonic_fine(seed=2):
    """The plasmonic cell with a finer mapped-cube sphere (750 tetrahedra;
    17,550 tetrahedra, 35,550 unknowns in all)."""
    return config_plasmonic(seed=seed, h_coarse=28.0, h_fine=9.5, particles="ball")


def config_plasmonic_sample(seed=2):
    """The plasmonic geometry at a much lower density (378 tets): the bounded
    sample on which the CPU oracle is timed."""
    return layered_cell(200.0, 200.0, [(40.0, "buffer"), (100.0, "active")],
                        spheres=[(100.0, 100.0, 90.0, 20.0, "ag")],
                        h_coarse=67.0, h_fine=20.0, h_z=30.0, jitter=0.1, seed=seed, lateral_fine=False,
                        name="plasmonic_200nm_r20_sample")


def config_sweep_geometry(seed=3):
    """The plasmonic geometry at the coarser density used for wavelength x angle
    sweeps: 4,860 tets, 9,882 SWG unknowns (a 162-tetrahedron mapped-cube sphere)."""
    return config_plasmonic(seed=seed, h_coarse=60.0, h_fine=14.5, h_z=40.0)


def serving_cell(index, master_seed=4):
    """One seeded random cell of the serving stream: square period U[150, 400] nm,
    an active layer and a buffer layer of thicknesses U[30, 150] nm, 0-4 Ag
    spheres of radius U[10, 40] nm (kept inside the active layer and apart
    laterally), mesh density aimed at a log-uniform 2k-40k SWG unknowns.
    Returns (cell, target_unknowns)."""
    rng = np.random.default_rng([master_seed, index])
    a = float(rng.uniform(150.0, 400.0))
    t_act = float(rng.uniform(30.0, 150.0))
    t_buf = float(rng.uniform(30.0, 150.0))
    n_sph = int(rng.integers(0, 5))
    target = float(np.exp(rng.uniform(np.log(2000.0), np.log(40000.0))))
    spheres = []
    slots = [(0.25, 0.25), (0.75, 0.75), (0.75, 0.25), (0.25, 0.75)]
    for k in range(n_sph):
        r = float(rng.uniform(10.0, 40.0))
        r = min(r, 0.4 * t_act, 0.2 * a)
        fx, fy = slots[k]
        spheres.append((fx * a, fy * a, t_buf + 0.5 * t_act, r, "ag"))
    # ~2.05 unknowns per tetrahedron, 6 tetrahedra per grid cell; the graded
    # tensor grid is counted before meshing and its coarse spacing scaled to the
    # target (cells whose spheres alone need more land above it)
    zb = [0.0, t_buf, t_buf + t_act]
    h0 = (a * a * (t_act + t_buf) / (target / 2.05 / 6.0)) ** (1.0 / 3.0)
    hf0 = min(h0, min(sp[3] for sp in spheres) / 1.2) if spheres else None

    r_min = min(sp[3] for sp in spheres) if spheres else None

    def spacing(sc, coarse_spheres=False):
        # the coarse spacing scales; spheres keep h_fine <= r / 1.2, or <= r
        # when that alone would exceed the target
        hc = h0 * sc
        hf = min(r_min if coarse_spheres else hf0, hc) if spheres else None
        pad = 0.5 * (hf or hc)
        fx = [(sp[0] - sp[3] - pad, sp[0] + sp[3] + pad) for sp in spheres]
        fy = [(sp[1] - sp[3] - pad, sp[1] + sp[3] + pad) for sp in spheres]
        fz = [(sp[2] - sp[3] - pad, sp[2] + sp[3] + pad) for sp in spheres]
        nx = len(grid_1d(0.0, a, (), fx, hf, hc)) - 1
        ny = len(grid_1d(0.0, a, (), fy, hf, hc)) - 1
        nz = len(grid_1d(0.0, zb[-1], zb[1:-1], fz, hf, hc)) - 1
        return 6 * nx * ny * nz, hc, hf

    coarse = spacing(20.0)[0] * 2.05 > 1.2 * target
    lo, hi = 0.1, 20.0
    for _ in range(40):                      # bisection on the spacing scale (count decreases with it)
        mid = math.sqrt(lo * hi)
        if spacing(mid, coarse)[0] * 2.05 > target:
            lo = mid
        else:
            hi = mid
    _, hc, hf = spacing(hi, coarse)
    cell = layered_cell(a, a, [(t_buf, "buffer"), (t_act, "active")], spheres=spheres,
                        h_coarse=hc, h_fine=hf, h_z=hc, jitter=0.1, seed=int(rng.integers(1 << 30)),
                        name="serving_%d" % index)
    return cell, target


def ball_cell(period, radius, n, material="const:4.0,1.0"):
    """A lone sphere centred in a period x period cell, in vacuum, meshed as a
    Kuhn-split n x n x n cube mapped radially onto the ball (each cube shell
    max|p| = s goes to the sphere of radius s r): a smooth surface without the
    slivers and steps of a snapped grid.  Its outer faces carry the body's
    boundary functions and none touches the lateral faces."""
    g = np.linspace(-1.0, 1.0, n + 1)
    verts, tets = kuhn_mesh(g, g, g)
    shell = np.abs(verts).max(axis=1)
    norm = np.linalg.norm(verts, axis=1)
    scale = np.where(norm > 0, shell / np.where(norm > 0, norm, 1.0), 0.0)
    verts = verts * scale[:, None] * radius + 0.5 * np.array([period, period, period])
    tets = _orient(verts, tets)
    return Cell(verts=verts, tets=tets.astype(np.int32), tet_domain=np.zeros(len(tets), dtype=np.int32),
                n_domains=1, period_a=float(period), period_b=float(period), active_domain=0,
                domain_names=(material,), name="ball")


def config_large(h_coarse=24.0, h_fine=12.0, h_z=20.0, particles="snap", seed=5, lateral_fine=True,
                 name="large_400nm_2x2"):
    """The large cell: period 400 nm, a 2 x 2 array of Ag spheres (r = 35 nm)
    centred in a 120 nm active layer, over a 40 nm periodic Ag back grating
    (ridges 40 nm wide along y, two per period, the gaps filled with the
    buffer material).  Domains: 0 grating gaps (buffer), 1 active, 2-5 the
    spheres, 6 the ridges.  The default density gives 44,550 tetrahedra and
    about 91k SWG unknowns (the dense FP32 Z is ~66 GB).  The spheres are
    snapped (a mapped-cube ball of r = 35 nm needs h_fine <= 12.5 nm inside the
    120 nm layer, which alone would exceed this size)."""
    spheres = [(x, y, 100.0, 35.0, "ag") for y in (100.0, 300.0) for x in (100.0, 300.0)]
    return layered_cell(400.0, 400.0, [(40.0, "buffer"), (120.0, "active")], spheres=spheres,
                        h_coarse=h_coarse, h_fine=h_fine, h_z=h_z, jitter=0.1, seed=seed, name=name,
                        particles=particles, lateral_fine=lateral_fine,
                        ridges=(0, [(80.0, 120.0), (280.0, 320.0)], "ag"))


def config_large_reduced(seed=5):
    """The large cell's geometry at a density the FP64 oracle solves in under a
    minute: 720 tetrahedra, 1,500 unknowns, every domain present."""
    return config_large(h_coarse=80.0, h_fine=50.0, h_z=40.0, seed=seed, lateral_fine=False, name="large_reduced")


def cube_cell(period, d_spacer, d_active, side, h_fine, h_coarse=None, particle=True, name=""):
    """The unit cell of the paper's Sec. 3 experiments (Fig. 1): a spacer layer
    (z in [0, D1], the synthetic "buffer" material) under the active layer
    (z in [D1, D1 + D2]) with one metal cube of side W centred in the active
    layer and in the period x period cell.  The tensor grid has planes on the
    layer interface and on the six cube faces (spacing <= h_fine across the
    cube, <= h_coarse elsewhere), so the cube is exactly W^3; no jitter.
    Domains: 0 spacer, 1 active, 2 the cube.  particle=False keeps the same
    mesh and domains but fills the cube with the active material (the cell
    "without NPs" of the paper's enhancement: A(with) / A(without), both
    integrated over the active material only)."""
    c, half = 0.5 * period, 0.5 * side
    zc = d_spacer + 0.5 * d_active
    if not (half < c and d_spacer < zc - half and zc + half < d_spacer + d_active):
        raise ValueError("the cube must lie inside the active layer and the cell")
    hc = h_coarse or h_fine
    xs = grid_1d(0.0, period, (c - half, c + half), [(c - half, c + half)], h_fine, hc)
    zs = grid_1d(0.0, d_spacer + d_active, (d_spacer, zc - half, zc + half), [(zc - half, zc + half)], h_fine, hc)
    verts, tets = kuhn_mesh(xs, xs, zs)
    cent = verts[tets].mean(axis=1)
    dom = (cent[:, 2] > d_spacer).astype(np.int32)
    inside = ((np.abs(cent[:, 0] - c) < half) & (np.abs(cent[:, 1] - c) < half) & (np.abs(cent[:, 2] - zc) < half))
    dom[inside] = 2
    names = ("buffer", "active", "ag" if particle else "active")
    return Cell(verts=verts, tets=tets.astype(np.int32), tet_domain=dom, n_domains=3, period_a=float(period),
                period_b=float(period), active_domain=1, domain_names=names,
                name=name or "cube_W%g_a%g%s" % (side, period, "" if particle else "_noNP"))


def paper_cube_cell(h_fine=5.0, h_coarse=10.0, particle=True, geometry=None):
    """The paper's preconditioner experiment (Sec. 3, Fig. 2-3): Ag cubes W = 20 nm
    on a square lattice a = b = 40 nm, 20 nm spacer, 60 nm active layer.
    `geometry` (a dict with cube_side_nm, period_nm, spacer_thickness_nm,
    active_thickness_nm) overrides those values."""
    g = geometry or {"cube_side_nm": 20.0, "period_nm": 40.0, "spacer_thickness_nm": 20.0,
                     "active_thickness_nm": 60.0}
    return cube_cell(g["period_nm"], g["spacer_thickness_nm"], g["active_thickness_nm"], g["cube_side_nm"],
                     h_fine, h_coarse, particle=particle, name="paper_fig2_cube")


def two_layer_cell(period, d_buffer, d_active, nxy, h_z, eps_buffer=None, eps_active=None):
    """A laterally homogeneous two-layer stack (buffer below, active on top, no
    particles) on a uniform nxy x nxy lateral grid: a case with a closed form
    (transfer matrix).  eps_* = None uses the synthetic dispersive models,
    else a constant complex permittivity."""
    def mat(e, named):
        return named if e is None else "const:%r,%r" % (float(np.real(e)), float(np.imag(e)))
    return layered_cell(period, period, [(d_buffer, mat(eps_buffer, "buffer")), (d_active, mat(eps_active, "active"))],
                        h_coarse=period / nxy, h_z=h_z, jitter=0.0, seed=0, active_domain=1,
                        name="two_layer_%dx%d_hz%g" % (nxy, nxy, h_z))


def small_cells():
    """Small cells the oracle finishes in seconds (parity cases)."""
    return {
        "slab_3x3x1": slab_cell(3, 3, 1, 200.0, 200.0, 40.0, (4.0, 0.5)),
        "slab_4x3x2_jit": slab_cell(4, 3, 2, 180.0, 150.0, 40.0, (3.0, 0.8), jitter=0.12, seed=11),
        "plasmonic_tiny": layered_cell(60.0, 54.0, [(20.0, "buffer"), (40.0, "active")],
                                       spheres=[(30.0, 27.0, 40.0, 13.0, "ag")],
                                       h_coarse=20.0, h_fine=10.0, h_z=20.0, jitter=0.1, seed=7,
                                       lateral_fine=False, name="plasmonic_tiny"),
        "plasmonic_mini": layered_cell(120.0, 120.0, [(30.0, "buffer"), (50.0, "active")],
                                       spheres=[(60.0, 60.0, 55.0, 15.0, "ag")],
                                       h_coarse=40.0, h_fine=15.0, h_z=30.0, jitter=0.1, seed=5,
                                       name="plasmonic_mini"),
    }
