"""Simplex quadrature rules used by the oracle (test infrastructure only).

The rules are part of the definition of the discrete problem: far element
pairs use the degree-2 rules, near pairs use the degree-5 rules for the outer
integral around a closed-form inner integral.  Points are barycentric
coordinates; weights sum to one (multiply by the element measure).

* tetrahedron, degree 2, 4 points: barycentric (alpha, beta, beta, beta) and
  permutations, alpha = (5 + 3 sqrt 5)/20, beta = (5 - sqrt 5)/20, weights 1/4.
* tetrahedron, degree 5, 14 points (fully symmetric rule of Walkington, also
  tabulated by Jaskowiec & Sukumar): orbits (a,a,a,1-3a) for two values of a
  and (c,c,1/2-c,1/2-c).
* triangle, degree 2, 3 points: (2/3, 1/6, 1/6) and permutations, weights 1/3.
* triangle, degree 5, 7 points (Radon): centroid plus two orbits with
  a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200, centroid 9/40.
"""
import itertools

import numpy as np


def _orbit(coords):
    return sorted(set(itertools.permutations(coords)))


def tet_deg2():
    s5 = np.sqrt(5.0)
    al, be = (5.0 + 3.0 * s5) / 20.0, (5.0 - s5) / 20.0
    pts = np.array(_orbit((al, be, be, be)))
    return pts, np.full(4, 0.25)


def tet_deg5():
    a1, w1 = 0.0927352503108912264, 0.0734930431163619495
    a2, w2 = 0.3108859192633006097, 0.1126879257180158507
    c3, w3 = 0.0455037041256496494, 0.0425460207770814664
    pts, wts = [], []
    for a, w in ((a1, w1), (a2, w2)):
        for p in _orbit((a, a, a, 1.0 - 3.0 * a)):
            pts.append(p)
            wts.append(w)
    for p in _orbit((c3, c3, 0.5 - c3, 0.5 - c3)):
        pts.append(p)
        wts.append(w3)
    return np.array(pts), np.array(wts)


def tri_deg2():
    pts = np.array(_orbit((2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0)))
    return pts, np.full(3, 1.0 / 3.0)


def tri_deg5():
    s15 = np.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    pts = [(1.0 / 3.0,) * 3]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        for p in _orbit((a, a, 1.0 - 2.0 * a)):
            pts.append(p)
            wts.append(w)
    return np.array(pts), np.array(wts)


def map_points(bary, verts):
    """Barycentric points [Q, k] on elements with vertices [..., k, 3] -> [..., Q, 3]."""
    return np.einsum("qk,...kd->...qd", bary, verts)
