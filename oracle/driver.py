"""One oracle solve of a meshed cell at one incidence (test infrastructure only)."""
import numpy as np

from .fill import Problem, assemble
from .post import absorption, reflect_transmit
from .solve import solve_dense
from .topology import build_topology


def solve_cell(cell, lam_nm, theta=0.0, phi=0.0, eps=None, topo=None, keep_matrix=False):
    """Fill Eq. (2), solve by dense LU, return absorption per domain, R, T per polarisation."""
    topo = topo or build_topology(cell)
    eps = cell.eps(lam_nm) if eps is None else np.asarray(eps, dtype=np.complex128)
    prob = Problem(topo, lam_nm, theta, phi, eps)
    Z, b = assemble(prob)
    x = solve_dense(Z, b)
    out = dict(topo=topo, prob=prob, x=x, A=[], R=[], T=[], dens=[])
    for p in range(2):
        A, dens = absorption(prob, x[:, p])
        R, T = reflect_transmit(prob, x[:, p], p)
        out["A"].append(A)
        out["dens"].append(dens)
        out["R"].append(R)
        out["T"].append(T)
    out["A"] = np.array(out["A"])
    out["R"] = np.array(out["R"])
    out["T"] = np.array(out["T"])
    out["residual"] = np.linalg.norm(Z @ x - b, axis=0) / np.linalg.norm(b, axis=0)
    if keep_matrix:
        out["Z"], out["b"] = Z, b
    return out
