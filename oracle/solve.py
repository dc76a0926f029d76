"""Linear solves for the oracle: dense LU, and the domain-block preconditioner (Eq. (5)-(6)).

The oracle's reference solution is a dense LU solve of Z x = b (LAPACK through
scipy).  The preconditioner of Sec. 2.3 is also restated: unknowns are grouped
by material domain (Eq. (5)), the diagonal blocks A_dd are factored, and the
left-preconditioned system diag(A_dd^-1) Z x = diag(A_dd^-1) b of Eq. (6) is
solved with a plain restarted GMRES that stops on the *unpreconditioned*
relative residual ||b - Z x|| / ||b||.

Domain of an unknown (the paper is silent on faces shared by two domains): a
face inside one domain belongs to it; an interface face belongs to the domain
with the larger |eps_r| (metal first), ties to the lower domain index; a half
function belongs to its tetrahedron's domain.
"""
import numpy as np
import scipy.linalg as sla

from .topology import KIND_HALF


def solve_dense(Z, b):
    lu = sla.lu_factor(Z)
    return sla.lu_solve(lu, b)


def unknown_domains(topo, eps_phys):
    dom = topo["domain"]
    dp = dom[topo["tp"]]
    dm = np.where(topo["kind"] == KIND_HALF, dp, dom[np.maximum(topo["tm"], 0)])
    mag = np.abs(np.asarray(eps_phys))
    pick_m = (mag[dm] > mag[dp]) | ((mag[dm] == mag[dp]) & (dm < dp))
    return np.where(pick_m, dm, dp)


def block_preconditioner(Z, udom):
    """LU factors of the diagonal blocks Z[d,d] of every domain d (Eq. (6))."""
    blocks = []
    for d in np.unique(udom):
        idx = np.nonzero(udom == d)[0]
        blocks.append((idx, sla.lu_factor(Z[np.ix_(idx, idx)])))

    def apply(v):
        out = np.empty_like(v)
        for idx, lu in blocks:
            out[idx] = sla.lu_solve(lu, v[idx])
        return out
    return apply


def gmres(Z, b, M=None, tol=1e-8, restart=100, maxiter=2000):
    """Left-preconditioned restarted GMRES; stops on ||b - Z x||/||b|| <= tol.

    Returns (x, iterations, history of true relative residuals at each check).
    """
    M = M or (lambda v: v)
    n = len(b)
    x = np.zeros(n, dtype=np.complex128)
    bn = np.linalg.norm(b)
    hist = []
    it = 0
    while it < maxiter:
        r_true = b - Z @ x
        rel = np.linalg.norm(r_true) / bn
        hist.append(rel)
        if rel <= tol:
            break
        r = M(r_true)
        beta = np.linalg.norm(r)
        V = np.zeros((n, restart + 1), np.complex128)
        H = np.zeros((restart + 1, restart), np.complex128)
        V[:, 0] = r / beta
        cs = np.zeros(restart, np.complex128)
        sn = np.zeros(restart, np.complex128)
        g = np.zeros(restart + 1, np.complex128)
        g[0] = beta
        # preconditioned target: a conservative fraction of the current residual
        target = beta * tol / max(rel, tol) * 0.5
        k_used = 0
        for k in range(restart):
            w = M(Z @ V[:, k])
            for j in range(k + 1):                 # modified Gram-Schmidt
                H[j, k] = np.vdot(V[:, j], w)
                w = w - H[j, k] * V[:, j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                V[:, k + 1] = w / H[k + 1, k]
            # Givens rotations: G_j = [[conj(c_j), conj(s_j)], [-s_j, c_j]] (unitary),
            # c = h_kk / den, s = h_(k+1)k / den zero the subdiagonal of column k
            for j in range(k):                     # apply previous rotations
                t = np.conj(cs[j]) * H[j, k] + np.conj(sn[j]) * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = np.hypot(abs(H[k, k]), abs(H[k + 1, k]))
            cs[k] = H[k, k] / den if den else 1.0
            sn[k] = H[k + 1, k] / den if den else 0.0
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) <= target or it >= maxiter:
                break
        y = sla.solve_triangular(H[:k_used, :k_used], g[:k_used])
        x = x + V[:, :k_used] @ y
    return x, it, hist
