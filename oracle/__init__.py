"""FP64 CPU oracle for the preconditioned periodic SWG volume integral equation.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it; the
product path (`paper_1809_05334_gb300`) never imports, links or calls it, and
it shares no code, tables or helpers with `paper_1809_05334_gb300/csrc`.

What it computes (He, Gu, Sha & Chen, "Efficient volumetric method of moments
for modeling plasmonic thin-film solar cells with periodic structures"):

* topology.py   SWG basis functions on a tetrahedral unit cell (Sec. 2.1), with
                Bloch-periodic pairing of lateral faces (Sec. 2.2).
* quadrature.py the simplex quadrature rules that define the discrete problem.
* greens.py     the 2D periodic Green's function, Eq. (3)-(4), by the Ewald
                split into spatial and spectral series (Sec. 2.2), plus the
                plain spectral and windowed spatial lattice sums used to pin it.
* potentials.py closed-form integrals of 1/R and R over triangles and
                tetrahedra (singularity extraction for touching elements).
* fill.py       the Galerkin impedance matrix Z and right-hand side, Eq. (2).
* solve.py      dense LU solve, and the domain-block preconditioner of
                Eq. (5)-(6) with a plain restarted GMRES.
* post.py       absorbed fraction, Eq. (7), reflectance and transmittance, and
                the relative current error of Eq. (8).

Every function is FP64 and written for clarity, not speed.
"""

from .topology import build_topology  # noqa: F401
from .fill import assemble, Problem  # noqa: F401
from .solve import solve_dense, block_preconditioner, gmres  # noqa: F401
from .post import absorption, reflect_transmit, relative_error  # noqa: F401
from .driver import solve_cell  # noqa: F401
