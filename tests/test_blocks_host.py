"""Host logic of the preconditioner's domain blocks (CPU, no GPU): csrc/blocks.cpp
(Eq. (5) grouping, the blocked permutation, the sub-block variant) against the
oracle's grouping rule (oracle/solve.py: unknown_domains).

A small C++ program compiled here against the library's topology.cpp and
blocks.cpp prints the permutation (canonical unknown -> matrix row) and the
blocks.  Every block must hold the unknowns of one domain (the oracle's rule:
a face between two materials goes to the larger |eps|, ties to the lower
index), the blocks in domain order and each by unknown id; with a sub-block
size, the pieces of a domain partition it, none larger than the size, and
each piece is spatially compact (a bisection: its centroid box is no longer
along any axis than its domain's).
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import cellgen
from oracle.solve import unknown_domains
from oracle.topology import build_topology

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05334_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "blocks.h"
using namespace vie;
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int hdr[5];
    double ab[2];
    if (fread(hdr, sizeof(int), 5, f) != 5 || fread(ab, sizeof(double), 2, f) != 2) return 2;
    const int nv = hdr[0], nt = hdr[1], nd = hdr[2], act = hdr[3], bmax = hdr[4];
    std::vector<double> v(3 * (size_t)nv), ea(nd);
    std::vector<int32_t> t(4 * (size_t)nt), d(nt);
    if (fread(v.data(), 8, v.size(), f) != v.size() || fread(t.data(), 4, t.size(), f) != t.size() ||
        fread(d.data(), 4, d.size(), f) != d.size() || fread(ea.data(), 8, ea.size(), f) != ea.size()) return 3;
    fclose(f);
    Topology T;
    if (!build_topology(v.data(), nv, t.data(), nt, d.data(), nd, ab[0], ab[1], act, T).empty()) return 4;
    std::vector<int32_t> perm;
    std::vector<int> off, n;
    domain_blocks(T, ea, bmax, perm, off, n);
    printf("{\"perm\": [");
    for (size_t i = 0; i < perm.size(); ++i) printf("%s%d", i ? "," : "", perm[i]);
    printf("], \"off\": [");
    for (size_t i = 0; i < off.size(); ++i) printf("%s%d", i ? "," : "", off[i]);
    printf("], \"n\": [");
    for (size_t i = 0; i < n.size(); ++i) printf("%s%d", i ? "," : "", n[i]);
    printf("]}\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("blocks")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-O1", "-std=c++17", "-fopenmp", "-I", CSRC, str(src), os.path.join(CSRC, "topology.cpp"),
                    os.path.join(CSRC, "blocks.cpp"), "-o", str(exe)], check=True)
    return str(exe), d


def _blocks(harness, cell, eps, bmax):
    exe, d = harness
    path = d / ("%s_%d.bin" % (cell.name, bmax))
    with open(path, "wb") as f:
        np.array([len(cell.verts), len(cell.tets), cell.n_domains, cell.active_domain, bmax], np.int32).tofile(f)
        np.array([cell.period_a, cell.period_b], np.float64).tofile(f)
        np.ascontiguousarray(cell.verts, np.float64).tofile(f)
        np.ascontiguousarray(cell.tets, np.int32).tofile(f)
        np.ascontiguousarray(cell.tet_domain, np.int32).tofile(f)
        np.abs(np.asarray(eps, np.complex128)).astype(np.float64).tofile(f)
    out = subprocess.run([exe, str(path)], check=True, capture_output=True, text=True).stdout
    r = json.loads(out)
    return np.array(r["perm"]), np.array(r["off"]), np.array(r["n"])


CASES = [("plasmonic_tiny", 520.0), ("plasmonic_mini", 500.0), ("plasmonic_mini", 780.0)]


@pytest.mark.parametrize("name,lam", CASES)
def test_blocks_follow_the_grouping_rule(harness, name, lam):
    cell = cellgen.small_cells()[name]
    eps = cell.eps(lam)
    perm, off, n = _blocks(harness, cell, eps, 0)
    topo = build_topology(cell)
    udom = unknown_domains(topo, eps)
    N = len(udom)
    assert sorted(perm.tolist()) == list(range(N))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(n)[:-1]])) and n.sum() == N
    doms = [d for d in range(cell.n_domains) if np.any(udom == d)]
    assert len(n) == len(doms)
    for k, d in enumerate(doms):   # block k: the unknowns of domain d, by unknown id
        ids = np.nonzero(udom == d)[0]
        assert n[k] == len(ids)
        assert np.array_equal(perm[ids], off[k] + np.arange(len(ids)))


def test_sub_blocks_partition_each_domain(harness):
    cell = cellgen.small_cells()["plasmonic_mini"]
    eps = cell.eps(500.0)
    bmax = 300
    perm, off, n = _blocks(harness, cell, eps, bmax)
    topo = build_topology(cell)
    udom = unknown_domains(topo, eps)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    assert np.all(n <= bmax) and n.sum() == len(perm)
    cen = cell.verts[cell.tets].mean(axis=1)[topo["tp"]]
    pieces_of = {}
    for o, m in zip(off, n):
        ids = inv[o:o + m]
        d = np.unique(udom[ids])
        assert len(d) == 1                               # a piece never mixes domains
        assert np.all(np.diff(ids) > 0)                  # by unknown id inside a piece
        pieces_of.setdefault(int(d[0]), []).append(ids)
    for d, pcs in pieces_of.items():
        allids = np.sort(np.concatenate(pcs))
        assert np.array_equal(allids, np.nonzero(udom == d)[0])
        if len(pcs) > 1:
            ext = np.ptp(cen[allids], axis=0)
            for ids in pcs:
                assert np.all(np.ptp(cen[ids], axis=0) <= ext + 1e-9)
            # bisection halves the longest extent: some piece is strictly shorter along it
            ax = int(np.argmax(ext))
            assert min(np.ptp(cen[ids], axis=0)[ax] for ids in pcs) < ext[ax]
