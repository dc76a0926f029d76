"""Host logic of the library's mesh set-up (CPU, no GPU): the SWG topology and
the near-pair lists of csrc/topology.cpp against the oracle's independent
construction (oracle/topology.py, oracle/fill.py).

A small C++ program, compiled here with the host compiler against the
library's own topology.cpp, builds the topology of a mesh and prints it.  The
unknowns must be the oracle's, in the same canonical order (the GPU parity
tests compare Z entry by entry in that order): per tetrahedron face the
unknown, its sign (T+ / T-) and the lattice shift of a Bloch-paired T- half;
per unknown its kind and tetrahedra; the charge-carrying faces; and per
ordered tetrahedron pair the 9-bit mask of the lattice images in which the
pair is near (Sec. 2.2 split of the static part).
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import cellgen
from oracle.fill import _near_images
from oracle.topology import build_topology

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05334_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "vie_internal.h"
using namespace vie;
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int hdr[4];
    double ab[2];
    if (fread(hdr, sizeof(int), 4, f) != 4 || fread(ab, sizeof(double), 2, f) != 2) return 2;
    const int nv = hdr[0], nt = hdr[1], nd = hdr[2], act = hdr[3];
    std::vector<double> v(3 * (size_t)nv);
    std::vector<int32_t> t(4 * (size_t)nt), d(nt);
    if (fread(v.data(), sizeof(double), v.size(), f) != v.size() || fread(t.data(), 4, t.size(), f) != t.size() ||
        fread(d.data(), 4, d.size(), f) != d.size()) return 3;
    fclose(f);
    Topology T;
    std::string e = build_topology(v.data(), nv, t.data(), nt, d.data(), nd, ab[0], ab[1], act, T);
    if (!e.empty()) { printf("{\"error\": \"%s\"}\n", e.c_str()); return 0; }
    auto arr = [](const char *name, const auto &x, bool last = false) {
        printf("\"%s\": [", name);
        for (size_t i = 0; i < x.size(); ++i) printf("%s%d", i ? "," : "", (int)x[i]);
        printf("]%s", last ? "" : ", ");
    };
    printf("{\"N\": %d, ", T.N);
    arr("basis", T.basis); arr("sgn", T.sgn); arr("shift", T.shift); arr("kind", T.kind);
    arr("tp", T.tp); arr("ip", T.ip); arr("tm", T.tm); arr("im", T.im); arr("cf", T.cf); arr("hf", T.hf);
    printf("\"near_tt\": [");
    for (size_t i = 0; i < T.near_tt.size(); ++i)
        printf("%s[%d,%d,%d]", i ? "," : "", T.near_tt[i].x, T.near_tt[i].y, (int)T.near_tt[i].mask);
    printf("]}\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("topo")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-O1", "-std=c++17", "-fopenmp", "-I", CSRC, str(src), os.path.join(CSRC, "topology.cpp"),
                    "-o", str(exe)], check=True)
    return str(exe), d


def _library_topology(harness, cell):
    exe, d = harness
    path = d / ("%s.bin" % cell.name)
    with open(path, "wb") as f:
        np.array([len(cell.verts), len(cell.tets), cell.n_domains, cell.active_domain], np.int32).tofile(f)
        np.array([cell.period_a, cell.period_b], np.float64).tofile(f)
        np.ascontiguousarray(cell.verts, np.float64).tofile(f)
        np.ascontiguousarray(cell.tets, np.int32).tofile(f)
        np.ascontiguousarray(cell.tet_domain, np.int32).tofile(f)
    out = subprocess.run([exe, str(path)], check=True, capture_output=True, text=True).stdout
    t = json.loads(out)
    assert "error" not in t, t
    return t


CELLS = ["slab_3x3x1", "slab_4x3x2_jit", "plasmonic_tiny"]


@pytest.mark.parametrize("name", CELLS)
def test_topology_equals_the_oracle(harness, name):
    cell = cellgen.small_cells()[name]
    lib = _library_topology(harness, cell)
    ref = build_topology(cell)
    nt = len(cell.tets)
    assert lib["N"] == ref["n"]
    assert np.array_equal(np.array(lib["basis"]).reshape(nt, 4), ref["basis"])
    assert np.array_equal(np.array(lib["sgn"]).reshape(nt, 4), ref["sign"].astype(int))
    # lattice shift of a paired T- half: 1 = (a, 0, 0), 2 = (0, b, 0)
    code = np.zeros((nt, 4), int)
    code[np.abs(ref["shift"][:, :, 0]) > 0] = 1
    code[np.abs(ref["shift"][:, :, 1]) > 0] = 2
    assert np.array_equal(np.array(lib["shift"]).reshape(nt, 4), code)
    for k in ("kind", "tp", "ip"):
        assert np.array_equal(np.array(lib[k]), ref[k]), k
    full = ref["kind"] != 1   # the T- side exists (interior and Bloch-paired functions)
    assert np.array_equal(np.array(lib["tm"])[full], ref["tm"][full])
    assert np.array_equal(np.array(lib["im"])[full], ref["im"][full])
    # charge-carrying faces: half functions and faces where the material changes
    charge = (ref["kind"] == 1) | ((ref["kind"] != 1) & (cell.tet_domain[ref["tp"]] !=
                                                         cell.tet_domain[np.maximum(ref["tm"], 0)]))
    assert sorted(lib["cf"]) == sorted(np.nonzero(charge)[0].tolist())
    assert len(lib["hf"]) == int(np.sum(ref["kind"] == 1))


@pytest.mark.parametrize("name", CELLS)
def test_near_pairs_equal_the_oracle(harness, name):
    cell = cellgen.small_cells()[name]
    lib = _library_topology(harness, cell)
    P = cell.verts[cell.tets]
    cen = P.mean(axis=1)
    rad = np.max(np.linalg.norm(P - cen[:, None, :], axis=2), axis=1)
    near = _near_images(cen, rad, cen, rad, cell.period_a, cell.period_b)
    mask = (near * (1 << np.arange(9))).sum(axis=2)
    got = np.zeros_like(mask)
    for x, y, m in lib["near_tt"]:
        got[x, y] = m
    assert np.array_equal(got, mask)
    assert np.all(np.diag(mask) & (1 << 4))   # every tetrahedron is near itself in image (0, 0)
