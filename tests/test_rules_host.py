"""Host logic of the library's quadrature tables (CPU, no GPU): csrc/rules.cpp,
typed independently of the oracle's tables (oracle/quadrature.py).

A small C++ program compiled here against rules.cpp prints the library's
barycentric points and weights.  Each rule integrates every monomial
x^a y^b z^c of its degree exactly over the unit simplex (a! b! c! / (a+b+c+3)!
on the tetrahedron, a! b! / (a+b+2)! on the triangle) and is not exact one
degree higher; and the library's tables hold the oracle's points and weights,
point for point (the fill kernels and the oracle must integrate the same
discrete problem).
"""
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import quadrature as qr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05334_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
namespace vie {
void tet_rule5(double (*pts)[4], double *w);
void tri_rule5(double (*pts)[3], double *w);
void tet_rule2(double (*pts)[4], double *w);
void tri_rule2(double (*pts)[3], double *w);
}
template <int D> void dump(const char *name, int n, void (*f)(double (*)[D], double *), bool last) {
    double p[16][D], w[16];
    f(p, w);
    printf("\"%s\": [", name);
    for (int i = 0; i < n; ++i) {
        printf("%s[%.17g", i ? "," : "", w[i]);
        for (int k = 0; k < D; ++k) printf(",%.17g", p[i][k]);
        printf("]");
    }
    printf("]%s", last ? "" : ",");
}
int main() {
    printf("{");
    dump<4>("tet2", 4, vie::tet_rule2, false);
    dump<4>("tet5", 14, vie::tet_rule5, false);
    dump<3>("tri2", 3, vie::tri_rule2, false);
    dump<3>("tri5", 7, vie::tri_rule5, true);
    printf("}\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if cxx is None or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("no C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("rules")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, str(src), os.path.join(CSRC, "rules.cpp"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: np.array(v) for k, v in json.loads(out).items()}


def _monomials(dim, deg):
    if dim == 3:
        return [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)
                if a + b + c == deg]
    return [(a, b) for a in range(deg + 1) for b in range(deg + 1 - a) if a + b == deg]


def _max_error(rule, dim, deg):
    w, bary = rule[:, 0], rule[:, 1:]
    x = bary[:, 1:]                     # Cartesian coordinates on the unit simplex
    worst = 0.0
    for e in _monomials(dim, deg):
        exact = math.prod(math.factorial(k) for k in e) / math.factorial(sum(e) + dim) * math.factorial(dim)
        got = np.sum(w * np.prod(x ** np.array(e), axis=1))
        worst = max(worst, abs(got - exact))
    return worst


@pytest.mark.parametrize("name,dim,deg", [("tet2", 3, 2), ("tet5", 3, 5), ("tri2", 2, 2), ("tri5", 2, 5)])
def test_library_rules_are_exact_to_their_degree(rules, name, dim, deg):
    rule = rules[name]
    assert abs(rule[:, 0].sum() - 1.0) < 1e-15
    assert np.allclose(rule[:, 1:].sum(axis=1), 1.0, atol=1e-15)
    for k in range(deg + 1):
        assert _max_error(rule, dim, k) < 1e-15, (name, k)
    assert _max_error(rule, dim, deg + 1) > 1e-6   # and no further


@pytest.mark.parametrize("name,oracle_rule", [("tet2", qr.tet_deg2), ("tet5", qr.tet_deg5), ("tri2", qr.tri_deg2),
                                              ("tri5", qr.tri_deg5)])
def test_library_rules_hold_the_oracles_points(rules, name, oracle_rule):
    bary, w = oracle_rule()
    lib = rules[name]
    assert len(lib) == len(w)
    # the same point set with the same weights (matched point for point)
    for row in lib:
        d = np.max(np.abs(bary - row[1:]), axis=1)
        k = int(np.argmin(d))
        assert d[k] < 1e-14 and abs(w[k] - row[0]) < 1e-15
