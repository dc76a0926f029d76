"""Host logic of the FP32 Ewald tables (CPU, no GPU): the Floquet-order maps of
the fill's short forms.

A small C++ program, compiled here with the host compiler against the
library's own host sources (csrc/ewald_tables.cpp, csrc/ewald_params.h), builds
the tables of one incidence and prints the order rectangle with its table per
entry, and the maps the short forms read (make_ewald_f32): the normal-incidence
quadrant (sq_off, sq_im), the oblique rectangle or its k_y = 0 fold (ob_off,
ob_im).  With random values of every table (real for the real decay
constants), the sums the short forms take must equal the plain sum over the
rectangle,
    sum_pq G_pq exp(-j k_t,pq . rho),
at d and, through g(-d) = conj(g(d)) + 2j conj(T), at -d.  A wrong index,
weight, fold or table offset fails it.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05334_gb300", "csrc")
NZTAB = 256

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "ewald_tables.h"
using namespace vie;
int main(int argc, char **argv) {
    const double a = atof(argv[1]), b = atof(argv[2]), lam = atof(argv[3]), th = atof(argv[4]), ph = atof(argv[5]);
    const double k0 = 6.283185307179586 / lam;
    static EwaldTables E;
    const char *why = "";
    int rc = build_ewald_tables(a, b, k0, k0 * sin(th) * cos(ph), k0 * sin(th) * sin(ph), 100.0, false, E, nullptr, &why);
    if (rc) { printf("{\"rc\": %d}\n", rc); return 0; }
    static EwaldF32 F;
    F = make_ewald_f32(E);
    printf("{\"rc\": 0, \"n_tab\": %d, \"sym\": %d, \"p0\": %d, \"np\": %d, \"q0\": %d, \"nq\": %d, \"n_img\": %d,",
           E.n_tab, E.sym, E.p0, E.np, E.q0, E.nq, E.n_img);
    printf("\"kx\": %.17g, \"ky\": %.17g, \"sx\": %.17g, \"sy\": %.17g, \"ob_kx0\": %.17g, \"ob_ky0\": %.17g,",
           (double)F.kx, (double)F.ky, (double)F.step_x, (double)F.step_y, (double)F.ob_kx0, (double)F.ob_ky0);
    printf("\"rect\": [");
    for (int i = 0; i < E.np * E.nq; ++i) printf("%s%d", i ? "," : "", E.rect_tab[i]);
    printf("], \"sq_pq\": %d, \"sq_im\": %d, \"sq_off\": [", F.sq_pq, F.sq_im);
    for (int p = 0; p <= SQ_MAX; ++p)
        for (int q = 0; q <= SQ_MAX; ++q) printf("%s%d", p + q ? "," : "", F.sq_off[p][q]);
    printf("], \"ob_nr\": %d, \"ob_nq1\": %d, \"ob_off\": [", F.ob_nr, F.ob_nq1);
    for (int i = 0; i < OB_MAX; ++i)
        for (int j = 0; j < OB_MAX; ++j) printf("%s%d", i + j ? "," : "", F.ob_off[i][j]);
    printf("], \"ob_im\": [");
    for (int i = 0; i < OB_MAX; ++i)
        for (int j = 0; j < OB_MAX; ++j) printf("%s%d", i + j ? "," : "", F.ob_im[i][j]);
    printf("]}\n");
    return 0;
}
"""

CASES = [(200.0, 200.0, 500.0, 0.0, 0.0), (150.0, 120.0, 430.0, 0.0, 0.0),      # normal incidence
         (200.0, 200.0, 500.0, 0.5, 0.0), (400.0, 400.0, 650.0, 0.9, 0.0),      # k_y = 0 fold
         (300.0, 240.0, 420.0, 1.2, 0.0),
         (180.0, 150.0, 430.0, 0.6, 0.3), (400.0, 400.0, 650.0, 0.9, 1.1)]     # full rectangle


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("ewald")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "ewald_tables.cpp"),
                    "-o", str(exe)], check=True)
    return str(exe)


def _tables(exe, case):
    out = subprocess.run([exe] + ["%r" % v for v in case], check=True, capture_output=True, text=True).stdout
    t = json.loads(out)
    assert t["rc"] == 0
    return t


def _values(t, rng):
    """Random table values: real where the decay constant is real (TAB_REAL)."""
    G = rng.standard_normal(t["n_tab"]) + 1j * rng.standard_normal(t["n_tab"])
    real = np.zeros(t["n_tab"], bool)
    for code in t["rect"]:
        if code >= 0 and code & (1 << 16):
            real[code & 0xFFFF] = True
    G[real] = G[real].real
    return G


def _full(t, G, dx, dy):
    # the rectangle's first order as the kernels receive it (FP32), the same
    # parameter the short forms start from; its rounding is checked apart
    kx0 = t["ob_kx0"] if not t["sym"] else t["kx"] + t["p0"] * t["sx"]
    ky0 = t["ob_ky0"] if not t["sym"] else t["ky"] + t["q0"] * t["sy"]
    s = 0j
    for i in range(t["np"]):
        for j in range(t["nq"]):
            code = t["rect"][i * t["nq"] + j]
            if code < 0:
                continue
            ktx = kx0 + i * t["sx"]
            kty = ky0 + j * t["sy"]
            s += G[code & 0xFFFF] * np.exp(-1j * (ktx * dx + kty * dy))
    return s


def _re(t, G, off):   # real part of the table at rtab offset `off` (the zero table after the n_tab tables)
    k = off // NZTAB
    return 0.0 if k == t["n_tab"] else G[k].real


def _im(t, G, off):   # imaginary part of the table whose imaginary copy sits at `off`
    return G[off // NZTAB - t["n_tab"] - 1].imag


@pytest.mark.parametrize("case", CASES)
def test_short_forms_reproduce_the_order_sum(harness, case):
    t = _tables(harness, case)
    rng = np.random.default_rng(7)
    normal, fold = case[3] == 0.0, case[3] != 0.0 and case[4] == 0.0
    if normal:
        assert t["sym"] == 1 and t["sq_pq"] > 0
    else:
        assert t["ob_nr"] > 0 and (t["ob_nq1"] > 0) == fold
    if not normal:   # the FP32 first order against k_par + 2 pi p0 / a in FP64
        assert abs(t["ob_kx0"] - (t["kx"] + t["p0"] * t["sx"])) <= 2.0 ** -23 * (abs(t["ob_kx0"]) + t["sx"])
        assert abs(t["ob_ky0"] - (t["ky"] + t["q0"] * t["sy"])) <= 2.0 ** -23 * (abs(t["ob_ky0"]) + t["sy"])
    sq = np.array(t["sq_off"]).reshape(5, 5)
    oo, oi = np.array(t["ob_off"]).reshape(8, 8), np.array(t["ob_im"]).reshape(8, 8)
    for _ in range(3):
        G = _values(t, rng)
        for dx, dy in rng.uniform(-1, 1, (6, 2)) * np.array([case[0], case[1]]):
            ref, ref_m = _full(t, G, dx, dy), _full(t, G, -dx, -dy)
            if normal:
                PQ = t["sq_pq"]
                D = lambda k, s, x: 1.0 if k == 0 else 2 * np.cos(k * s * x)
                g = sum(D(p, t["sx"], dx) * D(q, t["sy"], dy) * _re(t, G, sq[p, q])
                        for p in range(PQ + 1) for q in range(PQ + 1)) + 1j * _im(t, G, t["sq_im"])
                gm = g   # g_p(-d) = g_p(d) at normal incidence
            else:
                S = T = 0j
                for i in range(t["ob_nr"]):
                    X = np.exp(-1j * (t["ob_kx0"] + i * t["sx"]) * dx)
                    if fold:
                        cols = [(q, 1.0 if q == 0 else 2 * np.cos(q * t["sy"] * dy)) for q in range(t["ob_nq1"])]
                    else:
                        cols = [(j, np.exp(-1j * (t["ob_ky0"] + j * t["sy"]) * dy)) for j in range(t["ob_nr"])]
                    for j, w in cols:
                        S += X * w * _re(t, G, oo[i, j])
                        if oi[i, j] >= 0:
                            T += X * w * _im(t, G, oi[i, j])
                g = S + 1j * T
                gm = np.conj(g) + 2j * np.conj(T)
            scale = np.sum(np.abs(G)) * 4
            assert abs(g - ref) < 1e-11 * scale, (case, dx, dy, g, ref)
            assert abs(gm - ref_m) < 1e-11 * scale, (case, dx, dy, gm, ref_m)


def test_a_planted_fold_error_fails(harness):
    """Dropping the factor 2 of the folded orders q > 0 breaks the identity."""
    case = (200.0, 200.0, 500.0, 0.5, 0.0)
    t = _tables(harness, case)
    G = _values(t, np.random.default_rng(1))
    oo = np.array(t["ob_off"]).reshape(8, 8)
    dx, dy = 37.0, -61.0
    S = 0j
    for i in range(t["ob_nr"]):
        X = np.exp(-1j * (t["ob_kx0"] + i * t["sx"]) * dx)
        for q in range(t["ob_nq1"]):
            S += X * (1.0 if q == 0 else np.cos(q * t["sy"] * dy)) * _re(t, G, oo[i, q])
    ref = _full(t, G.real.astype(complex), dx, dy)
    assert abs(S - ref) > 1e-3 * np.sum(np.abs(G))


def _rc(exe, case):
    out = subprocess.run([exe] + ["%r" % v for v in case], check=True, capture_output=True, text=True).stdout
    return json.loads(out)["rc"]


@pytest.mark.parametrize("case,moved", [((400.0, 400.0, 400.0, 0.0, 0.0), (400.0, 400.0, 400.01, 0.0, 0.0)),
                                        # order (-1, 0) grazing: sin(theta) = lambda / a - 1
                                        ((200.0, 200.0, 300.0, float(np.arcsin(0.5)), 0.0),
                                         (200.0, 200.0, 300.01, float(np.arcsin(0.5)), 0.0))])
def test_rayleigh_anomaly_is_detected(harness, case, moved):
    """A Floquet order exactly at grazing (gamma_pq = 0: the spectral series is
    singular) returns VIE_RAYLEIGH_ANOMALY (-4); 0.01 nm away the tables build."""
    assert _rc(harness, case) == -4
    assert _rc(harness, moved) == 0
