// Host set-up of the Ewald series of one incidence (Sec. 2.2, Eq. (3)-(4)):
// the splitting parameter, the lattice images and Floquet orders inside the
// cut, and the Floquet-order rectangle and distinct decay constants of the
// FP32 tables.  Host code only (the library and the host-logic tests compile
// it).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/vie.h"
#include "ewald_tables.h"

namespace vie {

// Ewald parameters and tables of one incidence (Sec. 2.2, Eq. (3)-(4)): the
// splitting parameter, the lattice images and Floquet modes inside the cut of
// the FP64 (fp64) or FP32 series, the limit of the regularised image term, the
// rectangle of Floquet orders and the distinct decay constants of the FP32
// tables (z_extent = the largest |dz| they must cover).  `orders` (may be null)
// receives the propagating orders [n][4] (k_tx, k_ty, k_z, 1 for (0,0)).  The
// solver and the allocation-free entry point both build their tables here.
// Returns VIE_OK, VIE_RAYLEIGH_ANOMALY (a Floquet order at grazing) or
// VIE_EINVAL (a table would overflow), with *why set.
int build_ewald_tables(double a, double b, double k0, double kx, double ky, double z_extent, bool fp64,
                       EwaldTables &E, std::vector<double> *orders, const char **why, double split_mult) {
    std::memset(&E, 0, sizeof(E));
    if (orders) orders->clear();
    E.E = ewald_split(a, b, k0, !fp64, kx == 0.0 && ky == 0.0, split_mult);
    E.bb = k0 / (2.0 * E.E);
    E.a = a;
    E.b = b;
    E.xcut64 = FP64_XCUT;
    E.xcut32 = FP32_XCUT;
    const double xc = fp64 ? FP64_XCUT : (double)FP32_XCUT;
    const int mm = (int)std::ceil(xc / (E.E * a)) + 2, nn = (int)std::ceil(xc / (E.E * b)) + 2;
    int ni = 0;
    for (int m = -mm; m <= mm; ++m)
        for (int n = -nn; n <= nn; ++n) {
            const double dmin = std::hypot(std::max(std::abs(m) - 1, 0) * a, std::max(std::abs(n) - 1, 0) * b);
            const bool nearimg = std::abs(m) <= 1 && std::abs(n) <= 1;
            if (dmin * E.E > xc && !nearimg) continue;
            if (ni >= MAX_IMG) { *why = "period too small for the image table"; return VIE_EINVAL; }
            const double phs = kx * m * a + ky * n * b, f = std::exp(E.bb * E.bb) / (4.0 * M_PI);
            const double v[4] = {m * a, n * b, f * std::cos(phs), f * std::sin(phs)};
            for (int q = 0; q < 4; ++q) { E.img64[ni][q] = v[q]; E.img32[ni][q] = (float)v[q]; }
            if (nearimg) E.near_img[(m + 1) * 3 + (n + 1)] = ni;
            ++ni;
        }
    E.n_img = ni;
    const int pm = (int)std::ceil((2.0 * E.E * xc + std::fabs(kx)) * a / (2 * M_PI)) + 1;
    const int qm = (int)std::ceil((2.0 * E.E * xc + std::fabs(ky)) * b / (2 * M_PI)) + 1;
    int nm = 0;
    for (int p = -pm; p <= pm; ++p)
        for (int q = -qm; q <= qm; ++q) {
            const double ktx = kx + 2 * M_PI * p / a, kty = ky + 2 * M_PI * q / b;
            const double kt2 = ktx * ktx + kty * kty, g2 = kt2 - k0 * k0;
            if (std::fabs(g2) * std::max(a, b) * std::max(a, b) < 1e-10) {
                *why = "a Floquet order is at grazing (Rayleigh anomaly)";
                return VIE_RAYLEIGH_ANOMALY;
            }
            if (g2 < 0 && orders) orders->insert(orders->end(), {ktx, kty, std::sqrt(-g2), (p == 0 && q == 0) ? 1.0 : 0.0});
            if (std::sqrt(kt2) > 2.0 * E.E * xc + k0) continue;
            if (nm >= MAX_MODE) { *why = "too many Floquet modes for the table"; return VIE_EINVAL; }
            // gamma = sqrt(g2) (evanescent) or j sqrt(-g2) (propagating); 1/(4 a b gamma)
            const double gr = g2 >= 0 ? std::sqrt(g2) : 0.0, gi = g2 >= 0 ? 0.0 : std::sqrt(-g2);
            const double ir = gr / (4.0 * a * b * (gr * gr + gi * gi)), ii = -gi / (4.0 * a * b * (gr * gr + gi * gi));
            const double w8[8] = {ktx, kty, gr, gi, std::exp(-g2 / (4 * E.E * E.E)), ir, ii, 0};
            for (int c = 0; c < 8; ++c) { E.mode64[nm][c] = w8[c]; E.mode32[nm][c] = (float)w8[c]; }
            ++nm;
        }
    E.n_mode = nm;
    {   // erfi(b) by its series, for the limit R -> 0 of the regularised image term
        double term = E.bb, sum = E.bb;
        for (int n = 1; n < 200; ++n) {
            term *= E.bb * E.bb / n;
            const double add = term / (2 * n + 1);
            sum += add;
            if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
        }
        const double erfi = 2.0 / std::sqrt(M_PI) * sum;
        E.reg0_re = (E.E / (4 * M_PI)) * (2 * E.bb * erfi - 2.0 / std::sqrt(M_PI) * std::exp(E.bb * E.bb));
    }
    // tabulated FP32 path: the truncation of the FP32 series
    const double xc32 = FP32_XCUT, zr = std::max(z_extent, 1e-6) * (1.0 + 1e-6);
    E.xs_max = (float)(xc32 + 0.5);
    E.xs_inv_h = (float)(NSPAT / (xc32 + 0.5));
    E.z_max = (float)zr;
    E.z_inv_h = (float)(NZTAB / zr);
    E.e_mb2 = (float)std::exp(-E.bb * E.bb);
    E.Ef = (float)E.E;
    E.kx = (float)kx;
    E.ky = (float)ky;
    E.step_x = (float)(2 * M_PI / a);
    E.step_y = (float)(2 * M_PI / b);
    if (!mode_rect(kx, ky, a, b, 2.0 * E.E * xc32 + k0, E.p0, E.np, E.q0, E.nq)) {
        *why = "too many Floquet modes for the table";
        return VIE_EINVAL;
    }
    E.sym = (kx == 0.0 && ky == 0.0 && 2 * E.p0 + E.np == 1 && 2 * E.q0 + E.nq == 1) ? 1 : 0;
    int nt = 0;
    double g2s[MAX_MODE];
    for (int p = E.p0; p < E.p0 + E.np; ++p)
        for (int q = E.q0; q < E.q0 + E.nq; ++q) {
            const int idx = (p - E.p0) * E.nq + (q - E.q0);
            const double ktx = kx + 2 * M_PI * p / a, kty = ky + 2 * M_PI * q / b;
            const double kt2 = ktx * ktx + kty * kty;
            if (std::sqrt(kt2) > 2.0 * E.E * xc32 + k0) { E.rect_tab[idx] = -1; continue; }
            const double g2 = kt2 - k0 * k0;
            int found = -1;
            for (int j = 0; j < nt; ++j)
                if (std::fabs(g2s[j] - g2) <= 1e-12 * std::max(1e-6, std::fabs(g2))) { found = j; break; }
            if (found < 0) {
                found = nt++;
                g2s[found] = g2;
                const double gr = g2 >= 0 ? std::sqrt(g2) : 0.0, gi = g2 >= 0 ? 0.0 : std::sqrt(-g2);
                E.tab_gamma[found][0] = gr;
                E.tab_gamma[found][1] = gi;
                E.tab_ig[found][0] = gr / (4.0 * a * b * (gr * gr + gi * gi));
                E.tab_ig[found][1] = -gi / (4.0 * a * b * (gr * gr + gi * gi));
                E.tab_pre[found] = std::exp(-g2 / (4 * E.E * E.E));
            }
            // bit 16 marks a real decay constant (evanescent mode): its G is real
            E.rect_tab[idx] = found | (g2s[found] > 0 ? TAB_REAL : 0);
        }
    E.n_tab = nt;
    return VIE_OK;
}

}  // namespace vie
