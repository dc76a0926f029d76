// Ewald parameters of one incidence, shared by host (set-up) and device code.
#pragma once
#include <algorithm>
#include <cmath>

namespace vie {

// Ewald parameters of one incidence.  Spatial series (images R_mn):
//   phase_mn exp(b^2 - R^2 E^2) Re erfcx(R E + j b) / (4 pi R),  b = k/(2E)
// Spectral series (Floquet modes k_t = k_par + 2 pi (p/a, q/b)):
//   exp(-j k_t.rho) / (4 a b gamma) [e^{gamma z} erfc(gamma/2E + zE) + e^{-gamma z} erfc(gamma/2E - zE)]
constexpr int MAX_IMG = 160;
constexpr int MAX_MODE = 160;
struct EwaldTables {
    // per image: (m a, n b, Re, Im) of exp(j k_par.R_mn) exp(b^2)/(4 pi)
    double img64[MAX_IMG][4];
    float img32[MAX_IMG][4];
    // per mode: (k_tx, k_ty, gamma_re, gamma_im, exp(-gamma^2/4E^2), Re, Im of 1/(4ab gamma))
    double mode64[MAX_MODE][8];
    float mode32[MAX_MODE][8];
    int n_img, n_mode;
    int near_img[9];        // image-table index of (m,n) = (k/3-1, k%3-1)
    double E, bb, a, b, xcut64;
    float xcut32;
    double reg0_re;          // limit R->0 of (image term - static term), without the phase
    // tabulated FP32 evaluation (see green_tab): spatial kernel F(x) on [0, xs_max],
    // spectral G_g(z) per distinct gamma on [0, z_max], piecewise cubic Hermite
    float xs_max, xs_inv_h, z_max, z_inv_h, e_mb2, Ef;
    float kx, ky, step_x, step_y;   // k_t,pq = (kx + p step_x, ky + q step_y)
    int p0, np, q0, nq, n_tab;       // the smallest rectangle p0 <= p < p0 + np, q0 <= q < q0 + nq
                                     // holding every mode inside the cut
    int sym;                         // 1: k_par = 0 and the rectangle is symmetric about (0, 0)
    int rect_tab[MAX_MODE];  // table of rectangle entry (p-p0) nq + (q-q0) (| TAB_REAL if its G
                             // is real), -1 outside the cut
    double tab_gamma[MAX_MODE][2];   // gamma of each table
    double tab_ig[MAX_MODE][2];      // 1/(4ab gamma) of each table
    double tab_pre[MAX_MODE];        // exp(-gamma^2/4E^2)
};
constexpr int TAB_REAL = 1 << 16;   // flag in rect_tab: the table's G is real (real decay constant)
constexpr int TAB_INDEX = TAB_REAL - 1;
constexpr double FP64_XCUT = 6.0;   // Ewald truncation of the FP64 series: exp(-36) ~ 2e-16
constexpr float FP32_XCUT = 4.2f;   // of the FP32 series and tables: exp(-17.6) ~ 2e-8
constexpr int NSPAT = 512;    // spatial intervals
constexpr int NZTAB = 256;    // spectral intervals
// Normal incidence short form (k_par = 0, at most 32 lattice images, every
// Floquet order of the cut within |p|, |q| <= SQ_MAX, (0, 0) the only
// propagating order): the order quadrant p, q >= 0 unrolled at compile time,
// each entry naming its real spectral table (orders outside the cut name a
// table of zeros), and the imaginary part of the (0, 0) table beside it.  The
// real-part buffer `rtab` holds n_tab real tables, the zero table, then the
// n_tab imaginary tables, NZTAB float4 each.
constexpr int SQ_MAX = 4;
// Oblique incidence short form (at most 64 lattice images, an order rectangle
// of at most OB_MAX x OB_MAX): the rectangle unrolled at compile time, each
// entry naming its real table (a zero table outside the cut) and, for a
// propagating order, its imaginary table.
constexpr int OB_MAX = 8;
// EwaldTables lives in device global memory, one copy per request in flight, so
// independent solves can run concurrently.  The part of it that the FP32
// tabulated evaluation reads in its inner loops travels as a kernel parameter
// (EwaldF32 below, ~3.3 KB, __grid_constant__): warp-uniform reads of it are
// served by the constant cache and every launch carries its own copy.
struct EwaldF32 {
    float img[MAX_IMG][4];   // = EwaldTables::img32
    int rect_tab[MAX_MODE];
    int near_img[9];
    int n_img, p0, np, q0, nq, sym;
    float xs_max, xs_inv_h, z_inv_h, e_mb2, Ef, kx, ky, step_x, step_y;
    float Eih;                            // E * xs_inv_h: table abscissa per unit distance
    int sq_pq;                            // max(P, Q) >= 1 of the short form; 0 where it does not apply
    int sq_off[SQ_MAX + 1][SQ_MAX + 1];   // order (p, q): offset of its real table in rtab (float4 units)
    int sq_im;                            // offset of the (0, 0) order's imaginary table in rtab
    int ob_nr;                            // rectangle side (4, 6 or 8) of the oblique short form; 0: not used
    int ob_nq1;                           // k_y = 0 (orders even in q): q = 0 .. ob_nq1 - 1 (3 or 5) kept; 0: all q
    float ob_kx0, ob_ky0;                 // k_par + 2 pi (p0 / a, q0 / b): the rectangle's first order
    int ob_off[OB_MAX][OB_MAX];           // rectangle entry (i, j): offset of its real table in rtab
    int ob_im[OB_MAX][OB_MAX];            // offset of its imaginary table (propagating order), else -1
};
// Ewald splitting parameter: sqrt(pi / ab) balances the spatial and spectral
// series, bounded below by k0/6 (b = k0 / 2E <= 3 keeps exp(b^2) moderate).  The
// tabulated FP32 path makes the spectral terms cheaper than the images (table
// lookups against square roots and table interpolation per image), which
// moves the balance to a larger E: fewer lattice images inside the same erfc
// cut.  The FP64 series keeps the balanced value.
#ifndef VIE_SPLIT_NORMAL
#define VIE_SPLIT_NORMAL 1.5    // FP32 tables, normal incidence
#endif
#ifndef VIE_SPLIT_OBLIQUE
#define VIE_SPLIT_OBLIQUE 1.0   // FP32 tables, oblique incidence
#endif
// mult > 0 replaces the FP32 multiplier (the autotuner's candidates).
inline double ewald_split(double a, double b, double k0, bool fp32, bool normal, double mult = 0.0) {
    const double e = std::max(std::sqrt(3.141592653589793 / (a * b)), k0 / 6.0);
    if (!fp32) return e;
    return (mult > 0.0 ? mult : (normal ? VIE_SPLIT_NORMAL : VIE_SPLIT_OBLIQUE)) * e;
}

// The smallest rectangle of Floquet orders (p, q) holding every mode with
// |k_t,pq| <= kmax, k_t,pq = (kx + 2 pi p / a, ky + 2 pi q / b); np = nq = 0
// when there is none.  False when the rectangle has more than MAX_MODE entries.
inline bool mode_rect(double kx, double ky, double a, double b, double kmax, int &p0, int &np, int &q0, int &nq) {
    const double tp = 6.283185307179586;
    const int P = (int)((kmax + (kx < 0 ? -kx : kx)) * a / tp) + 2;
    const int Q = (int)((kmax + (ky < 0 ? -ky : ky)) * b / tp) + 2;
    int plo = P + 1, phi = -P - 1, qlo = Q + 1, qhi = -Q - 1;
    for (int p = -P; p <= P; ++p)
        for (int q = -Q; q <= Q; ++q) {
            const double ktx = kx + tp * p / a, kty = ky + tp * q / b;
            if (ktx * ktx + kty * kty > kmax * kmax * (1.0 + 1e-12)) continue;   // loose: callers test each mode
            plo = p < plo ? p : plo; phi = p > phi ? p : phi;
            qlo = q < qlo ? q : qlo; qhi = q > qhi ? q : qhi;
        }
    if (phi < plo) { p0 = q0 = np = nq = 0; return true; }
    p0 = plo; np = phi - plo + 1; q0 = qlo; nq = qhi - qlo + 1;
    return np * nq <= MAX_MODE;
}

inline EwaldF32 make_ewald_f32(const EwaldTables &t) {
    EwaldF32 f{};
    for (int i = 0; i < MAX_IMG; ++i)
        for (int k = 0; k < 4; ++k) f.img[i][k] = t.img32[i][k];
    for (int i = 0; i < MAX_MODE; ++i) f.rect_tab[i] = t.rect_tab[i];
    for (int k = 0; k < 9; ++k) f.near_img[k] = t.near_img[k];
    f.n_img = t.n_img; f.p0 = t.p0; f.np = t.np; f.q0 = t.q0; f.nq = t.nq; f.sym = t.sym;
    f.xs_max = t.xs_max; f.xs_inv_h = t.xs_inv_h; f.z_inv_h = t.z_inv_h; f.e_mb2 = t.e_mb2; f.Ef = t.Ef;
    f.kx = t.kx; f.ky = t.ky; f.step_x = t.step_x; f.step_y = t.step_y;
    f.Eih = t.Ef * t.xs_inv_h;
    f.sq_pq = 0;
    const int zero = t.n_tab * NZTAB;   // the zero table
    for (int p = 0; p <= SQ_MAX; ++p)
        for (int q = 0; q <= SQ_MAX; ++q) f.sq_off[p][q] = zero;
    f.sq_im = zero;
    // the rectangle of a symmetric request is -P..P x -Q..Q; its quadrant p, q >= 0
    if (t.sym && t.np > 0 && t.nq > 0 && t.n_img <= 32) {
        const int P = (t.np - 1) / 2, Q = (t.nq - 1) / 2;
        bool ok = P <= SQ_MAX && Q <= SQ_MAX;
        for (int p = 0; ok && p <= P; ++p)
            for (int q = 0; ok && q <= Q; ++q) {
                const int code = t.rect_tab[(P + p) * t.nq + (Q + q)];
                if (code < 0) continue;
                const int tb = code & TAB_INDEX;
                f.sq_off[p][q] = tb * NZTAB;
                if (!(code & TAB_REAL)) {
                    if (p == 0 && q == 0) f.sq_im = (t.n_tab + 1 + tb) * NZTAB;
                    else ok = false;   // another propagating order: the general form
                }
            }
        if (ok) f.sq_pq = P > Q ? (P > 1 ? P : 1) : (Q > 1 ? Q : 1);
    }
    f.ob_nr = 0;
    f.ob_nq1 = 0;
    f.ob_kx0 = (float)(t.kx + t.p0 * (double)t.step_x);
    f.ob_ky0 = (float)(t.ky + t.q0 * (double)t.step_y);
    for (int i = 0; i < OB_MAX; ++i)
        for (int j = 0; j < OB_MAX; ++j) { f.ob_off[i][j] = zero; f.ob_im[i][j] = -1; }
    // k_y = 0 and the rectangle symmetric in q: G_pq = G_p,-q, so the q sum folds
    // onto q >= 0 with the weights 1, 2 cos(q s_y dy)
    const int Qh = (t.nq - 1) / 2;
    if (!t.sym && t.ky == 0.f && t.np > 0 && t.nq > 0 && 2 * t.q0 + t.nq == 1 && t.np <= OB_MAX && Qh + 1 <= 5 &&
        t.n_img <= 64) {
        for (int i = 0; i < t.np; ++i)
            for (int q = 0; q <= Qh; ++q) {
                const int code = t.rect_tab[i * t.nq + (Qh + q)];
                if (code < 0) continue;
                const int tb = code & TAB_INDEX;
                f.ob_off[i][q] = tb * NZTAB;
                if (!(code & TAB_REAL)) f.ob_im[i][q] = (t.n_tab + 1 + tb) * NZTAB;
            }
        f.ob_nr = t.np <= 6 ? 6 : 8;
        f.ob_nq1 = Qh + 1 <= 3 ? 3 : 5;
    } else if (!t.sym && t.np > 0 && t.nq > 0 && t.np <= OB_MAX && t.nq <= OB_MAX && t.n_img <= 64) {
        for (int i = 0; i < t.np; ++i)
            for (int j = 0; j < t.nq; ++j) {
                const int code = t.rect_tab[i * t.nq + j];
                if (code < 0) continue;
                const int tb = code & TAB_INDEX;
                f.ob_off[i][j] = tb * NZTAB;
                if (!(code & TAB_REAL)) f.ob_im[i][j] = (t.n_tab + 1 + tb) * NZTAB;
            }
        const int nr = t.np > t.nq ? t.np : t.nq;
        f.ob_nr = nr <= 4 ? 4 : (nr <= 6 ? 6 : 8);
    }
    return f;
}


}  // namespace vie
