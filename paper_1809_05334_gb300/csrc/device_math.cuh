// Device math for the fill: complex helpers, Faddeeva function, Ewald-summed
// 2D periodic Green's function (Eq. (3)-(4), Sec. 2.2) and closed-form
// integrals of 1/R and R over triangles and tetrahedra.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include "ewald_params.h"

namespace vie {

template <typename T> struct cx { T re, im; };

template <typename T> __device__ __forceinline__ cx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }
template <typename T> __device__ __forceinline__ cx<T> crecip(cx<T> a) {
    // 1/a with scaling to avoid overflow of |a|^2
    T s = fmax(fabs(a.re), fabs(a.im));
    T ar = a.re / s, ai = a.im / s;
    T d = s * (ar * ar + ai * ai);
    return {ar / d, -ai / d};
}
template <typename T> __device__ __forceinline__ void cfma(cx<T> &acc, T s, cx<T> a) {
    acc.re = fma(s, a.re, acc.re);
    acc.im = fma(s, a.im, acc.im);
}

// ---------------------------------------------------------------------------
// Faddeeva function w(z) = exp(-z^2) erfc(-j z) for Im z >= 0 by Weideman's
// rational expansion (SIAM J. Numer. Anal. 31, 1994):
//   w(z) = 2 p(Zz) / (L - j z)^2 + 1 / (sqrt(pi) (L - j z)),  Zz = (L + j z)/(L - j z),
// p(Zz) = sum_{n=1}^{NW} a_n Zz^(n-1), a_n the Fourier coefficients of
// (L^2 + t^2) exp(-t^2) in the variable theta, t = L tan(theta/2).  The
// coefficients are computed on the host in FP64 and stored here.
constexpr int NW64 = 40;
constexpr int NW32 = 20;
struct WeidemanTables {
    double a64[NW64 + 1];
    float a32[NW32 + 1];
    double L64;
    float L32;
};
static __constant__ WeidemanTables c_weid;   // filled by upload_constants() (fill.cu)

template <typename T> struct WTraits;
template <> struct WTraits<double> {
    static constexpr int N = NW64;
    __device__ static double L() { return c_weid.L64; }
    __device__ static double a(int n) { return c_weid.a64[n]; }
};
template <> struct WTraits<float> {
    static constexpr int N = NW32;
    __device__ static float L() { return c_weid.L32; }
    __device__ static float a(int n) { return c_weid.a32[n]; }
};

template <typename T> __device__ __forceinline__ T rsqrt_pi() { return T(0.56418958354775628695); }

// erfcx(u) = exp(u^2) erfc(u) = w(j u), complex u with Re u >= 0.
template <typename T> __device__ __forceinline__ cx<T> erfcx_c(cx<T> u) {
    const T L = WTraits<T>::L();
    // z = j u: L - j z = L + u, L + j z = L - u
    cx<T> dm = {L + u.re, u.im};
    cx<T> dp = {L - u.re, -u.im};
    cx<T> inv = crecip(dm);
    cx<T> Z = dp * inv;
    cx<T> p = {WTraits<T>::a(WTraits<T>::N), T(0)};
#pragma unroll
    for (int n = WTraits<T>::N - 1; n >= 1; --n) {
        p = p * Z;
        p.re += WTraits<T>::a(n);
    }
    cx<T> t = inv * p;
    t.re = fma(T(2), t.re, rsqrt_pi<T>());
    t.im = T(2) * t.im;
    return inv * t;
}

// erfcx(x) for real x >= 0 (the expansion at z = j x stays real).
template <typename T> __device__ __forceinline__ T erfcx_r(T x) {
    const T L = WTraits<T>::L();
    T inv = T(1) / (L + x);
    T Z = (L - x) * inv;
    T p = WTraits<T>::a(WTraits<T>::N);
#pragma unroll
    for (int n = WTraits<T>::N - 1; n >= 1; --n) p = fma(p, Z, WTraits<T>::a(n));
    return inv * fma(T(2) * p, inv, rsqrt_pi<T>());
}

// Ewald parameter blocks (EwaldTables, EwaldF32): ewald_params.h

template <typename T> struct ETraits;
template <> struct ETraits<double> {
    __device__ static const double *img(const EwaldTables *ew, int i) { return ew->img64[i]; }
    __device__ static const double *mode(const EwaldTables *ew, int i) { return ew->mode64[i]; }
    __device__ static double xcut(const EwaldTables *ew) { return ew->xcut64; }
};
template <> struct ETraits<float> {
    __device__ static const float *img(const EwaldTables *ew, int i) { return ew->img32[i]; }
    __device__ static const float *mode(const EwaldTables *ew, int i) { return ew->mode32[i]; }
    __device__ static float xcut(const EwaldTables *ew) { return ew->xcut32; }
};

// g_p(d) for an in-cell difference d; images whose bit is set in `sub`
// (9-bit mask over (m,n) in {-1,0,1}^2) have their static part
// phase/(4 pi R) removed.
template <typename T>
__device__ cx<T> green_p(T dx, T dy, T dz, unsigned sub, const EwaldTables *__restrict__ ew) {
    const T E = T(ew->E);
    const T bb = T(ew->bb);
    const T xc = ETraits<T>::xcut(ew) + T(0.5);
    cx<T> acc = {T(0), T(0)};
    // spectral series
    const T z = fabs(dz);
    const T ez = exp(-(z * E) * (z * E));
    const T inv2E = T(0.5) / E;
    for (int i = 0; i < ew->n_mode; ++i) {
        const T *md = ETraits<T>::mode(ew, i);
        T s, c;
        sincos(-(md[0] * dx + md[1] * dy), &s, &c);
        cx<T> ph = {c, s};
        cx<T> br;
        if (md[3] == T(0)) {                       // evanescent: gamma real
            T g = md[2];
            T pre = md[4] * ez;
            T t1 = pre * erfcx_r(g * inv2E + z * E);
            T u = g * inv2E - z * E;
            T t2 = (u >= T(0)) ? pre * erfcx_r(u) : T(2) * exp(-g * z) - pre * erfcx_r(-u);
            br = {t1 + t2, T(0)};
        } else {                                    // propagating: gamma = j gi
            T gi = md[3];
            T pre = md[4] * ez;
            cx<T> e1 = erfcx_c(cx<T>{z * E, gi * inv2E});
            // erfcx(zE - j gi/2E) = conj(e1)
            T sg, cg;
            sincos(gi * z, &sg, &cg);
            // t1 = pre e1; t2 = 2 e^{-j gi z} - pre conj(e1)
            br = {pre * e1.re + T(2) * cg - pre * e1.re, pre * e1.im - T(2) * sg + pre * e1.im};
        }
        cx<T> ig = {md[5], md[6]};
        acc = acc + ph * (br * ig);
    }
    // spatial series
    for (int i = 0; i < ew->n_img; ++i) {
        const T *im = ETraits<T>::img(ew, i);
        T x = dx + im[0], y = dy + im[1];
        T R2 = x * x + y * y + dz * dz;
        T R = sqrt(R2);
        if (R * E > xc) continue;
        bool regular = false;
        if (sub) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (((sub >> k) & 1u) && ew->near_img[k] == i) regular = true;
        }
        if (regular && R * E < T(1e-6)) {
            // continuous limit at R = 0 of (image term - static term):
            // reg0 = (E/4pi)[2 b erfi(b) - (2/sqrt pi) exp(b^2)]; the table
            // phase carries exp(b^2)/(4 pi), undone here
            cx<T> ph = {im[2], im[3]};
            T unscale = T(4.0 * CUDART_PI) * exp(-bb * bb) * T(ew->reg0_re);
            acc = acc + unscale * ph;
            continue;
        }
        T val = exp(-R2 * E * E) * erfcx_c(cx<T>{R * E, bb}).re / R;
        if (regular) val -= exp(-bb * bb) / R;   // static part phase/(4 pi R) in table units
        cx<T> ph = {im[2], im[3]};
        acc = acc + val * ph;
    }
    return acc;
}

// FP32 g_p from per-request tables (same series, same truncation as green_p):
//  spectral: sum_pq exp(-j k_t,pq . rho) G_pq(|z|), G = [e^{gz}erfc(..) + e^{-gz}erfc(..)]/(4ab g)
//            tabulated per distinct gamma; phases by recurrence over the (p, q) rectangle
//  spatial:  phase_mn exp(b^2)/(4 pi) F(R E)/R with F(x) = exp(-x^2) Re erfcx(x + j b);
//            the regularised near image uses (F(RE) - F(0))/R, formed without
//            cancellation in the first interval
// stab: [NSPAT][4] cubic coefficients (shared memory); ztab: [n_tab][NZTAB][4] complex
// With PAIR the same pass also returns gm = g_p(-d): the spectral terms of -d
// carry the conjugate phases, and the spatial term of image -R_mn at -d is the
// table value of image R_mn at d with the conjugate lattice phase (the image
// list and the near-image masks are symmetric under (m,n) -> (-m,-n)).
// rtab (may be null): the real parts of the tables as one float4 per
// interval; used for the tables flagged TAB_REAL (their imaginary parts are 0)
// SYM (normal incidence, k_par = 0, mode rectangle symmetric about (0, 0)):
// G_pq = G_-p-q, so the orders pair up into 2 G_pq cos(k_t,pq . rho) over the
// half plane p > 0 or (p = 0, q > 0), plus G_00; g_p is even in d, so gm = gp.
template <bool PAIR, bool SYM = false>
__device__ __forceinline__ void green_tab_impl(float dx, float dy, float dz, unsigned sub, const float *stab,
                                               const float2 *__restrict__ ztab, const EwaldF32 &ew,
                                               cx<float> &gp, cx<float> &gm,
                                               const float4 *__restrict__ rtab = nullptr,
                                               unsigned long long imask = ~0ull) {
    cx<float> acc = {0.f, 0.f}, acc2 = {0.f, 0.f};
    const float z = fabsf(dz);
    float zu = fminf(z * ew.z_inv_h, float(NZTAB));
    int iz = min((int)zu, NZTAB - 1);
    const float u = zu - iz;
    // G of the mode table `code` at |z| (real tables: one 16-byte load)
    auto table = [&](int code, float &gr, float &gi) {
        const int tb = code & TAB_INDEX;
        if (rtab && (code & TAB_REAL)) {
            const float4 c = __ldg(rtab + (size_t)tb * NZTAB + iz);
            gr = fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
            gi = 0.f;
            return true;
        }
        const float2 *cf = ztab + ((size_t)tb * NZTAB + iz) * 4;
        const float2 c0 = __ldg(cf), c1 = __ldg(cf + 1), c2 = __ldg(cf + 2), c3 = __ldg(cf + 3);
        gr = fmaf(u, fmaf(u, fmaf(u, c3.x, c2.x), c1.x), c0.x);
        gi = fmaf(u, fmaf(u, fmaf(u, c3.y, c2.y), c1.y), c0.y);
        return false;
    };
    const int np = ew.np, nq = ew.nq;
    float s, c;
    if constexpr (SYM) {
        if (np > 0) {
            // G_pq depends on |k_t,pq| alone, so it is even in p and in q separately:
            // sum_pq G_pq exp(-j k_t,pq . rho) = sum_{p,q >= 0} w_p w_q G_pq cos(k_p x) cos(k_q y)
            // (w_0 = 1, w_>0 = 2; the sine products cancel), one table evaluation per
            // order of the quadrant; D_q = 2 cos(k_q y) and D_p by Chebyshev recurrence
            const int P = (np - 1) / 2, Q = (nq - 1) / 2;
            const float d1x = 2.f * cospif(ew.step_x * dx * 0.31830988618f);
            const float d1y = 2.f * cospif(ew.step_y * dy * 0.31830988618f);
            float dp_prev = 2.f, dp = d1x;   // D_0, D_1 in x
            for (int p = 0; p <= P; ++p) {
                const int row = (P + p) * nq + Q;
                float rr = 0.f, ri = 0.f, gr, gi;
                const int c0 = ew.rect_tab[row];
                if (c0 >= 0) { table(c0, rr, ri); }
                float dq_prev = 2.f, dq = d1y;   // D_0, D_1 in y
                for (int q = 1; q <= Q; ++q) {
                    const int code = ew.rect_tab[row + q];
                    if (code >= 0) {
                        if (table(code, gr, gi)) rr = fmaf(dq, gr, rr);
                        else { rr = fmaf(dq, gr, rr); ri = fmaf(dq, gi, ri); }
                    }
                    const float dn = fmaf(d1y, dq, -dq_prev);
                    dq_prev = dq;
                    dq = dn;
                }
                const float wp = p == 0 ? 1.f : dp;
                acc.re = fmaf(wp, rr, acc.re);
                acc.im = fmaf(wp, ri, acc.im);
                if (p >= 1) {   // D_{p+1} = d1x D_p - D_{p-1}
                    const float dn = fmaf(d1x, dp, -dp_prev);
                    dp_prev = dp;
                    dp = dn;
                }
            }
        }
    } else {
        sincospif(-(ew.kx + ew.p0 * ew.step_x) * dx * 0.31830988618f, &s, &c);
        cx<float> ex = {c, s};
        sincospif(-ew.step_x * dx * 0.31830988618f, &s, &c);
        const cx<float> sx = {c, s};
        sincospif(-(ew.ky + ew.q0 * ew.step_y) * dy * 0.31830988618f, &s, &c);
        const cx<float> ey0 = {c, s};
        sincospif(-ew.step_y * dy * 0.31830988618f, &s, &c);
        const cx<float> sy = {c, s};
        for (int p = 0; p < np; ++p) {
            cx<float> inner = {0.f, 0.f}, inner2 = {0.f, 0.f};
            cx<float> ey = ey0;
            for (int q = 0; q < nq; ++q) {
                const int code = ew.rect_tab[p * nq + q];
                if (code >= 0) {
                    float gr, gi;
                    if (table(code, gr, gi)) {   // real G: real products
                        inner.re = fmaf(ey.re, gr, inner.re);
                        inner.im = fmaf(ey.im, gr, inner.im);
                        if (PAIR) {
                            inner2.re = fmaf(ey.re, gr, inner2.re);
                            inner2.im = fmaf(-ey.im, gr, inner2.im);
                        }
                    } else {
                        const cx<float> g = {gr, gi};
                        inner = inner + ey * g;
                        if (PAIR) inner2 = inner2 + cconj(ey) * g;
                    }
                }
                ey = ey * sy;
            }
            acc = acc + ex * inner;
            if (PAIR) acc2 = acc2 + cconj(ex) * inner2;
            ex = ex * sx;
        }
    }
    const float E = ew.Ef;
    const float xmax = ew.xs_max, ih = ew.xs_inv_h;
    const float r2max = (xmax / E) * (xmax / E) * 1.0001f;   // loose: the exact test follows
    float sv = 0.f;   // SYM: the sum of the image values before their common factor
    auto image = [&](int i) {
        const float *im = ew.img[i];
        const float x = dx + im[0], y = dy + im[1];
        const float R2 = x * x + y * y + dz * dz;
        if (R2 > r2max) return;            // outside the cut: skip before the square root
        const float rinv = R2 > 0.f ? rsqrtf(R2) : 0.f;   // R = 0 only on a regularised image (no 1/R)
        const float R = R2 * rinv;
        const float xr = R * E;
        if (xr > xmax) return;
        bool regular = false;
        if (sub) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (((sub >> k) & 1u) && ew.near_img[k] == i) regular = true;
        }
        const float xu = xr * ih;
        const int ix = min((int)xu, NSPAT - 1);
        const float v = xu - ix;
        const float4 cs = *reinterpret_cast<const float4 *>(stab + 4 * ix);   // one 16-byte load
        float val;
        if (regular) {
            if (ix == 0)   // (F(x) - F(0))/R = E (c1 + v (c2 + v c3)) / h
                val = E * ih * fmaf(v, fmaf(v, cs.w, cs.z), cs.y);
            else
                val = (fmaf(v, fmaf(v, fmaf(v, cs.w, cs.z), cs.y), cs.x) - ew.e_mb2) * rinv;
        } else {
            val = fmaf(v, fmaf(v, fmaf(v, cs.w, cs.z), cs.y), cs.x) * rinv;
        }
        if (SYM) {   // k_par = 0: every image carries the same real phase factor
            sv += val;
            return;
        }
        acc.re = fmaf(val, im[2], acc.re);
        acc.im = fmaf(val, im[3], acc.im);
        if (PAIR) {
            acc2.re = fmaf(val, im[2], acc2.re);
            acc2.im = fmaf(-val, im[3], acc2.im);
        }
    };
    // images 0..63 as the caller's mask selects them (it leaves out only images
    // beyond the cut), the rest one by one
    if (ew.n_img < 64) imask &= (1ull << ew.n_img) - 1ull;
    for (unsigned long long mk = imask; mk; mk &= mk - 1ull) image(__ffsll((long long)mk) - 1);
    for (int i = 64; i < ew.n_img; ++i) image(i);
    if (SYM) acc.re = fmaf(ew.img[0][2], sv, acc.re);
    gp = acc;
    gm = SYM ? acc : acc2;
}

// Images (of the first 64) that can lie inside the spatial cut for some
// displacement within `rad` of (cx, cy, cz): every image whose shifted centre
// distance exceeds the cut radius + rad is left out.
__device__ __forceinline__ unsigned long long image_mask(const EwaldF32 &ew, float cx, float cy, float cz,
                                                         float rad) {
    const float rc = ew.xs_max / ew.Ef * 1.0001f + rad * 1.0001f + 1e-6f * (fabsf(cx) + fabsf(cy) + fabsf(cz));
    const float rc2 = rc * rc;
    const int n = min(ew.n_img, 64);
    unsigned long long m = 0ull;
    for (int i = 0; i < n; ++i) {
        const float x = cx + ew.img[i][0], y = cy + ew.img[i][1];
        if (x * x + y * y + cz * cz <= rc2) m |= 1ull << i;
    }
    return m;
}

__device__ __forceinline__ cx<float> green_tab(float dx, float dy, float dz, unsigned sub, const float *stab,
                                               const float2 *__restrict__ ztab, const EwaldF32 &ew) {
    cx<float> g, unused;
    green_tab_impl<false>(dx, dy, dz, sub, stab, ztab, ew, g, unused);
    return g;
}

// ---------------------------------------------------------------------------
// Closed forms (divergence theorem, polygonal / polyhedral sources):
//  triangle: int 1/R = sum_i t_i ln[(R+_i + s+_i)/(R-_i + s-_i)]
//                      - |h| sum_i [atan(t s+/(R0^2+|h|R+)) - atan(t s-/(R0^2+|h|R-))]
//            int R   = ( h^2 int 1/R + 1/2 sum_i t_i (s+R+ - s-R- + R0^2 ln(..)) ) / 3
//  tetrahedron: int 1/R = 1/2 sum_f d_f int_f 1/R,  int (r'-r)/R = sum_f n_f int_f R
template <typename T>
__host__ __device__ __forceinline__ T log_rs(T R, T s, T R0sq) {
    // ln(R + s) without cancellation for s < 0: R + s = R0^2 / (R - s)
    return (s >= T(0)) ? log(R + s) : log(R0sq) - log(R - s);
}

template <typename T>
__host__ __device__ void tri_integrals(const T r[3], const T *v, T &inv, T &rint, bool want_r) {
    T e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    T e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    T n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    T nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    T h = n[0] * (r[0] - v[0]) + n[1] * (r[1] - v[1]) + n[2] * (r[2] - v[2]);
    T ah = fabs(h);
    T scale = fmax(sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]),
                   sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
    T tiny = (sizeof(T) == 8 ? T(1e-13) : T(1e-6)) * scale;
    T slog = 0, satan = 0, sr = 0;
    T Rv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T d0 = r[0] - v[3 * j], d1 = r[1] - v[3 * j + 1], d2 = r[2] - v[3 * j + 2];
        Rv[j] = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int ja = e, jb = (e + 1) % 3;
        const T *pa = v + 3 * ja, *pb = v + 3 * jb;
        T L[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        T ll = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
        L[0] /= ll; L[1] /= ll; L[2] /= ll;
        // in-plane outward normal u = l x n
        T u[3] = {L[1] * n[2] - L[2] * n[1], L[2] * n[0] - L[0] * n[2], L[0] * n[1] - L[1] * n[0]};
        T t = u[0] * (pa[0] - r[0]) + u[1] * (pa[1] - r[1]) + u[2] * (pa[2] - r[2]);
        T sm = L[0] * (pa[0] - r[0]) + L[1] * (pa[1] - r[1]) + L[2] * (pa[2] - r[2]);
        T sp = sm + ll;
        T Rm = Rv[ja], Rp = Rv[jb];
        T R0sq = t * t + h * h;
        if (fabs(t) > tiny) {
            T lr = log_rs(Rp, sp, R0sq) - log_rs(Rm, sm, R0sq);
            slog += t * lr;
            if (want_r) sr += t * (sp * Rp - sm * Rm + R0sq * lr);
            if (ah > tiny) satan += atan2(t * sp, R0sq + ah * Rp) - atan2(t * sm, R0sq + ah * Rm);
        }
    }
    inv = slog - ah * satan;
    rint = want_r ? (h * h * inv + T(0.5) * sr) / T(3) : T(0);
}

template <typename T>
__host__ __device__ void tet_integrals(const T r[3], const T *tv, T &inv, T vec[3], bool want_vec) {
    inv = 0;
    vec[0] = vec[1] = vec[2] = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T f[9];
        int k = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j != i) {
                f[3 * k] = tv[3 * j]; f[3 * k + 1] = tv[3 * j + 1]; f[3 * k + 2] = tv[3 * j + 2];
                ++k;
            }
        T e1[3] = {f[3] - f[0], f[4] - f[1], f[5] - f[2]};
        T e2[3] = {f[6] - f[0], f[7] - f[1], f[8] - f[2]};
        T n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        T nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        T o = n[0] * (f[0] - tv[3 * i]) + n[1] * (f[1] - tv[3 * i + 1]) + n[2] * (f[2] - tv[3 * i + 2]);
        T sg = (o >= T(0)) ? T(1) / nn : T(-1) / nn;   // outward unit normal
        n[0] *= sg; n[1] *= sg; n[2] *= sg;
        T d = n[0] * (f[0] - r[0]) + n[1] * (f[1] - r[1]) + n[2] * (f[2] - r[2]);
        T fi, fr;
        tri_integrals<T>(r, f, fi, fr, want_vec);
        inv += T(0.5) * d * fi;
        if (want_vec) {
            vec[0] += n[0] * fr; vec[1] += n[1] * fr; vec[2] += n[2] * fr;
        }
    }
}

// The same tetrahedron closed forms with the per-edge quantities shared by the
// two faces of each edge: 4 vertex distances, 6 edge logarithms
// ln[(R_b + s_b)/(R_a + s_a)] (orientation independent) and one combined
// arctangent per (face, edge): atan2(t s_b, R0^2+|h|R_b) - atan2(t s_a, R0^2+|h|R_a)
// = atan2(y_b x_a - x_b y_a, x_a x_b + y_a y_b) (both angles lie in (-pi/2, pi/2)).
// tv holds the vertices relative to the observer (the observer is the origin).
__host__ __device__ inline void tet_integrals_shared(const double *tv, double &inv, double vec[3]) {
    constexpr int EA[6] = {0, 0, 0, 1, 1, 2}, EB[6] = {1, 2, 3, 2, 3, 3};
    // edges of face f (opposite vertex f) in the face's vertex order, and the face's third vertex per edge
    constexpr int FE[4][3] = {{3, 5, 4}, {1, 5, 2}, {0, 4, 2}, {0, 3, 1}};
    constexpr int FC[4][3] = {{3, 1, 2}, {3, 0, 2}, {3, 0, 1}, {2, 0, 1}};
    double Rv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) Rv[v] = sqrt(tv[3 * v] * tv[3 * v] + tv[3 * v + 1] * tv[3 * v + 1] + tv[3 * v + 2] * tv[3 * v + 2]);
    double scale = 0;
    double L[6], lh[6][3], sa[6], sb[6], sR[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const double *pa = tv + 3 * EA[e], *pb = tv + 3 * EB[e];
        double d[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        scale = fmax(scale, len);
        for (int q = 0; q < 3; ++q) lh[e][q] = d[q] / len;
        sa[e] = lh[e][0] * pa[0] + lh[e][1] * pa[1] + lh[e][2] * pa[2];   // along the edge, observer at 0
        sb[e] = sa[e] + len;
        const double c0 = pa[1] * lh[e][2] - pa[2] * lh[e][1], c1 = pa[2] * lh[e][0] - pa[0] * lh[e][2],
                     c2 = pa[0] * lh[e][1] - pa[1] * lh[e][0];
        const double d2 = c0 * c0 + c1 * c1 + c2 * c2;   // squared distance to the edge line
        const double Ra = Rv[EA[e]], Rb = Rv[EB[e]];
        // ln[(Rb + sb)/(Ra + sa)] with R + s = d2/(R - s) for s < 0
        double lv;
        if (sa[e] >= 0) lv = log((Rb + sb[e]) / (Ra + sa[e]));
        else if (sb[e] <= 0) lv = log((Ra - sa[e]) / (Rb - sb[e]));
        else lv = (d2 > 0) ? log((Rb + sb[e]) * (Ra - sa[e]) / d2) : 0.0;
        L[e] = lv;
        sR[e] = sb[e] * Rb - sa[e] * Ra;
    }
    const double tiny = 1e-13 * scale;
    inv = 0;
    vec[0] = vec[1] = vec[2] = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        // face opposite vertex f; outward normal
        const int fv[3] = {f == 0 ? 1 : 0, f <= 1 ? 2 : 1, f <= 2 ? 3 : 2};
        const double *p0 = tv + 3 * fv[0], *p1 = tv + 3 * fv[1], *p2 = tv + 3 * fv[2];
        const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const double o = n[0] * (p0[0] - tv[3 * f]) + n[1] * (p0[1] - tv[3 * f + 1]) + n[2] * (p0[2] - tv[3 * f + 2]);
        const double sg = (o >= 0) ? 1.0 / nn : -1.0 / nn;
        n[0] *= sg; n[1] *= sg; n[2] *= sg;
        const double dfc = n[0] * p0[0] + n[1] * p0[1] + n[2] * p0[2];   // n.(p0 - r): signed distance
        const double h = -dfc, ah = fabs(h);
        double slog = 0, satan = 0, sr = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int e = FE[f][q];
            // in-plane outward normal of the edge: u = l x n, its sign fixed by
            // pointing away from the face's third vertex
            const double *pc = tv + 3 * FC[f][q];
            double u[3] = {lh[e][1] * n[2] - lh[e][2] * n[1], lh[e][2] * n[0] - lh[e][0] * n[2],
                           lh[e][0] * n[1] - lh[e][1] * n[0]};
            const double *pa = tv + 3 * EA[e];
            if (u[0] * (pa[0] - pc[0]) + u[1] * (pa[1] - pc[1]) + u[2] * (pa[2] - pc[2]) < 0) {
                u[0] = -u[0]; u[1] = -u[1]; u[2] = -u[2];
            }
            const double t = u[0] * pa[0] + u[1] * pa[1] + u[2] * pa[2];
            if (fabs(t) <= tiny) continue;
            const double R0sq = t * t + h * h;
            slog += t * L[e];
            sr += t * (sR[e] + R0sq * L[e]);
            if (ah > tiny) {
                const double xa = R0sq + ah * Rv[EA[e]], ya = t * sa[e];
                const double xb = R0sq + ah * Rv[EB[e]], yb = t * sb[e];
                satan += atan2(yb * xa - xb * ya, xa * xb + ya * yb);
            }
        }
        const double fi = slog - ah * satan;
        const double fr = (h * h * fi + 0.5 * sr) / 3.0;
        inv += 0.5 * dfc * fi;
        vec[0] += n[0] * fr; vec[1] += n[1] * fr; vec[2] += n[2] * fr;
    }
}

}  // namespace vie
