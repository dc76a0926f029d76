// Matrix fill of the periodic SWG VIE (Eq. (2)) on the GPU.
//
// Z_mn = int f_m.f_n/eps_r - k0^2 int int f_m . kappa' f_n g_p + int int div f_m q_n g_p
// (lengths in nm, scaled by eps0), with q_n = div'(kappa f_n) including the
// surface charge (kappa- - kappa+) on face n and the surface term -delta of a
// half test function.  Every Z entry is a sum over element pairs (tetrahedra
// and charge-carrying faces); each element pair is integrated once and its
// contributions are added into Z with atomics.
//
//  far pairs : degree-2 product rules (4 points per tetrahedron, 3 per
//              triangle), g_p by the Ewald series, precision T (FP32 or FP64).
//  near pairs: the static part exp(j k_par.R)/(4 pi R) of every near image is
//              integrated in closed form over one element at the degree-5
//              points of the other, averaged over both orders, plus the
//              remainder of g_p with the degree-2 product rules.  The closed
//              forms run in FP64 when the elements touch, in T otherwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "device_math.cuh"
#include "fill.h"

namespace vie {

__constant__ double c_w5tet[14];
__constant__ double c_w5tri[7];

// ---------------------------------------------------------------------------
// host set-up of the constant tables
// ---------------------------------------------------------------------------
static void weideman_coeffs(int N, double &L, std::vector<double> &a) {
    L = std::sqrt(N / std::sqrt(2.0));
    const int M = 16 * N;
    a.assign(N + 1, 0.0);
    for (int k = 0; k < M; ++k) {
        double th = -M_PI + (k + 0.5) * 2.0 * M_PI / M;
        double t = L * std::tan(0.5 * th);
        double F = std::exp(-t * t) * (L * L + t * t);
        for (int n = 0; n <= N; ++n) a[n] += F * std::cos(n * th) / M;
    }
}

cudaError_t upload_constants() {
    WeidemanTables w{};
    std::vector<double> a;
    double L;
    weideman_coeffs(NW64, L, a);
    w.L64 = L;
    for (int n = 0; n <= NW64; ++n) w.a64[n] = a[n];
    weideman_coeffs(NW32, L, a);
    w.L32 = (float)L;
    for (int n = 0; n <= NW32; ++n) w.a32[n] = (float)a[n];
    cudaError_t e = cudaMemcpyToSymbol(c_weid, &w, sizeof(w));
    if (e != cudaSuccess) return e;
    double w5t[14], w5f[7];
    tet_rule5(nullptr, w5t);
    tri_rule5(nullptr, w5f);
    e = cudaMemcpyToSymbol(c_w5tet, w5t, sizeof(w5t));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_w5tri, w5f, sizeof(w5f));
}

cudaError_t upload_ewald(EwaldTables *dev, const EwaldTables &t, cudaStream_t st) {
    return cudaMemcpyAsync(dev, &t, sizeof(t), cudaMemcpyHostToDevice, st);
}

// ---------------------------------------------------------------------------
// per-request tables of the FP32 path (built in FP64 from the Ewald series):
// cubic Hermite coefficients per interval, in the local variable u in [0, 1)
// ---------------------------------------------------------------------------
__device__ void hermite(double f0, double d0, double f1, double d1, double h, double c[4]) {
    c[0] = f0;
    c[1] = h * d0;
    c[2] = 3.0 * (f1 - f0) - h * (2.0 * d0 + d1);
    c[3] = 2.0 * (f0 - f1) + h * (d0 + d1);
}

__device__ void spatial_node(const EwaldTables *ew, double x, double &F, double &dF) {
    // F(x) = exp(-x^2) Re erfcx(x + j b),  F'(x) = -exp(-x^2) (2 b Im erfcx(x + j b) + 2/sqrt(pi))
    const double b = ew->bb;
    cx<double> w = erfcx_c<double>(cx<double>{x, b});
    const double g = exp(-x * x);
    F = g * w.re;
    dF = -g * (2.0 * b * w.im + 2.0 * rsqrt_pi<double>());
}

__device__ void spectral_node(const EwaldTables *ew, int tb, double z, cx<double> &G, cx<double> &dG) {
    // G(z) = (t1 + t2)/(4ab gamma), G'(z) = gamma (t1 - t2)/(4ab gamma)
    const double E = ew->E;
    const cx<double> g = {ew->tab_gamma[tb][0], ew->tab_gamma[tb][1]};
    const cx<double> ig = {ew->tab_ig[tb][0], ew->tab_ig[tb][1]};
    const double pre = ew->tab_pre[tb] * exp(-(z * E) * (z * E));
    cx<double> t1, t2;
    if (g.im == 0.0) {
        const double gr = g.re;
        t1 = {pre * erfcx_r<double>(gr / (2 * E) + z * E), 0.0};
        const double u = gr / (2 * E) - z * E;
        t2 = {(u >= 0) ? pre * erfcx_r<double>(u) : 2.0 * exp(-gr * z) - pre * erfcx_r<double>(-u), 0.0};
    } else {
        const double gi = g.im;
        cx<double> e1 = erfcx_c<double>(cx<double>{z * E, gi / (2 * E)});
        double sg, cg;
        sincos(gi * z, &sg, &cg);
        t1 = pre * e1;
        t2 = cx<double>{2.0 * cg - pre * e1.re, -2.0 * sg + pre * e1.im};
    }
    G = (t1 + t2) * ig;
    dG = (g * (t1 - t2)) * ig;
}

__global__ void k_build_tables(const EwaldTables *__restrict__ ew, float *stab, float2 *ztab, int n_tab,
                               float4 *rtab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NSPAT) {
        const double h = double(ew->xs_max) / NSPAT;
        double F0, D0, F1, D1, c[4];
        spatial_node(ew, i * h, F0, D0);
        spatial_node(ew, (i + 1) * h, F1, D1);
        hermite(F0, D0, F1, D1, h, c);
        for (int k = 0; k < 4; ++k) stab[4 * i + k] = float(c[k]);
        return;
    }
    const int j = i - NSPAT;
    const int tb = j / NZTAB, iz = j % NZTAB;
    if (rtab && tb == n_tab) {   // the zero table after the real tables
        rtab[(size_t)n_tab * NZTAB + iz] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    if (tb >= n_tab) return;
    const double h = double(ew->z_max) / NZTAB;
    cx<double> G0, D0, G1, D1;
    spectral_node(ew, tb, iz * h, G0, D0);
    spectral_node(ew, tb, (iz + 1) * h, G1, D1);
    double cr[4], ci[4];
    hermite(G0.re, D0.re, G1.re, D1.re, h, cr);
    hermite(G0.im, D0.im, G1.im, D1.im, h, ci);
    for (int k = 0; k < 4; ++k) ztab[((size_t)tb * NZTAB + iz) * 4 + k] = make_float2(float(cr[k]), float(ci[k]));
    // the real and the imaginary parts apart, 16 bytes per interval each
    if (rtab) {
        rtab[(size_t)tb * NZTAB + iz] = make_float4(float(cr[0]), float(cr[1]), float(cr[2]), float(cr[3]));
        rtab[(size_t)(n_tab + 1 + tb) * NZTAB + iz] = make_float4(float(ci[0]), float(ci[1]), float(ci[2]), float(ci[3]));
    }
}

cudaError_t launch_build_tables(const EwaldTables *ew, float *stab, float2 *ztab, int n_tab, cudaStream_t st,
                                float4 *rtab) {
    const int n = NSPAT + (n_tab + (rtab ? 1 : 0)) * NZTAB;
    k_build_tables<<<(n + 127) / 128, 128, 0, st>>>(ew, stab, ztab, n_tab, rtab); ++g_launches;
    return cudaGetLastError();
}

// near-image mask of the reversed pair: image (m,n) <-> (-m,-n), i.e. bit k <-> bit 8-k
__device__ __forceinline__ unsigned mirror_mask(unsigned sub) {
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if ((sub >> k) & 1u) r |= 1u << (8 - k);
    return r;
}

// g_p for the fill kernels: FP64 by the Ewald series, FP32 from the tables
template <typename T> struct Green;
// eval2 returns g_p(d) and g_p(-d) (the same near-image mask applies to both)
template <> struct Green<double> {
    template <bool SYM = false>
    __device__ static cx<double> eval(double dx, double dy, double dz, unsigned sub, const float *, const float2 *,
                                      const EwaldTables *ew, const EwaldF32 &, const float4 * = nullptr,
                                      unsigned long long = ~0ull) {
        return green_p<double>(dx, dy, dz, sub, ew);
    }
    template <bool SYM = false>
    __device__ static void eval2(double dx, double dy, double dz, unsigned sub, const float *, const float2 *,
                                 const EwaldTables *ew, const EwaldF32 &, cx<double> &gp, cx<double> &gm,
                                 const float4 * = nullptr, unsigned long long = ~0ull) {
        gp = green_p<double>(dx, dy, dz, sub, ew);
        gm = green_p<double>(-dx, -dy, -dz, mirror_mask(sub), ew);
    }
};
template <> struct Green<float> {
    template <bool SYM = false>
    __device__ static cx<float> eval(float dx, float dy, float dz, unsigned sub, const float *stab,
                                     const float2 *ztab, const EwaldTables *, const EwaldF32 &ef,
                                     const float4 *rtab = nullptr, unsigned long long imask = ~0ull) {
        cx<float> g, unused;
        green_tab_impl<false, SYM>(dx, dy, dz, sub, stab, ztab, ef, g, unused, rtab, imask);
        return g;
    }
    template <bool SYM = false>
    __device__ static void eval2(float dx, float dy, float dz, unsigned sub, const float *stab, const float2 *ztab,
                                 const EwaldTables *, const EwaldF32 &ef, cx<float> &gp, cx<float> &gm,
                                 const float4 *rtab = nullptr, unsigned long long imask = ~0ull) {
        green_tab_impl<true, SYM>(dx, dy, dz, sub, stab, ztab, ef, gp, gm, rtab, imask);
    }
};

// stage the spatial table in shared memory (FP32 path only)
template <typename T>
__device__ __forceinline__ const float *stage_stab(const DevReq &q, float *smem) {
    if (sizeof(T) == 8) return nullptr;
    for (int i = threadIdx.x; i < 4 * NSPAT; i += blockDim.x) smem[i] = q.stab[i];
    __syncthreads();
    return smem;
}

template <typename T> constexpr size_t stab_bytes() { return sizeof(T) == 4 ? 4 * NSPAT * sizeof(float) : 0; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <typename T> struct Mom {
    cx<T> S, A[3], B[3], C;
    __device__ void zero() {
        S = {0, 0}; C = {0, 0};
        for (int d = 0; d < 3; ++d) { A[d] = {0, 0}; B[d] = {0, 0}; }
    }
};

template <typename T>
__device__ __forceinline__ void atomic_add_c(T *Z, size_t idx, cx<T> v) {
    atomicAdd(Z + 2 * idx, v.re);
    atomicAdd(Z + 2 * idx + 1, v.im);
}

__device__ __forceinline__ cx<double> ld2(const double *p) { return {p[0], p[1]}; }

// scatter the 16 face-pair contributions of one tetrahedron pair
template <typename T>
__device__ void scatter_tt(const DevMesh &m, const DevReq &q, T *Z, size_t N, int t, int s,
                           const Mom<T> &mo) {
    const T *ft = m.far<T>(t);
    const T *fs = m.far<T>(s);
    const T k2 = T(q.k0 * q.k0);
    cx<T> kap = {T(q.kap[2 * s]), T(q.kap[2 * s + 1])};
    cx<T> kS = kap * mo.S;
    for (int i = 0; i < 4; ++i) {
        const T wi[3] = {ft[15 + 3 * i], ft[16 + 3 * i], ft[17 + 3 * i]};
        const T ci = T(q.coef[4 * t + i]);
        cx<T> wti = {T(q.wt[2 * (4 * t + i)]), T(q.wt[2 * (4 * t + i) + 1])};
        size_t row = (size_t)q.row[4 * t + i];
        cx<T> wB = wi[0] * mo.B[0] + wi[1] * mo.B[1] + wi[2] * mo.B[2];
        for (int j = 0; j < 4; ++j) {
            const T wj[3] = {fs[15 + 3 * j], fs[16 + 3 * j], fs[17 + 3 * j]};
            const T cj = T(q.coef[4 * s + j]);
            cx<T> wsj = {T(q.wt[2 * (4 * s + j)]), -T(q.wt[2 * (4 * s + j) + 1])};
            size_t col = (size_t)q.row[4 * s + j];
            cx<T> M = mo.C - (wj[0] * mo.A[0] + wj[1] * mo.A[1] + wj[2] * mo.A[2]) - wB +
                      (wi[0] * wj[0] + wi[1] * wj[1] + wi[2] * wj[2]) * mo.S;
            cx<T> val = (-k2 * ci * cj) * (kap * M) + (T(9) * ci * cj) * kS;
            val = (wti * wsj) * val;
            atomic_add_c(Z, row * N + col, val);
        }
    }
}

// ---------------------------------------------------------------------------
// all tetrahedron pairs: degree-2 product rule of g_p; for the near images of a
// pair the static part is removed here and integrated by k_pr_tt / k_touch_tt
// ---------------------------------------------------------------------------
// Each unordered pair {t, s} (s >= t) is evaluated once: one pass over the 16
// point pairs gives g_p(x_a - y_b) for the block (t, s) and g_p(y_b - x_a) for
// the block (s, t) (the reversed pair's moments swap the roles of the offsets).
// SYM: normal incidence (the tabulated path's symmetric mode sum, gm = gp).
// Eight CTAs per SM for the FP32 tables (64 registers; the kernel is
// issue-bound and its fixed-latency waits need the extra warps), six for FP64.
template <typename T, bool SYM>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 6)
    k_far_tt(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N) {
    extern __shared__ float smem_tab[];
    const int t = blockIdx.y;
    if ((int)(blockIdx.x * blockDim.x + blockDim.x) <= t) return;   // the whole block is below the diagonal
    const float *stab = stage_stab<T>(q, smem_tab);
    const int s0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s0 < m.nt && s0 >= t;   // lanes off the pair range stay until the warp's image mask is formed
    const int s = live ? s0 : t;
    // near images of this pair: their static part is integrated separately
    const unsigned sub = m.mk_tt[(size_t)t * m.nt + s];
    const T *ft = m.far<T>(t);
    const T *fs = m.far<T>(s);
    Mom<T> mo, mr;   // blocks (t, s) and (s, t)
    mo.zero();
    mr.zero();
    const T wgt = ft[27] * fs[27];
    // images that can reach the cut from some point pair of {t, s}, decided once
    // for the 16 point pairs (FP32 tables only): every point pair lies within
    // rt + rs of the centroid offset
    unsigned long long imask = ~0ull;
    if (sizeof(T) == 4) {
        float rt = 0.f, rs = 0.f;
        for (int a = 0; a < 4; ++a) {
            const float ux = float(ft[3 * a] - ft[12]), uy = float(ft[3 * a + 1] - ft[13]), uz = float(ft[3 * a + 2] - ft[14]);
            const float vx = float(fs[3 * a] - fs[12]), vy = float(fs[3 * a + 1] - fs[13]), vz = float(fs[3 * a + 2] - fs[14]);
            rt = fmaxf(rt, sqrtf(ux * ux + uy * uy + uz * uz));
            rs = fmaxf(rs, sqrtf(vx * vx + vy * vy + vz * vz));
        }
        imask = image_mask(q.ef, float(ft[12] - fs[12]), float(ft[13] - fs[13]), float(ft[14] - fs[14]), rt + rs);
        // one image list for the whole warp (the union of its pairs' lists): the
        // image index is warp-uniform, so the image loop runs on the uniform
        // datapath and its table entries are broadcast loads
        if (!live) imask = 0ull;
        const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)imask);
        const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(imask >> 32));
        imask = ((unsigned long long)hi << 32) | lo;
    }
    if (!live) return;
    for (int a = 0; a < 4; ++a) {
        const T xa[3] = {ft[3 * a], ft[3 * a + 1], ft[3 * a + 2]};
        const T ra[3] = {xa[0] - ft[12], xa[1] - ft[13], xa[2] - ft[14]};
        for (int b = 0; b < 4; ++b) {
            const T yb[3] = {fs[3 * b], fs[3 * b + 1], fs[3 * b + 2]};
            const T rb[3] = {yb[0] - fs[12], yb[1] - fs[13], yb[2] - fs[14]};
            cx<T> g, gr;
            Green<T>::template eval2<SYM>(xa[0] - yb[0], xa[1] - yb[1], xa[2] - yb[2], sub, stab, q.ztab, q.ew,
                                          q.ef, g, gr, q.rtab, imask);
            g = wgt * g;
            const T rr = ra[0] * rb[0] + ra[1] * rb[1] + ra[2] * rb[2];
            mo.S = mo.S + g;
            for (int d = 0; d < 3; ++d) {
                mo.A[d] = mo.A[d] + ra[d] * g;
                mo.B[d] = mo.B[d] + rb[d] * g;
            }
            mo.C = mo.C + rr * g;
            if (!SYM) {
                gr = wgt * gr;
                mr.S = mr.S + gr;
                for (int d = 0; d < 3; ++d) {
                    mr.A[d] = mr.A[d] + rb[d] * gr;
                    mr.B[d] = mr.B[d] + ra[d] * gr;
                }
                mr.C = mr.C + rr * gr;
            }
        }
    }
    if (SYM) {   // g_p(-d) = g_p(d): the reversed pair's moments swap A and B
        mr.S = mo.S;
        mr.C = mo.C;
        for (int d = 0; d < 3; ++d) { mr.A[d] = mo.B[d]; mr.B[d] = mo.A[d]; }
    }
    scatter_tt<T>(m, q, Z, N, t, s, mo);
    if (s != t) scatter_tt<T>(m, q, Z, N, s, t, mr);
}

// Interval min(floor(x), n - 1) of a table of n intervals and the offset v in
// it (v in [0, 1]; x >= 0 clamped to n first, so x = n gives interval n - 1 at
// v = 1), without float <-> int conversions (they run on the quarter-rate
// pipe): x + 2^23 rounded down holds floor(x) in its low mantissa bits.
// Callers test the unclamped x against the table's range where it can exceed it.
__device__ __forceinline__ int table_index(float x, int n, float &v) {
    const float xc = fminf(x, float(n));
    const float t = __fadd_rd(xc, 8388608.f);
    v = xc - fminf(t - 8388608.f, float(n - 1));
    return min(__float_as_int(t) - 0x4B000000, n - 1);
}

// ---------------------------------------------------------------------------
// Normal incidence (k_par = 0), short form of the tabulated evaluation.  The
// same sum as green_tab_impl's symmetric form,
//   g_p = sum_{p,q >= 0} w_p w_q G_pq(|z|) cos(p th_x) cos(q th_y)
//         + exp(b^2)/(4 pi) sum_i F(R_i E) / R_i,   th = 2 pi (dx / a, dy / b),
// (w_0 = 1, w_k = 2; the static part 1/R removed on the images in regm), with
// the order quadrant unrolled at compile time (every order of the cut has
// |p|, |q| <= PQ; entries outside the cut are skipped on a uniform branch), the
// images from a 32-bit warp-uniform mask, and d1 = (2 cos th_x, 2 cos th_y)
// supplied by the caller; D_k = 2 cos(k th) by the Chebyshev recurrence
// D_k = d1 D_{k-1} - D_{k-2}, D_0 = 2.  REG: some lane of the warp has images
// whose static part is removed (else R > 0 on every image of every lane).
// ---------------------------------------------------------------------------
template <bool REG>
__device__ __forceinline__ float image_term(int i, float dx, float dy, float dz2, unsigned regm, const float4 *stab4,
                                            const EwaldF32 &ef) {
    const float x = dx + ef.img[i][0], y = dy + ef.img[i][1];
    const float R2 = fmaf(x, x, fmaf(y, y, dz2));
    float rinv = rsqrtf(R2);
    if (REG) rinv = R2 > 0.f ? rinv : 0.f;   // R = 0 only on an image whose static part is removed
    const float xu = R2 * rinv * ef.Eih;
    float v;
    const int ix = table_index(xu, NSPAT, v);
    const float4 c = stab4[ix];
    const float q1 = fmaf(v, fmaf(v, c.w, c.z), c.y);
    float val = fmaf(v, q1, c.x) * rinv;
    if (REG && ((regm >> i) & 1u))   // (F(x) - F(0)) / R; near R = 0 from the first interval's slope
        val = ix == 0 ? ef.Eih * q1 : fmaf(-ef.e_mb2, rinv, val);
    return xu <= float(NSPAT) ? val : 0.f;   // beyond the table: outside the cut
}

template <int PQ, bool REG>
__device__ __forceinline__ cx<float> green_sym_short(float dx, float dy, float dz, float2 d1, unsigned imask,
                                                     unsigned regm, const float4 *stab4,
                                                     const float4 *__restrict__ rtab, const EwaldF32 &ef) {
    float Dx[PQ + 1], Dy[PQ + 1];
    Dx[0] = 1.f;
    Dy[0] = 1.f;
    Dx[1] = d1.x;
    Dy[1] = d1.y;
#pragma unroll
    for (int k = 2; k <= PQ; ++k) {
        Dx[k] = fmaf(d1.x, Dx[k - 1], k == 2 ? -2.f : -Dx[k - 2]);
        Dy[k] = fmaf(d1.y, Dy[k - 1], k == 2 ? -2.f : -Dy[k - 2]);
    }
    float u;
    const int iz = table_index(fabsf(dz) * ef.z_inv_h, NZTAB, u);
    const float4 *rt = rtab + iz;
    // every entry of the quadrant, no branch: orders outside the cut read zeros
    float ar = 0.f;
#pragma unroll
    for (int p = 0; p <= PQ; ++p) {
        float rr = 0.f;
#pragma unroll
        for (int q = 0; q <= PQ; ++q) {
            const float4 c = __ldg(rt + ef.sq_off[p][q]);
            const float g = fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
            rr = q == 0 ? g : fmaf(Dy[q], g, rr);
        }
        ar = p == 0 ? rr : fmaf(Dx[p], rr, ar);
    }
    const float4 ci = __ldg(rt + ef.sq_im);
    const float ai = fmaf(u, fmaf(u, fmaf(u, ci.w, ci.z), ci.y), ci.x);
    // lattice images, two at a time (the mask is warp-uniform)
    const float dz2 = dz * dz;
    float sv = 0.f;
    for (unsigned mk = imask; mk;) {
        const int i0 = __ffs((int)mk) - 1;
        mk &= mk - 1u;
        if (mk) {
            const int i1 = __ffs((int)mk) - 1;
            mk &= mk - 1u;
            const float v0 = image_term<REG>(i0, dx, dy, dz2, regm, stab4, ef);
            const float v1 = image_term<REG>(i1, dx, dy, dz2, regm, stab4, ef);
            sv += v0 + v1;
        } else {
            sv += image_term<REG>(i0, dx, dy, dz2, regm, stab4, ef);
        }
    }
    ar = fmaf(ef.img[0][2], sv, ar);
    return {ar, ai};
}

// Images (32-bit mask) that can lie inside the cut for some displacement within
// `rad` of (cx, cy, cz); n_img <= 32.
__device__ __forceinline__ unsigned image_mask32(const EwaldF32 &ew, float cx, float cy, float cz, float rad) {
    const float rc = ew.xs_max / ew.Ef * 1.0001f + rad * 1.0001f + 1e-6f * (fabsf(cx) + fabsf(cy) + fabsf(cz));
    const float rc2 = rc * rc;
    const int n = ew.n_img;
    unsigned m = 0u;
    for (int i = 0; i < n; ++i) {
        const float x = cx + ew.img[i][0], y = cy + ew.img[i][1];
        if (x * x + y * y + cz * cz <= rc2) m |= 1u << i;
    }
    return m;
}

// 4 x 4 point pairs of one tetrahedron pair in the short form.  tpt: the test
// tetrahedron's points [a] = (x_a, x_a - c) and phases (2 cos, 2 cos, 2 sin,
// 2 sin) of 2 pi (x / a, y / b); sph (stride 128): the source points' (cos,
// cos, sin, sin).  The moments are accumulated without the weight.
template <int PQ, bool REG>
__device__ __forceinline__ void far_tt_short(const float *__restrict__ fs, const float4 (*tpt)[3],
                                             const float4 *sph, unsigned imask, unsigned regm,
                                             const float4 *stab4, const DevReq &q, Mom<float> &mo) {
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
        const float yb0 = fs[3 * b], yb1 = fs[3 * b + 1], yb2 = fs[3 * b + 2];
        const float rb[3] = {yb0 - fs[12], yb1 - fs[13], yb2 - fs[14]};
        const float4 pb = sph[128 * b];
#pragma unroll 1
        for (int a = 0; a < 4; ++a) {
            const float4 xa = tpt[a][0], ra = tpt[a][1], pa = tpt[a][2];
            // 2 cos(k (x_a - y_b)) = 2 cos(k x_a) cos(k y_b) + 2 sin(k x_a) sin(k y_b)
            const float2 d1 = {fmaf(pa.x, pb.x, pa.z * pb.z), fmaf(pa.y, pb.y, pa.w * pb.w)};
            const cx<float> g = green_sym_short<PQ, REG>(xa.x - yb0, xa.y - yb1, xa.z - yb2, d1, imask, regm,
                                                         stab4, q.rtab, q.ef);
            const float rr = ra.x * rb[0] + ra.y * rb[1] + ra.z * rb[2];
            mo.S = mo.S + g;
            cfma(mo.A[0], ra.x, g);
            cfma(mo.A[1], ra.y, g);
            cfma(mo.A[2], ra.z, g);
#pragma unroll
            for (int d = 0; d < 3; ++d) cfma(mo.B[d], rb[d], g);
            cfma(mo.C, rr, g);
        }
    }
}

// Far tetrahedron pairs at normal incidence in the short form: one thread per
// unordered pair {t, s} (s >= t) as in k_far_tt, the reversed pair's moments
// taken from the pair's own (g_p(-d) = g_p(d)).
#ifndef VIE_FAR_N_MINB
// CTAs per SM of the normal-incidence far kernels: the short form waits on its
// table loads, so registers (85 at six) pay more than warps (bench cell: 39.8 /
// 37.5 / 37.0 ms at eight / seven / six, eight spilling at 64 registers)
#define VIE_FAR_N_MINB 6
#endif
template <int PQ>
__global__ void __launch_bounds__(128, VIE_FAR_N_MINB) k_far_tt_n(DevMesh m, const __grid_constant__ DevReq q, float *Z, size_t N) {
    __shared__ float4 s_tab[NSPAT];   // spatial table
    __shared__ float4 s_sph[4 * 128];  // per thread: its source points' phases, [b][thread]
    __shared__ float4 s_tpt[4][3];     // the test tetrahedron's points, relative points, phases times 2
    const int t = blockIdx.y;
    if ((int)(blockIdx.x * blockDim.x + blockDim.x) <= t) return;   // the whole block is below the diagonal
    const EwaldF32 &ef = q.ef;
    const float4 *gtab = reinterpret_cast<const float4 *>(q.stab);
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = gtab[i];
    const float *ft = m.far<float>(t);
    const float sx = ef.step_x * 0.31830988618f, sy = ef.step_y * 0.31830988618f;   // 2/a, 2/b
    if (threadIdx.x < 4) {
        const int a = threadIdx.x;
        float sn_x, cs_x, sn_y, cs_y;
        sincospif(sx * ft[3 * a], &sn_x, &cs_x);
        sincospif(sy * ft[3 * a + 1], &sn_y, &cs_y);
        s_tpt[a][0] = make_float4(ft[3 * a], ft[3 * a + 1], ft[3 * a + 2], 0.f);
        s_tpt[a][1] = make_float4(ft[3 * a] - ft[12], ft[3 * a + 1] - ft[13], ft[3 * a + 2] - ft[14], 0.f);
        s_tpt[a][2] = make_float4(2.f * cs_x, 2.f * cs_y, 2.f * sn_x, 2.f * sn_y);
    }
    const int s0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s0 < m.nt && s0 >= t;   // lanes off the pair range stay until the warp's masks are formed
    const int s = live ? s0 : t;
    const float *fs = m.far<float>(s);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float sn_x, cs_x, sn_y, cs_y;
        sincospif(sx * fs[3 * b], &sn_x, &cs_x);
        sincospif(sy * fs[3 * b + 1], &sn_y, &cs_y);
        s_sph[128 * b + threadIdx.x] = make_float4(cs_x, cs_y, sn_x, sn_y);
    }
    // images that can reach the cut from some point pair of {t, s}: every point
    // pair lies within rt + rs of the centroid offset; one list for the warp
    float rt = 0.f, rs = 0.f;
    for (int a = 0; a < 4; ++a) {
        const float ux = ft[3 * a] - ft[12], uy = ft[3 * a + 1] - ft[13], uz = ft[3 * a + 2] - ft[14];
        const float vx = fs[3 * a] - fs[12], vy = fs[3 * a + 1] - fs[13], vz = fs[3 * a + 2] - fs[14];
        rt = fmaxf(rt, sqrtf(ux * ux + uy * uy + uz * uz));
        rs = fmaxf(rs, sqrtf(vx * vx + vy * vy + vz * vz));
    }
    unsigned imask = live ? image_mask32(ef, ft[12] - fs[12], ft[13] - fs[13], ft[14] - fs[14], rt + rs) : 0u;
    imask = __reduce_or_sync(0xffffffffu, imask);
    // near images of this pair: their static part is integrated separately
    const unsigned sub = live ? (unsigned)m.mk_tt[(size_t)t * m.nt + s] : 0u;
    unsigned regm = 0u;
    if (sub) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if ((sub >> k) & 1u) regm |= 1u << ef.near_img[k];
    }
    const bool reg = __any_sync(0xffffffffu, regm != 0u);
    __syncthreads();
    if (!live) return;
    Mom<float> mo, mr;
    mo.zero();
    if (reg) far_tt_short<PQ, true>(fs, s_tpt, s_sph + threadIdx.x, imask, regm, s_tab, q, mo);
    else far_tt_short<PQ, false>(fs, s_tpt, s_sph + threadIdx.x, imask, regm, s_tab, q, mo);
    const float wgt = ft[27] * fs[27];
    mo.S = wgt * mo.S;
    mo.C = wgt * mo.C;
    for (int d = 0; d < 3; ++d) { mo.A[d] = wgt * mo.A[d]; mo.B[d] = wgt * mo.B[d]; }
    // g_p(-d) = g_p(d): the reversed pair's moments swap A and B
    mr.S = mo.S;
    mr.C = mo.C;
    for (int d = 0; d < 3; ++d) { mr.A[d] = mo.B[d]; mr.B[d] = mo.A[d]; }
    scatter_tt<float>(m, q, Z, N, t, s, mo);
    if (s != t) scatter_tt<float>(m, q, Z, N, s, t, mr);
}

// ---------------------------------------------------------------------------
// Oblique incidence, short form of the tabulated evaluation.  With
// X_i = exp(-j (k_x0 + i s_x) dx), Y_j = exp(-j (k_y0 + j s_y) dy) (k_x0, k_y0
// the first order of the rectangle, s = 2 pi / period) and the spectral table
// G_ij(|z|) = Re G + j Im G of rectangle entry (i, j):
//   S = sum_ij X_i Y_j Re G_ij,   T = sum_ij X_i Y_j Im G_ij (propagating orders only),
//   g_p(d) = S + j T + sum_i F(R_i E)/R_i ph_i      (ph_i: image phase exp(j k_par.R_i) exp(b^2)/(4 pi)).
// Re G is real, so the spectral part of g_p(-d) = sum G conj(X Y) is
// conj(S) + j conj(T), and the image part is the conjugate of the image part
// of g_p(d): g_p(-d) = conj(g_p(d)) + 2 j conj(T).  The returned T carries
// that correction.  X0, SX, Y0, SY: X_0, exp(-j s_x dx), Y_0, exp(-j s_y dy).
// ---------------------------------------------------------------------------
template <bool REG>
__device__ __forceinline__ float image_term64(int i, float dx, float dy, float dz2, unsigned long long regm,
                                              const float4 *stab4, const EwaldF32 &ef) {
    const float x = dx + ef.img[i][0], y = dy + ef.img[i][1];
    const float R2 = fmaf(x, x, fmaf(y, y, dz2));
    float rinv = rsqrtf(R2);
    if (REG) rinv = R2 > 0.f ? rinv : 0.f;   // R = 0 only on an image whose static part is removed
    const float xu = R2 * rinv * ef.Eih;
    float v;
    const int ix = table_index(xu, NSPAT, v);
    const float4 c = stab4[ix];
    const float q1 = fmaf(v, fmaf(v, c.w, c.z), c.y);
    float val = fmaf(v, q1, c.x) * rinv;
    if (REG && ((regm >> i) & 1ull))   // (F(x) - F(0)) / R; near R = 0 from the first interval's slope
        val = ix == 0 ? ef.Eih * q1 : fmaf(-ef.e_mb2, rinv, val);
    return xu <= float(NSPAT) ? val : 0.f;   // beyond the table: outside the cut
}

template <int NR, bool REG>
__device__ __forceinline__ cx<float> green_obl_short(float dx, float dy, float dz, cx<float> X0, cx<float> SX,
                                                     cx<float> Y0, cx<float> SY, unsigned long long imask,
                                                     unsigned long long regm, const float4 *stab4,
                                                     const float4 *__restrict__ rtab, const EwaldF32 &ef,
                                                     cx<float> &T) {
    cx<float> Y[NR];
    Y[0] = Y0;
#pragma unroll
    for (int j = 1; j < NR; ++j) Y[j] = Y[j - 1] * SY;
    float u;
    const int iz = table_index(fabsf(dz) * ef.z_inv_h, NZTAB, u);
    const float4 *rt = rtab + iz;
    cx<float> S = {0.f, 0.f}, X = X0;
    T = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        cx<float> inr = {0.f, 0.f}, ini = {0.f, 0.f};
        bool cplx = false;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const float4 c = __ldg(rt + ef.ob_off[i][j]);   // entries outside the cut read zeros
            const float g = fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
            cfma(inr, g, Y[j]);
            const int im = ef.ob_im[i][j];
            if (im >= 0) {   // propagating order (uniform branch)
                const float4 ci = __ldg(rt + im);
                cfma(ini, fmaf(u, fmaf(u, fmaf(u, ci.w, ci.z), ci.y), ci.x), Y[j]);
                cplx = true;
            }
        }
        S = S + X * inr;
        if (cplx) T = T + X * ini;
        if (i + 1 < NR) X = X * SX;
    }
    // lattice images, two at a time (the mask is warp-uniform)
    const float dz2 = dz * dz;
    cx<float> acc = {S.re - T.im, S.im + T.re};
    for (unsigned long long mk = imask; mk;) {
        const int i0 = __ffsll((long long)mk) - 1;
        mk &= mk - 1ull;
        const float v0 = image_term64<REG>(i0, dx, dy, dz2, regm, stab4, ef);
        acc.re = fmaf(v0, ef.img[i0][2], acc.re);
        acc.im = fmaf(v0, ef.img[i0][3], acc.im);
        if (mk) {
            const int i1 = __ffsll((long long)mk) - 1;
            mk &= mk - 1ull;
            const float v1 = image_term64<REG>(i1, dx, dy, dz2, regm, stab4, ef);
            acc.re = fmaf(v1, ef.img[i1][2], acc.re);
            acc.im = fmaf(v1, ef.img[i1][3], acc.im);
        }
    }
    return acc;
}

// The same at k_y = 0 with the order rectangle symmetric in q: G_pq = G_p,-q,
// so sum_q Y_q G_pq = sum_{q >= 0} w_q cos(q s_y dy) G_pq (w_0 = 1, w_q = 2),
// a real weight D_q = 2 cos(q s_y dy) (D_0 -> 1) by the Chebyshev recurrence
// from d1y = 2 cos(s_y dy); entry (i, q) of the tables is order (p0 + i, q).
template <int NP, int NQ1, bool REG>
__device__ __forceinline__ cx<float> green_obl_ky0(float dx, float dy, float dz, cx<float> X0, cx<float> SX,
                                                   float d1y, unsigned long long imask, unsigned long long regm,
                                                   const float4 *stab4, const float4 *__restrict__ rtab,
                                                   const EwaldF32 &ef, cx<float> &T) {
    float Dy[NQ1];
    Dy[0] = 1.f;
    Dy[1] = d1y;
#pragma unroll
    for (int k = 2; k < NQ1; ++k) Dy[k] = fmaf(d1y, Dy[k - 1], k == 2 ? -2.f : -Dy[k - 2]);
    float u;
    const int iz = table_index(fabsf(dz) * ef.z_inv_h, NZTAB, u);
    const float4 *rt = rtab + iz;
    cx<float> S = {0.f, 0.f}, X = X0;
    T = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float inr = 0.f, ini = 0.f;
        bool cplx = false;
#pragma unroll
        for (int q = 0; q < NQ1; ++q) {
            const float4 c = __ldg(rt + ef.ob_off[i][q]);   // entries outside the cut read zeros
            const float g = fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
            inr = q == 0 ? g : fmaf(Dy[q], g, inr);
            const int im = ef.ob_im[i][q];
            if (im >= 0) {   // propagating order (uniform branch)
                const float4 ci = __ldg(rt + im);
                const float gi = fmaf(u, fmaf(u, fmaf(u, ci.w, ci.z), ci.y), ci.x);
                ini = q == 0 ? ini + gi : fmaf(Dy[q], gi, ini);
                cplx = true;
            }
        }
        S.re = fmaf(X.re, inr, S.re);
        S.im = fmaf(X.im, inr, S.im);
        if (cplx) {
            T.re = fmaf(X.re, ini, T.re);
            T.im = fmaf(X.im, ini, T.im);
        }
        if (i + 1 < NP) X = X * SX;
    }
    const float dz2 = dz * dz;
    cx<float> acc = {S.re - T.im, S.im + T.re};
    for (unsigned long long mk = imask; mk;) {
        const int i0 = __ffsll((long long)mk) - 1;
        mk &= mk - 1ull;
        const float v0 = image_term64<REG>(i0, dx, dy, dz2, regm, stab4, ef);
        acc.re = fmaf(v0, ef.img[i0][2], acc.re);
        acc.im = fmaf(v0, ef.img[i0][3], acc.im);
        if (mk) {
            const int i1 = __ffsll((long long)mk) - 1;
            mk &= mk - 1ull;
            const float v1 = image_term64<REG>(i1, dx, dy, dz2, regm, stab4, ef);
            acc.re = fmaf(v1, ef.img[i1][2], acc.re);
            acc.im = fmaf(v1, ef.img[i1][3], acc.im);
        }
    }
    return acc;
}

// the oblique evaluation of one point pair: NQ1 = 0 the full rectangle (NR x NR),
// else the k_y = 0 fold (NR x NQ1); sa, sb carry (cos, sin) of s_x x and s_y y
template <int NR, int NQ1, bool REG>
__device__ __forceinline__ cx<float> green_obl(float dx, float dy, float dz, float4 pa, float4 sa, float4 pb,
                                               float4 sb, unsigned long long imask, unsigned long long regm,
                                               const float4 *stab4, const float4 *__restrict__ rtab,
                                               const EwaldF32 &ef, cx<float> &T);

// e^{-j th_a} conj(e^{-j th_b}) = e^{-j (th_a - th_b)} from (cos, sin) of th_a and th_b
__device__ __forceinline__ cx<float> phase_diff(float ca, float sa, float cb, float sb) {
    return {fmaf(ca, cb, sa * sb), fmaf(ca, sb, -sa * cb)};
}

template <int NR, int NQ1, bool REG>
__device__ __forceinline__ cx<float> green_obl(float dx, float dy, float dz, float4 pa, float4 sa, float4 pb,
                                               float4 sb, unsigned long long imask, unsigned long long regm,
                                               const float4 *stab4, const float4 *__restrict__ rtab,
                                               const EwaldF32 &ef, cx<float> &T) {
    const cx<float> X0 = phase_diff(pa.x, pa.y, pb.x, pb.y), SX = phase_diff(sa.x, sa.y, sb.x, sb.y);
    if constexpr (NQ1 > 0) {
        const float d1y = 2.f * fmaf(sa.z, sb.z, sa.w * sb.w);   // 2 cos(s_y (y_a - y_b))
        return green_obl_ky0<NR, NQ1, REG>(dx, dy, dz, X0, SX, d1y, imask, regm, stab4, rtab, ef, T);
    } else {
        const cx<float> Y0 = phase_diff(pa.z, pa.w, pb.z, pb.w), SY = phase_diff(sa.z, sa.w, sb.z, sb.w);
        return green_obl_short<NR, REG>(dx, dy, dz, X0, SX, Y0, SY, imask, regm, stab4, rtab, ef, T);
    }
}

// 4 x 4 point pairs of one tetrahedron pair in the oblique short form.  tpt:
// the test points [a] = (x_a, x_a - c, (cos, sin) of k_x0 x and k_y0 y,
// (cos, sin) of s_x x and s_y y); sph (stride 128, two float4 per point): the
// same phases of the source points.  mo: moments of g_p(x_a - y_b); mc: the
// correction 2 j conj(T) of g_p(y_b - x_a) with the reversed pair's roles.
template <int NR, int NQ1, bool REG>
__device__ __forceinline__ void far_tt_obl(const float *__restrict__ fs, const float4 (*tpt)[4], const float4 *sph,
                                           unsigned long long imask, unsigned long long regm, const float4 *stab4,
                                           const DevReq &q, Mom<float> &mo, Mom<float> &mc) {
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
        const float yb0 = fs[3 * b], yb1 = fs[3 * b + 1], yb2 = fs[3 * b + 2];
        const float rb[3] = {yb0 - fs[12], yb1 - fs[13], yb2 - fs[14]};
        const float4 pb = sph[256 * b], sb = sph[256 * b + 128];
#pragma unroll 1
        for (int a = 0; a < 4; ++a) {
            const float4 xa = tpt[a][0], ra = tpt[a][1], pa = tpt[a][2], sa = tpt[a][3];
            cx<float> T;
            const cx<float> g = green_obl<NR, NQ1, REG>(xa.x - yb0, xa.y - yb1, xa.z - yb2, pa, sa, pb, sb, imask,
                                                        regm, stab4, q.rtab, q.ef, T);
            const cx<float> c = {2.f * T.im, 2.f * T.re};   // 2 j conj(T)
            const float rr = ra.x * rb[0] + ra.y * rb[1] + ra.z * rb[2];
            mo.S = mo.S + g;
            cfma(mo.A[0], ra.x, g);
            cfma(mo.A[1], ra.y, g);
            cfma(mo.A[2], ra.z, g);
            mc.S = mc.S + c;
            cfma(mc.B[0], ra.x, c);
            cfma(mc.B[1], ra.y, c);
            cfma(mc.B[2], ra.z, c);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cfma(mo.B[d], rb[d], g);
                cfma(mc.A[d], rb[d], c);
            }
            cfma(mo.C, rr, g);
            cfma(mc.C, rr, c);
        }
    }
}

// (cos, sin) of k_x0 x, k_y0 y and of s_x x, s_y y of one point
__device__ __forceinline__ void obl_point_phases(const EwaldF32 &ef, float x, float y, float4 &p, float4 &st) {
    float s0, c0, s1, c1, s2, c2, s3, c3;
    sincospif(ef.ob_kx0 * 0.31830988618f * x, &s0, &c0);
    sincospif(ef.ob_ky0 * 0.31830988618f * y, &s1, &c1);
    sincospif(ef.step_x * 0.31830988618f * x, &s2, &c2);
    sincospif(ef.step_y * 0.31830988618f * y, &s3, &c3);
    p = make_float4(c0, s0, c1, s1);
    st = make_float4(c2, s2, c3, s3);
}

#ifndef VIE_FAR_O_MINB
// CTAs per SM of the oblique-incidence far kernels (bench cell at theta = 0.3,
// the general order rectangle: 81.6 / 78.3 / 82.3 ms at six / five / four)
#define VIE_FAR_O_MINB 5
#endif
// Far tetrahedron pairs at oblique incidence in the short form: one thread per
// unordered pair {t, s} (s >= t); the reversed pair's moments are the
// conjugates of the pair's own, exchanged, plus the propagating-order correction.
template <int NR, int NQ1>
__global__ void __launch_bounds__(128, VIE_FAR_O_MINB) k_far_tt_o(DevMesh m, const __grid_constant__ DevReq q, float *Z,
                                                                  size_t N) {
    __shared__ float4 s_tab[NSPAT];
    __shared__ float4 s_sph[4 * 2 * 128];   // [b][phase pair][thread]
    __shared__ float4 s_tpt[4][4];
    const int t = blockIdx.y;
    if ((int)(blockIdx.x * blockDim.x + blockDim.x) <= t) return;   // the whole block is below the diagonal
    const EwaldF32 &ef = q.ef;
    const float4 *gtab = reinterpret_cast<const float4 *>(q.stab);
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = gtab[i];
    const float *ft = m.far<float>(t);
    if (threadIdx.x < 4) {
        const int a = threadIdx.x;
        float4 p, st;
        obl_point_phases(ef, ft[3 * a], ft[3 * a + 1], p, st);
        s_tpt[a][0] = make_float4(ft[3 * a], ft[3 * a + 1], ft[3 * a + 2], 0.f);
        s_tpt[a][1] = make_float4(ft[3 * a] - ft[12], ft[3 * a + 1] - ft[13], ft[3 * a + 2] - ft[14], 0.f);
        s_tpt[a][2] = p;
        s_tpt[a][3] = st;
    }
    const int s0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s0 < m.nt && s0 >= t;
    const int s = live ? s0 : t;
    const float *fs = m.far<float>(s);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float4 p, st;
        obl_point_phases(ef, fs[3 * b], fs[3 * b + 1], p, st);
        s_sph[256 * b + threadIdx.x] = p;
        s_sph[256 * b + 128 + threadIdx.x] = st;
    }
    float rt = 0.f, rs = 0.f;
    for (int a = 0; a < 4; ++a) {
        const float ux = ft[3 * a] - ft[12], uy = ft[3 * a + 1] - ft[13], uz = ft[3 * a + 2] - ft[14];
        const float vx = fs[3 * a] - fs[12], vy = fs[3 * a + 1] - fs[13], vz = fs[3 * a + 2] - fs[14];
        rt = fmaxf(rt, sqrtf(ux * ux + uy * uy + uz * uz));
        rs = fmaxf(rs, sqrtf(vx * vx + vy * vy + vz * vz));
    }
    unsigned long long imask = live ? image_mask(ef, ft[12] - fs[12], ft[13] - fs[13], ft[14] - fs[14], rt + rs) : 0ull;
    {
        const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)imask);
        const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(imask >> 32));
        imask = ((unsigned long long)hi << 32) | lo;
    }
    const unsigned sub = live ? (unsigned)m.mk_tt[(size_t)t * m.nt + s] : 0u;
    unsigned long long regm = 0ull;
    if (sub) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if ((sub >> k) & 1u) regm |= 1ull << ef.near_img[k];
    }
    const bool reg = __any_sync(0xffffffffu, regm != 0ull);
    __syncthreads();
    if (!live) return;
    Mom<float> mo, mc;
    mo.zero();
    mc.zero();
    if (reg) far_tt_obl<NR, NQ1, true>(fs, s_tpt, s_sph + threadIdx.x, imask, regm, s_tab, q, mo, mc);
    else far_tt_obl<NR, NQ1, false>(fs, s_tpt, s_sph + threadIdx.x, imask, regm, s_tab, q, mo, mc);
    const float wgt = ft[27] * fs[27];
    Mom<float> mr;
    mr.S = wgt * (cconj(mo.S) + mc.S);
    mr.C = wgt * (cconj(mo.C) + mc.C);
    for (int d = 0; d < 3; ++d) {
        mr.A[d] = wgt * (cconj(mo.B[d]) + mc.A[d]);
        mr.B[d] = wgt * (cconj(mo.A[d]) + mc.B[d]);
    }
    mo.S = wgt * mo.S;
    mo.C = wgt * mo.C;
    for (int d = 0; d < 3; ++d) { mo.A[d] = wgt * mo.A[d]; mo.B[d] = wgt * mo.B[d]; }
    scatter_tt<float>(m, q, Z, N, t, s, mo);
    if (s != t) scatter_tt<float>(m, q, Z, N, s, t, mr);
}

// ---------------------------------------------------------------------------
// near tetrahedron pairs: one warp per pair
// ---------------------------------------------------------------------------
template <typename U>
__device__ void static_tt_term(const double *r5, double w, const double *tv_other, const double *R,
                               double sgnR, const double *c_self, const double *c_other, bool order_i,
                               cx<double> ph, Mom<double> &acc) {
    // outer point r (double), closed form over the other tetrahedron shifted by
    // sgnR*R; coordinates relative to r are formed in FP64 before narrowing to U
    U r[3] = {U(0), U(0), U(0)};
    U tv[12];
    for (int j = 0; j < 4; ++j)
        for (int d = 0; d < 3; ++d) tv[3 * j + d] = U((tv_other[3 * j + d] + sgnR * R[d]) - r5[d]);
    U inv, vec[3];
    tet_integrals<U>(r, tv, inv, vec, true);
    double I = double(inv);
    double f[3], rho[3];
    for (int d = 0; d < 3; ++d) {
        // int (r' - c_other_shifted)/R dV' and the outer point relative to its centroid
        f[d] = double(vec[d]) + (r5[d] - (c_other[d] + sgnR * R[d])) * I;
        rho[d] = r5[d] - c_self[d];
    }
    cx<double> pw = {ph.re * w, ph.im * w};
    acc.S = acc.S + I * pw;
    if (order_i) {   // outer on test: A gets rho*I, B gets f
        for (int d = 0; d < 3; ++d) {
            acc.A[d] = acc.A[d] + (rho[d] * I) * pw;
            acc.B[d] = acc.B[d] + f[d] * pw;
        }
    } else {          // outer on source: B gets rho'*I, A gets f
        for (int d = 0; d < 3; ++d) {
            acc.B[d] = acc.B[d] + (rho[d] * I) * pw;
            acc.A[d] = acc.A[d] + f[d] * pw;
        }
    }
    acc.C = acc.C + (rho[0] * f[0] + rho[1] * f[1] + rho[2] * f[2]) * pw;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// near image of a pair, elements not touching: degree-5 x degree-5 product
// rule of exp(j k_par.R)/(4 pi R), one thread per (pair, image)
template <typename T>
__global__ void __launch_bounds__(128) k_pr_tt(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N, const NearEntry *list, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const NearEntry en = list[e];
    const int t = en.x, s = en.y, k = en.k;
    const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
    const double *ct = m.cen + 3 * (size_t)t, *cs = m.cen + 3 * (size_t)s;
    const T *nx = m.nrel<T>(t), *ny = m.nrel<T>(s);
    const T dc[3] = {T(ct[0] - cs[0] + R[0]), T(ct[1] - cs[1] + R[1]), T(ct[2] - cs[2])};
    T s0 = 0, sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0}, sC = 0;
    for (int a = 0; a < 14; ++a) {
        const T xa[4] = {nx[4 * a], nx[4 * a + 1], nx[4 * a + 2], nx[4 * a + 3]};
        T f0 = 0, fb[3] = {0, 0, 0};
        for (int b = 0; b < 14; ++b) {
            const T *yb = ny + 4 * b;
            const T dx = xa[0] - yb[0] + dc[0], dy = xa[1] - yb[1] + dc[1], dz = xa[2] - yb[2] + dc[2];
            const T f = yb[3] * rsqrt(dx * dx + dy * dy + dz * dz);
            f0 += f;
            fb[0] += f * yb[0];
            fb[1] += f * yb[1];
            fb[2] += f * yb[2];
        }
        f0 *= xa[3];
        for (int d = 0; d < 3; ++d) fb[d] *= xa[3];
        s0 += f0;
        for (int d = 0; d < 3; ++d) {
            sA[d] += f0 * xa[d];
            sB[d] += fb[d];
        }
        sC += xa[0] * fb[0] + xa[1] * fb[1] + xa[2] * fb[2];
    }
    const cx<T> pt = {T(q.img_ph[2 * k]), T(q.img_ph[2 * k + 1])};
    Mom<T> mo;
    mo.S = s0 * pt;
    mo.C = sC * pt;
    for (int d = 0; d < 3; ++d) {
        mo.A[d] = sA[d] * pt;
        mo.B[d] = sB[d] * pt;
    }
    scatter_tt<T>(m, q, Z, N, t, s, mo);
}

// near image of a pair whose elements touch: closed form over one element at
// the degree-5 points of the other, both orders averaged, in FP64; one warp per
// (pair, image), lanes 0..13 order (i), 14..27 order (ii)
template <typename T>
__global__ void __launch_bounds__(128) k_touch_tt(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N, const NearEntry *list,
                                                  int n) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;
    const NearEntry en = list[wid];
    const int t = en.x, s = en.y, k = en.k;
    Mom<double> acc;
    acc.zero();
    if (lane < 28) {
        const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
        const cx<double> hph = {0.5 * q.img_ph[2 * k], 0.5 * q.img_ph[2 * k + 1]};
        const bool oi = lane < 14;
        const int qi = oi ? lane : lane - 14;
        const int self = oi ? t : s, other = oi ? s : t;
        const double *r5 = m.q5 + (size_t)self * 42 + 3 * qi;
        const double w = m.vol[self] * c_w5tet[qi];
        static_tt_term<double>(r5, w, m.tv + 12 * (size_t)other, R, oi ? -1.0 : 1.0, m.cen + 3 * self,
                               m.cen + 3 * other, oi, hph, acc);
    }
    double v[16] = {acc.S.re, acc.S.im, acc.C.re, acc.C.im, acc.A[0].re, acc.A[0].im, acc.A[1].re, acc.A[1].im,
                    acc.A[2].re, acc.A[2].im, acc.B[0].re, acc.B[0].im, acc.B[1].re, acc.B[1].im, acc.B[2].re,
                    acc.B[2].im};
    for (int i = 0; i < 16; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
        Mom<T> mo;
        mo.S = {T(v[0]), T(v[1])};
        mo.C = {T(v[2]), T(v[3])};
        for (int d = 0; d < 3; ++d) {
            mo.A[d] = {T(v[4 + 2 * d]), T(v[5 + 2 * d])};
            mo.B[d] = {T(v[10 + 2 * d]), T(v[11 + 2 * d])};
        }
        scatter_tt<T>(m, q, Z, N, t, s, mo);
    }
}

// Touching images, exploiting the symmetry of the two integration orders:
// order (ii) of the entry (t, s, k) is order (i) of its partner (s, t, 8-k)
// with the test and source polynomial moments exchanged.  k_touch_half
// computes order (i) of every entry once (phase-free real moments, FP64;
// half a warp per entry, lane q = degree-5 point q of the test element);
// k_touch_combine averages each entry with its partner and scatters.
__global__ void __launch_bounds__(128) k_touch_half(DevMesh m, const NearEntry *list, int n, double *out) {
    const int e = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2 + ((threadIdx.x >> 4) & 1);
    const int hl = threadIdx.x & 15;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e < n && hl < 14) {
        const NearEntry en = list[e];
        const int t = en.x, s = en.y, k = en.k;
        const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
        const double *r5 = m.q5 + (size_t)t * 42 + 3 * hl;
        const double w = m.vol[t] * c_w5tet[hl];
        const double *src = m.tv + 12 * (size_t)s;
        const double *ct = m.cen + 3 * (size_t)t, *cs = m.cen + 3 * (size_t)s;
        double rel[12];
        for (int j = 0; j < 4; ++j)
            for (int d = 0; d < 3; ++d) rel[3 * j + d] = (src[3 * j + d] - R[d]) - r5[d];
        double I, vec[3];
        tet_integrals_shared(rel, I, vec);
        double f[3], rho[3];
        for (int d = 0; d < 3; ++d) {
            f[d] = vec[d] + (r5[d] - (cs[d] - R[d])) * I;   // int (r' - c_s)/R over the image source
            rho[d] = r5[d] - ct[d];
        }
        acc[0] = w * I;
        for (int d = 0; d < 3; ++d) {
            acc[1 + d] = w * rho[d] * I;   // test polynomial
            acc[4 + d] = w * f[d];         // source polynomial
        }
        acc[7] = w * (rho[0] * f[0] + rho[1] * f[1] + rho[2] * f[2]);
    }
    for (int i = 0; i < 8; ++i)
        for (int o = 8; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o, 16);
    if (e < n && hl == 0)
        for (int i = 0; i < 8; ++i) out[8 * (size_t)e + i] = acc[i];
}

template <typename T>
__global__ void __launch_bounds__(128) k_touch_combine(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N, const NearEntry *list,
                                                       const int32_t *partner, const double *half, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const NearEntry en = list[e];
    const double *a = half + 8 * (size_t)e;
    const double *b = half + 8 * (size_t)partner[e];
    const double pr = 0.5 * q.img_ph[2 * en.k], pi = 0.5 * q.img_ph[2 * en.k + 1];
    // moments of this entry: S and C symmetric, test/source polynomials exchanged in the partner
    double v[8];
    v[0] = a[0] + b[0];
    for (int d = 0; d < 3; ++d) {
        v[1 + d] = a[1 + d] + b[4 + d];
        v[4 + d] = a[4 + d] + b[1 + d];
    }
    v[7] = a[7] + b[7];
    Mom<T> mo;
    mo.S = {T(pr * v[0]), T(pi * v[0])};
    mo.C = {T(pr * v[7]), T(pi * v[7])};
    for (int d = 0; d < 3; ++d) {
        mo.A[d] = {T(pr * v[1 + d]), T(pi * v[1 + d])};
        mo.B[d] = {T(pr * v[4 + d]), T(pi * v[4 + d])};
    }
    scatter_tt<T>(m, q, Z, N, en.x, en.y, mo);
}

// ---------------------------------------------------------------------------
// scalar element pairs involving charge faces:
//   TF: test tet t, source charge face f   -> Z[row(t,i), frow(f)] += wt 3c qs_f S
//   FT: test half face h, source tet s     -> Z[frow(hf h), row(s,j)] -= conj(wt) kappa_s 3c S
//   FF: test half face h, source face f    -> Z[frow(hf h), frow(f)] -= qs_f S
// ---------------------------------------------------------------------------
enum PairKind { PK_TF = 0, PK_FT = 1, PK_FF = 2 };

template <int PK> struct PKTraits;
template <> struct PKTraits<PK_TF> { static constexpr bool xtet = true, ytet = false; };
template <> struct PKTraits<PK_FT> { static constexpr bool xtet = false, ytet = true; };
template <> struct PKTraits<PK_FF> { static constexpr bool xtet = false, ytet = false; };

template <typename T, int PK>
__device__ void scatter_scalar(const DevMesh &m, const DevReq &q, T *Z, size_t N, int x, int y, cx<T> S) {
    if (PK == PK_TF) {
        cx<T> qs = {T(q.qs[2 * y]), T(q.qs[2 * y + 1])};
        size_t col = (size_t)q.frow[y];
        cx<T> qS = qs * S;
        for (int i = 0; i < 4; ++i) {
            cx<T> wti = {T(q.wt[2 * (4 * x + i)]), T(q.wt[2 * (4 * x + i) + 1])};
            T di = T(3) * T(q.coef[4 * x + i]);
            atomic_add_c(Z, (size_t)q.row[4 * x + i] * N + col, di * (wti * qS));
        }
    } else if (PK == PK_FT) {
        size_t row = (size_t)q.frow[m.hf[x]];
        cx<T> kap = {T(q.kap[2 * y]), T(q.kap[2 * y + 1])};
        cx<T> kS = kap * S;
        for (int j = 0; j < 4; ++j) {
            cx<T> wsj = {T(q.wt[2 * (4 * y + j)]), -T(q.wt[2 * (4 * y + j) + 1])};
            T dj = T(3) * T(q.coef[4 * y + j]);
            atomic_add_c(Z, row * N + (size_t)q.row[4 * y + j], (-dj) * (wsj * kS));
        }
    } else {
        size_t row = (size_t)q.frow[m.hf[x]];
        cx<T> qs = {T(q.qs[2 * y]), T(q.qs[2 * y + 1])};
        atomic_add_c(Z, row * N + (size_t)q.frow[y], T(-1) * (qs * S));
    }
}

template <typename T, bool TET>
__device__ __forceinline__ const T *far_el(const DevMesh &m, int e) {
    return TET ? m.far<T>(e) : m.ffar<T>(e);
}

// SYM: normal incidence (the tabulated path's symmetric mode sum).
template <typename T, int PK, bool SYM>
__global__ void __launch_bounds__(128) k_far_scalar(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N, int nx, int ny,
                                                    const uint16_t *mk) {
    extern __shared__ float smem_tab[];
    const float *stab = stage_stab<T>(q, smem_tab);
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (y >= ny) return;
    const unsigned sub = mk[(size_t)x * ny + y];
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    // a test face is addressed by its half-function index; geometry by charge-face index
    const T *fx = far_el<T, XT>(m, XT ? x : m.hf[x]);
    const T *fy = far_el<T, YT>(m, y);
    const int qx = XT ? 4 : 3, qy = YT ? 4 : 3;
    const T wgt = fx[XT ? 27 : 9] * fy[YT ? 27 : 9];
    // images that can reach the cut from some point pair, decided once per
    // element pair (FP32 tables only): centres and radii of the two point sets
    unsigned long long imask = ~0ull;
    if (sizeof(T) == 4) {
        float c1[3] = {0.f, 0.f, 0.f}, c2[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < qx; ++a)
            for (int d = 0; d < 3; ++d) c1[d] += float(fx[3 * a + d]) / qx;
        for (int b = 0; b < qy; ++b)
            for (int d = 0; d < 3; ++d) c2[d] += float(fy[3 * b + d]) / qy;
        float r1 = 0.f, r2 = 0.f;
        for (int a = 0; a < qx; ++a) {
            const float ux = float(fx[3 * a]) - c1[0], uy = float(fx[3 * a + 1]) - c1[1], uz = float(fx[3 * a + 2]) - c1[2];
            r1 = fmaxf(r1, sqrtf(ux * ux + uy * uy + uz * uz));
        }
        for (int b = 0; b < qy; ++b) {
            const float ux = float(fy[3 * b]) - c2[0], uy = float(fy[3 * b + 1]) - c2[1], uz = float(fy[3 * b + 2]) - c2[2];
            r2 = fmaxf(r2, sqrtf(ux * ux + uy * uy + uz * uz));
        }
        imask = image_mask(q.ef, c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2], r1 + r2);
    }
    cx<T> S = {0, 0};
    for (int a = 0; a < qx; ++a)
        for (int b = 0; b < qy; ++b) {
            cx<T> g = Green<T>::template eval<SYM>(fx[3 * a] - fy[3 * b], fx[3 * a + 1] - fy[3 * b + 1],
                                                   fx[3 * a + 2] - fy[3 * b + 2], sub, stab, q.ztab, q.ew, q.ef,
                                                   q.rtab, imask);
            S = S + g;
        }
    S = wgt * S;
    scatter_scalar<T, PK>(m, q, Z, N, x, y, S);
}

// Far scalar pairs (charge faces) at normal incidence in the short form: one
// thread per element pair as in k_far_scalar; the x element's points and their
// phases (times 2) staged once per block, each thread's y points' phases in
// shared memory [b][thread].
template <int PQ, int PK>
__global__ void __launch_bounds__(128, VIE_FAR_N_MINB)
    k_far_scalar_n(DevMesh m, const __grid_constant__ DevReq q, float *Z, size_t N, int nx, int ny,
                   const uint16_t *mk) {
    __shared__ float4 s_tab[NSPAT];
    __shared__ float4 s_yph[4 * 128];
    __shared__ float4 s_xpt[4][2];
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    constexpr int qx = XT ? 4 : 3, qy = YT ? 4 : 3;
    const EwaldF32 &ef = q.ef;
    const int x = blockIdx.y;
    const float4 *gtab = reinterpret_cast<const float4 *>(q.stab);
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = gtab[i];
    // a test face is addressed by its half-function index; geometry by charge-face index
    const float *fx = far_el<float, XT>(m, XT ? x : m.hf[x]);
    const float sx = ef.step_x * 0.31830988618f, sy = ef.step_y * 0.31830988618f;
    if (threadIdx.x < qx) {
        const int a = threadIdx.x;
        float sn_x, cs_x, sn_y, cs_y;
        sincospif(sx * fx[3 * a], &sn_x, &cs_x);
        sincospif(sy * fx[3 * a + 1], &sn_y, &cs_y);
        s_xpt[a][0] = make_float4(fx[3 * a], fx[3 * a + 1], fx[3 * a + 2], 0.f);
        s_xpt[a][1] = make_float4(2.f * cs_x, 2.f * cs_y, 2.f * sn_x, 2.f * sn_y);
    }
    const int y0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = y0 < ny;
    const int y = live ? y0 : ny - 1;
    const float *fy = far_el<float, YT>(m, y);
#pragma unroll
    for (int b = 0; b < qy; ++b) {
        float sn_x, cs_x, sn_y, cs_y;
        sincospif(sx * fy[3 * b], &sn_x, &cs_x);
        sincospif(sy * fy[3 * b + 1], &sn_y, &cs_y);
        s_yph[128 * b + threadIdx.x] = make_float4(cs_x, cs_y, sn_x, sn_y);
    }
    // images that can reach the cut from some point pair: centres and radii of the point sets
    float c1[3] = {0.f, 0.f, 0.f}, c2[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < qx; ++a)
        for (int d = 0; d < 3; ++d) c1[d] += fx[3 * a + d] / qx;
    for (int b = 0; b < qy; ++b)
        for (int d = 0; d < 3; ++d) c2[d] += fy[3 * b + d] / qy;
    float r1 = 0.f, r2 = 0.f;
    for (int a = 0; a < qx; ++a) {
        const float ux = fx[3 * a] - c1[0], uy = fx[3 * a + 1] - c1[1], uz = fx[3 * a + 2] - c1[2];
        r1 = fmaxf(r1, sqrtf(ux * ux + uy * uy + uz * uz));
    }
    for (int b = 0; b < qy; ++b) {
        const float ux = fy[3 * b] - c2[0], uy = fy[3 * b + 1] - c2[1], uz = fy[3 * b + 2] - c2[2];
        r2 = fmaxf(r2, sqrtf(ux * ux + uy * uy + uz * uz));
    }
    unsigned imask = live ? image_mask32(ef, c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2], r1 + r2) : 0u;
    imask = __reduce_or_sync(0xffffffffu, imask);
    const unsigned sub = live ? (unsigned)mk[(size_t)x * ny + y] : 0u;
    unsigned regm = 0u;
    if (sub) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if ((sub >> k) & 1u) regm |= 1u << ef.near_img[k];
    }
    const bool reg = __any_sync(0xffffffffu, regm != 0u);
    __syncthreads();
    if (!live) return;
    cx<float> S = {0.f, 0.f};
#pragma unroll 1
    for (int b = 0; b < qy; ++b) {
        const float yb0 = fy[3 * b], yb1 = fy[3 * b + 1], yb2 = fy[3 * b + 2];
        const float4 pb = s_yph[128 * b + threadIdx.x];
#pragma unroll 1
        for (int a = 0; a < qx; ++a) {
            const float4 xa = s_xpt[a][0], pa = s_xpt[a][1];
            const float2 d1 = {fmaf(pa.x, pb.x, pa.z * pb.z), fmaf(pa.y, pb.y, pa.w * pb.w)};
            const cx<float> g = reg ? green_sym_short<PQ, true>(xa.x - yb0, xa.y - yb1, xa.z - yb2, d1, imask, regm,
                                                                s_tab, q.rtab, ef)
                                    : green_sym_short<PQ, false>(xa.x - yb0, xa.y - yb1, xa.z - yb2, d1, imask, 0u,
                                                                 s_tab, q.rtab, ef);
            S = S + g;
        }
    }
    S = (fx[XT ? 27 : 9] * fy[YT ? 27 : 9]) * S;
    scatter_scalar<float, PK>(m, q, Z, N, x, y, S);
}

// Far scalar pairs (charge faces) at oblique incidence in the short form.
template <int NR, int NQ1, int PK>
__global__ void __launch_bounds__(128, VIE_FAR_O_MINB)
    k_far_scalar_o(DevMesh m, const __grid_constant__ DevReq q, float *Z, size_t N, int nx, int ny,
                   const uint16_t *mk) {
    __shared__ float4 s_tab[NSPAT];
    __shared__ float4 s_yph[4 * 2 * 128];
    __shared__ float4 s_xpt[4][3];
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    constexpr int qx = XT ? 4 : 3, qy = YT ? 4 : 3;
    const EwaldF32 &ef = q.ef;
    const int x = blockIdx.y;
    const float4 *gtab = reinterpret_cast<const float4 *>(q.stab);
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = gtab[i];
    const float *fx = far_el<float, XT>(m, XT ? x : m.hf[x]);
    if (threadIdx.x < qx) {
        const int a = threadIdx.x;
        float4 p, st;
        obl_point_phases(ef, fx[3 * a], fx[3 * a + 1], p, st);
        s_xpt[a][0] = make_float4(fx[3 * a], fx[3 * a + 1], fx[3 * a + 2], 0.f);
        s_xpt[a][1] = p;
        s_xpt[a][2] = st;
    }
    const int y0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = y0 < ny;
    const int y = live ? y0 : ny - 1;
    const float *fy = far_el<float, YT>(m, y);
#pragma unroll
    for (int b = 0; b < qy; ++b) {
        float4 p, st;
        obl_point_phases(ef, fy[3 * b], fy[3 * b + 1], p, st);
        s_yph[256 * b + threadIdx.x] = p;
        s_yph[256 * b + 128 + threadIdx.x] = st;
    }
    float c1[3] = {0.f, 0.f, 0.f}, c2[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < qx; ++a)
        for (int d = 0; d < 3; ++d) c1[d] += fx[3 * a + d] / qx;
    for (int b = 0; b < qy; ++b)
        for (int d = 0; d < 3; ++d) c2[d] += fy[3 * b + d] / qy;
    float r1 = 0.f, r2 = 0.f;
    for (int a = 0; a < qx; ++a) {
        const float ux = fx[3 * a] - c1[0], uy = fx[3 * a + 1] - c1[1], uz = fx[3 * a + 2] - c1[2];
        r1 = fmaxf(r1, sqrtf(ux * ux + uy * uy + uz * uz));
    }
    for (int b = 0; b < qy; ++b) {
        const float ux = fy[3 * b] - c2[0], uy = fy[3 * b + 1] - c2[1], uz = fy[3 * b + 2] - c2[2];
        r2 = fmaxf(r2, sqrtf(ux * ux + uy * uy + uz * uz));
    }
    unsigned long long imask = live ? image_mask(ef, c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2], r1 + r2) : 0ull;
    {
        const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)imask);
        const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(imask >> 32));
        imask = ((unsigned long long)hi << 32) | lo;
    }
    const unsigned sub = live ? (unsigned)mk[(size_t)x * ny + y] : 0u;
    unsigned long long regm = 0ull;
    if (sub) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if ((sub >> k) & 1u) regm |= 1ull << ef.near_img[k];
    }
    const bool reg = __any_sync(0xffffffffu, regm != 0ull);
    __syncthreads();
    if (!live) return;
    cx<float> S = {0.f, 0.f};
#pragma unroll 1
    for (int b = 0; b < qy; ++b) {
        const float yb0 = fy[3 * b], yb1 = fy[3 * b + 1], yb2 = fy[3 * b + 2];
        const float4 pb = s_yph[256 * b + threadIdx.x], sb = s_yph[256 * b + 128 + threadIdx.x];
#pragma unroll 1
        for (int a = 0; a < qx; ++a) {
            const float4 xa = s_xpt[a][0], pa = s_xpt[a][1], sa = s_xpt[a][2];
            cx<float> T;
            const cx<float> g = reg ? green_obl<NR, NQ1, true>(xa.x - yb0, xa.y - yb1, xa.z - yb2, pa, sa, pb, sb,
                                                               imask, regm, s_tab, q.rtab, ef, T)
                                    : green_obl<NR, NQ1, false>(xa.x - yb0, xa.y - yb1, xa.z - yb2, pa, sa, pb, sb,
                                                                imask, 0ull, s_tab, q.rtab, ef, T);
            S = S + g;
        }
    }
    S = (fx[XT ? 27 : 9] * fy[YT ? 27 : 9]) * S;
    scatter_scalar<float, PK>(m, q, Z, N, x, y, S);
}

template <typename U>
__device__ double static_scalar(const double *r5, bool other_tet, const double *verts_other, const double *R,
                                double sgnR) {
    U r[3] = {U(0), U(0), U(0)};   // coordinates relative to the outer point (formed in FP64)
    U inv;
    if (other_tet) {
        U tv[12], vec[3];
        for (int j = 0; j < 4; ++j)
            for (int d = 0; d < 3; ++d) tv[3 * j + d] = U((verts_other[3 * j + d] + sgnR * R[d]) - r5[d]);
        tet_integrals<U>(r, tv, inv, vec, false);
    } else {
        U fv[9], rr;
        for (int j = 0; j < 3; ++j)
            for (int d = 0; d < 3; ++d) fv[3 * j + d] = U((verts_other[3 * j + d] + sgnR * R[d]) - r5[d]);
        tri_integrals<U>(r, fv, inv, rr, false);
    }
    return double(inv);
}

template <typename T, int PK>
__global__ void __launch_bounds__(128) k_pr_scalar(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N, const NearEntry *list,
                                                   int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    const NearEntry en = list[e];
    const int x = en.x, y = en.y, k = en.k;
    const int xf = XT ? x : m.hf[x];
    constexpr int nqx = XT ? 14 : 7, nqy = YT ? 14 : 7;
    const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
    const T *nx = XT ? m.nrel<T>(xf) : m.fnrel<T>(xf);
    const T *ny = YT ? m.nrel<T>(y) : m.fnrel<T>(y);
    const double *cxp = XT ? m.cen + 3 * (size_t)xf : m.fcen + 3 * (size_t)xf;
    const double *cyp = YT ? m.cen + 3 * (size_t)y : m.fcen + 3 * (size_t)y;
    const T dc[3] = {T(cxp[0] - cyp[0] + R[0]), T(cxp[1] - cyp[1] + R[1]), T(cxp[2] - cyp[2])};
    T s0 = 0;
    for (int a = 0; a < nqx; ++a) {
        const T *xa = nx + 4 * a;
        T f0 = 0;
        for (int b = 0; b < nqy; ++b) {
            const T *yb = ny + 4 * b;
            const T dx = xa[0] - yb[0] + dc[0], dy = xa[1] - yb[1] + dc[1], dz = xa[2] - yb[2] + dc[2];
            f0 += yb[3] * rsqrt(dx * dx + dy * dy + dz * dz);
        }
        s0 += xa[3] * f0;
    }
    scatter_scalar<T, PK>(m, q, Z, N, x, y, s0 * cx<T>{T(q.img_ph[2 * k]), T(q.img_ph[2 * k + 1])});
}

// Touching face entries: the static integral, both integration orders
// averaged, summed over the degree-5 points (phase-free, FP64; one warp per
// entry, lanes = the points of the two elements).  Request independent.
template <int PK>
__global__ void __launch_bounds__(128) k_touch_scalar(DevMesh m, const NearEntry *list, int n, double *out) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    const NearEntry en = list[wid];
    const int x = en.x, y = en.y, k = en.k;
    const int xf = XT ? x : m.hf[x];
    const int yf = y;
    constexpr int nqx = XT ? 14 : 7, nqy = YT ? 14 : 7;
    const double *x5 = XT ? m.q5 + (size_t)xf * 42 : m.f5 + (size_t)xf * 21;
    const double *y5 = YT ? m.q5 + (size_t)yf * 42 : m.f5 + (size_t)yf * 21;
    const double mx = XT ? m.vol[xf] : m.farea[xf];
    const double my = YT ? m.vol[yf] : m.farea[yf];
    double acc = 0;
    if (lane < nqx + nqy) {
        const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
        const bool oi = lane < nqx;
        const int qi = oi ? lane : lane - nqx;
        const bool self_tet = oi ? XT : YT;
        const bool other_tet = oi ? YT : XT;
        const int other = oi ? yf : xf;
        const double *r5 = (oi ? x5 : y5) + 3 * qi;
        const double w = (oi ? mx : my) * (self_tet ? c_w5tet[qi] : c_w5tri[qi]);
        const double *vo = other_tet ? m.tv + 12 * (size_t)other : m.fv + 9 * (size_t)other;
        const double I = static_scalar<double>(r5, other_tet, vo, R, oi ? -1.0 : 1.0);
        acc = 0.5 * w * I;
    }
    const double sum = warp_sum(acc);
    if (lane == 0) out[wid] = sum;
}

// scatter the cached static integral of every touching face entry with the
// request's image phase exp(j k_par.R)/(4 pi)
template <typename T, int PK>
__global__ void __launch_bounds__(128) k_touch_apply(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N,
                                                     const NearEntry *list, const double *sc, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const NearEntry en = list[e];
    const double v = sc[e];
    scatter_scalar<T, PK>(m, q, Z, N, en.x, en.y,
                          cx<T>{T(v * q.img_ph[2 * en.k]), T(v * q.img_ph[2 * en.k + 1])});
}

// ---------------------------------------------------------------------------
// local (Gram) term and right-hand side, per tetrahedron
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gram(DevMesh m, const __grid_constant__ DevReq q, T *Z, size_t N) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nt) return;
    const double *P = m.tv + 12 * (size_t)t;
    const double *c = m.cen + 3 * (size_t)t;
    double d[4][3], sq = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) {
            d[i][k] = P[3 * i + k] - c[k];
            sq += d[i][k] * d[i][k];
        }
    const double V = m.vol[t];
    cx<double> ie = ld2(q.ieps + 2 * t);
    for (int i = 0; i < 4; ++i) {
        cx<double> wti = ld2(q.wt + 2 * (4 * t + i));
        for (int j = 0; j < 4; ++j) {
            cx<double> wsj = cconj(ld2(q.wt + 2 * (4 * t + j)));
            double G = V * (sq / 20.0 + d[i][0] * d[j][0] + d[i][1] * d[j][1] + d[i][2] * d[j][2]);
            cx<double> val = (q.coef[4 * t + i] * q.coef[4 * t + j] * G) * ((wti * wsj) * ie);
            atomic_add_c<T>(Z, (size_t)q.row[4 * t + i] * N + q.row[4 * t + j], cx<T>{T(val.re), T(val.im)});
        }
    }
}

__global__ void k_rhs(DevMesh m, const __grid_constant__ DevReq q, double *b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nt) return;
    const double *P = m.tv + 12 * (size_t)t;
    const double *c = m.cen + 3 * (size_t)t;
    const double V = m.vol[t];
    for (int pol = 0; pol < 2; ++pol) {
        const double *pv = q.pol + 3 * pol;
        cx<double> s0 = {0, 0}, s1 = {0, 0};   // sum w e^{..}, sum w ((x-c).p) e^{..}
        for (int k = 0; k < 14; ++k) {
            const double *x = m.q5 + (size_t)t * 42 + 3 * k;
            double ph = -(q.kinc[0] * x[0] + q.kinc[1] * x[1] + q.kinc[2] * x[2]);
            double sn, cs;
            sincos(ph, &sn, &cs);
            double w = V * c_w5tet[k];
            double xp = (x[0] - c[0]) * pv[0] + (x[1] - c[1]) * pv[1] + (x[2] - c[2]) * pv[2];
            s0.re += w * cs; s0.im += w * sn;
            s1.re += w * xp * cs; s1.im += w * xp * sn;
        }
        for (int i = 0; i < 4; ++i) {
            double vp = (P[3 * i] - c[0]) * pv[0] + (P[3 * i + 1] - c[1]) * pv[1] + (P[3 * i + 2] - c[2]) * pv[2];
            cx<double> integ = {s1.re - vp * s0.re, s1.im - vp * s0.im};
            cx<double> val = q.coef[4 * t + i] * (ld2(q.wt + 2 * (4 * t + i)) * integ);
            size_t r = (size_t)q.row[4 * t + i];
            atomicAdd(b + 4 * r + 2 * pol, val.re);
            atomicAdd(b + 4 * r + 2 * pol + 1, val.im);
        }
    }
}

// ---------------------------------------------------------------------------
// checks of the special functions
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_erfcx(const double *u, double *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cx<T> r = erfcx_c<T>(cx<T>{T(u[2 * i]), T(u[2 * i + 1])});
    out[2 * i] = double(r.re);
    out[2 * i + 1] = double(r.im);
}

template <typename T, bool SYM = false>
__global__ void k_green(const double *d, double *out, int n, const float *stab, const float2 *ztab,
                        const EwaldTables *ew, const __grid_constant__ EwaldF32 ef) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cx<T> r = Green<T>::template eval<SYM>(T(d[3 * i]), T(d[3 * i + 1]), T(d[3 * i + 2]), 0u, stab, ztab, ew, ef);
    out[2 * i] = double(r.re);
    out[2 * i + 1] = double(r.im);
}

// the short normal-incidence form at single displacements (every image visited)
template <int PQ>
__global__ void k_green_short(const double *d, double *out, int n, const float *stab, const float2 *ztab,
                              const float4 *rtab, const __grid_constant__ EwaldF32 ef) {
    __shared__ float4 s_tab[NSPAT];
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = reinterpret_cast<const float4 *>(stab)[i];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dx = float(d[3 * i]), dy = float(d[3 * i + 1]), dz = float(d[3 * i + 2]);
    const float2 d1 = {2.f * cospif(ef.step_x * dx * 0.31830988618f), 2.f * cospif(ef.step_y * dy * 0.31830988618f)};
    const unsigned all = ef.n_img >= 32 ? 0xffffffffu : (1u << ef.n_img) - 1u;
    cx<float> r = green_sym_short<PQ, true>(dx, dy, dz, d1, all, 0u, s_tab, rtab, ef);
    out[2 * i] = double(r.re);
    out[2 * i + 1] = double(r.im);
}

// the oblique short form at single displacements (every image visited)
template <int NR, int NQ1>
__global__ void k_green_obl(const double *d, double *out, int n, const float *stab, const float4 *rtab,
                            const __grid_constant__ EwaldF32 ef) {
    __shared__ float4 s_tab[NSPAT];
    for (int i = threadIdx.x; i < NSPAT; i += blockDim.x) s_tab[i] = reinterpret_cast<const float4 *>(stab)[i];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dx = float(d[3 * i]), dy = float(d[3 * i + 1]), dz = float(d[3 * i + 2]);
    float s0, c0, s1, c1, s2, c2, s3, c3;
    sincospif(ef.ob_kx0 * 0.31830988618f * dx, &s0, &c0);
    sincospif(ef.ob_ky0 * 0.31830988618f * dy, &s1, &c1);
    sincospif(ef.step_x * 0.31830988618f * dx, &s2, &c2);
    sincospif(ef.step_y * 0.31830988618f * dy, &s3, &c3);
    const unsigned long long all = ef.n_img >= 64 ? ~0ull : (1ull << ef.n_img) - 1ull;
    cx<float> T;
    // point a at d, point b at the origin: (cos, sin) of the phases of d
    const float4 pa = make_float4(c0, s0, c1, s1), sa = make_float4(c2, s2, c3, s3);
    const float4 pb = make_float4(1.f, 0.f, 1.f, 0.f), sb = make_float4(1.f, 0.f, 1.f, 0.f);
    cx<float> r = green_obl<NR, NQ1, true>(dx, dy, dz, pa, sa, pb, sb, all, 0ull, s_tab, rtab, ef, T);
    out[2 * i] = double(r.re);
    out[2 * i + 1] = double(r.im);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// template variant of the oblique short form: 0-2 the full rectangle of side
// 4, 6, 8; 3-5 the k_y = 0 fold (6 x 3, 8 x 3, 8 x 5)
inline int obl_variant(const EwaldF32 &ef) {
    if (ef.ob_nq1 == 0) return ef.ob_nr == 4 ? 0 : (ef.ob_nr == 6 ? 1 : 2);
    return ef.ob_nq1 == 3 ? (ef.ob_nr == 6 ? 3 : 4) : 5;
}

template <typename T, int PK>
void far_scalar(bool sym, dim3 grid, size_t sm, cudaStream_t st, const DevMesh &m, const DevReq &q, T *Z, size_t N,
                int nx, int ny, const uint16_t *mk) {
    if constexpr (sizeof(T) == 4) {
        if (sym && q.ef.sq_pq > 0) {   // normal incidence, short form
            switch (q.ef.sq_pq) {
                case 1: k_far_scalar_n<1, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 2: k_far_scalar_n<2, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 3: k_far_scalar_n<3, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                default: k_far_scalar_n<4, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
            }
        } else if (!sym && q.ef.ob_nr > 0) {   // oblique incidence, short form
            switch (obl_variant(q.ef)) {
                case 0: k_far_scalar_o<4, 0, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 1: k_far_scalar_o<6, 0, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 2: k_far_scalar_o<8, 0, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 3: k_far_scalar_o<6, 3, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                case 4: k_far_scalar_o<8, 3, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
                default: k_far_scalar_o<8, 5, PK><<<grid, 128, 0, st>>>(m, q, Z, N, nx, ny, mk); break;
            }
        } else if (sym) k_far_scalar<T, PK, true><<<grid, 128, sm, st>>>(m, q, Z, N, nx, ny, mk);
        else k_far_scalar<T, PK, false><<<grid, 128, sm, st>>>(m, q, Z, N, nx, ny, mk);
    } else {
        k_far_scalar<T, PK, false><<<grid, 128, sm, st>>>(m, q, Z, N, nx, ny, mk);
    }
    ++g_launches;
}

template <typename T>
cudaError_t launch_fill(const DevMesh &m, const DevReq &q, T *Z, size_t ld, double *b, cudaStream_t st,
                        cudaEvent_t far0, cudaEvent_t far1) {
    // Z: N rows of ld complex entries (row stride ld >= N), domain-blocked order
    const size_t N = ld;
    cudaMemsetAsync(Z, 0, sizeof(T) * 2 * ld * (size_t)m.N, st);
    if (b) cudaMemsetAsync(b, 0, sizeof(double) * 4 * (size_t)m.N, st);
    dim3 blk(128);
    k_gram<T><<<(m.nt + 127) / 128, blk, 0, st>>>(m, q, Z, N); ++g_launches;
    if (b) { k_rhs<<<(m.nt + 127) / 128, blk, 0, st>>>(m, q, b); ++g_launches; }
    const size_t sm = stab_bytes<T>();
    if (far0) cudaEventRecord(far0, st);
    const bool sym = sizeof(T) == 4 && q.ef.sym;   // normal incidence: the symmetric tabulated path
    if constexpr (sizeof(T) == 4) {
        const dim3 gtt((m.nt + 127) / 128, m.nt);
        if (sym && q.ef.sq_pq > 0) {   // normal incidence, short form
            switch (q.ef.sq_pq) {
                case 1: k_far_tt_n<1><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 2: k_far_tt_n<2><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 3: k_far_tt_n<3><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                default: k_far_tt_n<4><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
            }
        } else if (!sym && q.ef.ob_nr > 0) {   // oblique incidence, short form
            switch (obl_variant(q.ef)) {
                case 0: k_far_tt_o<4, 0><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 1: k_far_tt_o<6, 0><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 2: k_far_tt_o<8, 0><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 3: k_far_tt_o<6, 3><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                case 4: k_far_tt_o<8, 3><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
                default: k_far_tt_o<8, 5><<<gtt, blk, 0, st>>>(m, q, Z, N); break;
            }
        } else if (sym) k_far_tt<T, true><<<gtt, blk, sm, st>>>(m, q, Z, N);
        else k_far_tt<T, false><<<gtt, blk, sm, st>>>(m, q, Z, N);
    } else {
        k_far_tt<T, false><<<dim3((m.nt + 127) / 128, m.nt), blk, sm, st>>>(m, q, Z, N);
    }
    ++g_launches;
    if (far1) cudaEventRecord(far1, st);
    auto grid1 = [](int n) { return (unsigned)((n + 127) / 128); };
    if (m.npr[0]) { k_pr_tt<T><<<grid1(m.npr[0]), blk, 0, st>>>(m, q, Z, N, m.pr[0], m.npr[0]); ++g_launches; }
    if (m.nto[0]) {
        k_touch_combine<T><<<grid1(m.nto[0]), blk, 0, st>>>(m, q, Z, N, m.to[0], m.touch_partner, m.touch_half,
                                                            m.nto[0]); ++g_launches;
    }
    if (m.nf) {
        far_scalar<T, PK_TF>(sym, dim3((m.nf + 127) / 128, m.nt), sm, st, m, q, Z, N, m.nt, m.nf, m.mk_tf);
        if (m.npr[1]) { k_pr_scalar<T, PK_TF><<<grid1(m.npr[1]), blk, 0, st>>>(m, q, Z, N, m.pr[1], m.npr[1]); ++g_launches; }
        if (m.nto[1]) { k_touch_apply<T, PK_TF><<<grid1(m.nto[1]), blk, 0, st>>>(m, q, Z, N, m.to[1], m.touch_sc[1], m.nto[1]); ++g_launches; }
    }
    if (m.nh) {
        far_scalar<T, PK_FT>(sym, dim3((m.nt + 127) / 128, m.nh), sm, st, m, q, Z, N, m.nh, m.nt, m.mk_ft);
        if (m.npr[2]) { k_pr_scalar<T, PK_FT><<<grid1(m.npr[2]), blk, 0, st>>>(m, q, Z, N, m.pr[2], m.npr[2]); ++g_launches; }
        if (m.nto[2]) { k_touch_apply<T, PK_FT><<<grid1(m.nto[2]), blk, 0, st>>>(m, q, Z, N, m.to[2], m.touch_sc[2], m.nto[2]); ++g_launches; }
        far_scalar<T, PK_FF>(sym, dim3((m.nf + 127) / 128, m.nh), sm, st, m, q, Z, N, m.nh, m.nf, m.mk_ff);
        if (m.npr[3]) { k_pr_scalar<T, PK_FF><<<grid1(m.npr[3]), blk, 0, st>>>(m, q, Z, N, m.pr[3], m.npr[3]); ++g_launches; }
        if (m.nto[3]) { k_touch_apply<T, PK_FF><<<grid1(m.nto[3]), blk, 0, st>>>(m, q, Z, N, m.to[3], m.touch_sc[3], m.nto[3]); ++g_launches; }
    }
    return cudaGetLastError();
}

cudaError_t launch_static_cache(const DevMesh &m, double *touch_half, double *const touch_sc[4], cudaStream_t st) {
    const dim3 blk(128);
    auto gridw = [](int n) { return (unsigned)(((size_t)n * 32 + 127) / 128); };
    if (m.nto[0]) {
        k_touch_half<<<(unsigned)(((size_t)(m.nto[0] + 1) / 2 * 32 + 127) / 128), blk, 0, st>>>(m, m.to[0], m.nto[0],
                                                                                              touch_half); ++g_launches;
    }
    if (m.nto[1]) { k_touch_scalar<PK_TF><<<gridw(m.nto[1]), blk, 0, st>>>(m, m.to[1], m.nto[1], touch_sc[1]); ++g_launches; }
    if (m.nto[2]) { k_touch_scalar<PK_FT><<<gridw(m.nto[2]), blk, 0, st>>>(m, m.to[2], m.nto[2], touch_sc[2]); ++g_launches; }
    if (m.nto[3]) { k_touch_scalar<PK_FF><<<gridw(m.nto[3]), blk, 0, st>>>(m, m.to[3], m.nto[3], touch_sc[3]); ++g_launches; }
    return cudaGetLastError();
}

template cudaError_t launch_fill<float>(const DevMesh &, const DevReq &, float *, size_t, double *, cudaStream_t,
                                        cudaEvent_t, cudaEvent_t);
template cudaError_t launch_fill<double>(const DevMesh &, const DevReq &, double *, size_t, double *, cudaStream_t,
                                         cudaEvent_t, cudaEvent_t);

cudaError_t launch_erfcx(const double *u, double *out, int n, bool fp64, cudaStream_t st) {
    if (fp64) { k_erfcx<double><<<(n + 127) / 128, 128, 0, st>>>(u, out, n); ++g_launches; }
    else { k_erfcx<float><<<(n + 127) / 128, 128, 0, st>>>(u, out, n); ++g_launches; }
    return cudaGetLastError();
}

cudaError_t launch_green(const double *d, double *out, int n, bool fp64, const float *stab, const float2 *ztab,
                         const EwaldTables *ew, const EwaldF32 &ef, cudaStream_t st, const float4 *rtab) {
    const unsigned gb = (unsigned)((n + 127) / 128);
    if (fp64) { k_green<double><<<(n + 127) / 128, 128, 0, st>>>(d, out, n, stab, ztab, ew, ef); ++g_launches; }
    else if (ef.sym && ef.sq_pq > 0 && rtab) {   // the fill's normal-incidence form
        switch (ef.sq_pq) {
            case 1: k_green_short<1><<<gb, 128, 0, st>>>(d, out, n, stab, ztab, rtab, ef); break;
            case 2: k_green_short<2><<<gb, 128, 0, st>>>(d, out, n, stab, ztab, rtab, ef); break;
            case 3: k_green_short<3><<<gb, 128, 0, st>>>(d, out, n, stab, ztab, rtab, ef); break;
            default: k_green_short<4><<<gb, 128, 0, st>>>(d, out, n, stab, ztab, rtab, ef); break;
        }
        ++g_launches;
    }
    else if (!ef.sym && ef.ob_nr > 0 && rtab) {   // the fill's oblique form
        switch (obl_variant(ef)) {
            case 0: k_green_obl<4, 0><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
            case 1: k_green_obl<6, 0><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
            case 2: k_green_obl<8, 0><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
            case 3: k_green_obl<6, 3><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
            case 4: k_green_obl<8, 3><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
            default: k_green_obl<8, 5><<<gb, 128, 0, st>>>(d, out, n, stab, rtab, ef); break;
        }
        ++g_launches;
    }
    else if (ef.sym) { k_green<float, true><<<(n + 127) / 128, 128, 0, st>>>(d, out, n, stab, ztab, ew, ef); ++g_launches; }
    else { k_green<float><<<(n + 127) / 128, 128, 0, st>>>(d, out, n, stab, ztab, ew, ef); ++g_launches; }
    return cudaGetLastError();
}

}  // namespace vie

// ===========================================================================
// Allocation-free evaluation of the periodic Green's function.
//
// Some callers cannot allocate device memory while they run: a host framework
// that reserves all of HBM up front through its own pool and forbids
// cudaMalloc/cudaFree afterwards (a long-running serving process, for
// example), or code that must not let an allocation synchronise the device.
// vie_green_noalloc serves them: the caller passes device buffers for the
// inputs and outputs, and the only scratch -- the FP32 interpolation tables of
// the Ewald series -- lives in the file-scope array below, which every GPU
// that loads this library holds until the process exits.
// ===========================================================================
#include <mutex>
#include <vector>

#include "../../include/vie.h"

namespace vie {


constexpr int NOALLOC_MAX_TAB = 96;   // distinct Floquet decay constants the scratch can hold
// whole 16-byte units: the spatial table after it is read with 16-byte loads
constexpr size_t NOALLOC_EW_FLOAT2 = (sizeof(EwaldTables) + 15) / 16 * 2;
constexpr size_t NOALLOC_FLOAT2 = NOALLOC_EW_FLOAT2 + 2 * NSPAT + (size_t)NOALLOC_MAX_TAB * NZTAB * 4;
// Ewald parameter block (~49 KB), spatial table (4*NSPAT floats), spectral tables
// (float2): about 0.85 MB in total
static __device__ __align__(256) float2 g_noalloc_scratch[NOALLOC_FLOAT2];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;                                   // guards the per-device set-up below
float2 *g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};           // device address of the array, per device

}  // namespace
}  // namespace vie

extern "C" int vie_green_noalloc(double lambda_nm, double theta, double phi, double period_a, double period_b,
                                 double z_extent, const double *d_dev, double *out_dev, int32_t n,
                                 int32_t precision, void *stream) {
    using namespace vie;
    if (n < 0 || (n > 0 && (!d_dev || !out_dev))) return VIE_EINVAL;
    if (!(lambda_nm > 0) || !(period_a > 0) || !(period_b > 0) || !(std::fabs(theta) < M_PI / 2) ||
        !(z_extent >= 0) || !std::isfinite(lambda_nm + period_a + period_b + z_extent))
        return VIE_EINVAL;
    if (precision != VIE_FP64 && precision != VIE_FP32) return VIE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return VIE_ECUDA;
    float2 *base = nullptr;
    {
        // one-time set-up per device, with the device current, under one lock
        // across threads: the library's constant tables (the same once-per-device
        // upload that vie_create does, so a device whose solves are running is
        // never written again) and the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_scratch_ptr[dev]) {
            if (upload_device_constants(dev) != cudaSuccess) return VIE_ECUDA;
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VIE_ECUDA;
            g_scratch_ptr[dev] = static_cast<float2 *>(p);
        }
        base = g_scratch_ptr[dev];
    }
    if (n == 0) return VIE_OK;
    static thread_local EwaldTables tabs;
    const double k0 = 2.0 * M_PI / lambda_nm;
    const char *why = "";
    const int rc = build_ewald_tables(period_a, period_b, k0, k0 * std::sin(theta) * std::cos(phi),
                                      k0 * std::sin(theta) * std::sin(phi), z_extent, precision == VIE_FP64, tabs,
                                      nullptr, &why);
    if (rc != VIE_OK) return rc;
    if (precision == VIE_FP32 && tabs.n_tab > NOALLOC_MAX_TAB) return VIE_EINVAL;   // scratch too small
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EwaldTables *ewd = reinterpret_cast<EwaldTables *>(base);
    if (upload_ewald(ewd, tabs, st) != cudaSuccess) return VIE_ECUDA;
    float *stab = reinterpret_cast<float *>(base + NOALLOC_EW_FLOAT2);
    float2 *ztab = base + NOALLOC_EW_FLOAT2 + 2 * NSPAT;
    if (precision == VIE_FP32 && launch_build_tables(ewd, stab, ztab, tabs.n_tab, st) != cudaSuccess) return VIE_ECUDA;
    if (launch_green(d_dev, out_dev, n, precision == VIE_FP64, stab, ztab, ewd, make_ewald_f32(tabs), st) !=
        cudaSuccess)
        return VIE_ECUDA;
    return VIE_OK;
}
