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

#include <cmath>
#include <cstdio>
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

cudaError_t upload_ewald(const EwaldTables &t, cudaStream_t st) {
    return cudaMemcpyToSymbolAsync(c_ew, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st);
}

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

__device__ __forceinline__ bool bit_set(const uint32_t *bm, size_t i) { return (bm[i >> 5] >> (i & 31)) & 1u; }

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
// far tetrahedron pairs
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_far_tt(DevMesh m, DevReq q, T *Z, size_t N) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (s >= m.nt) return;
    if (bit_set(m.bm_tt, (size_t)t * m.nt + s)) return;
    const T *ft = m.far<T>(t);
    const T *fs = m.far<T>(s);
    Mom<T> mo;
    mo.zero();
    const T wgt = ft[27] * fs[27];
    for (int a = 0; a < 4; ++a) {
        const T xa[3] = {ft[3 * a], ft[3 * a + 1], ft[3 * a + 2]};
        const T ra[3] = {xa[0] - ft[12], xa[1] - ft[13], xa[2] - ft[14]};
        for (int b = 0; b < 4; ++b) {
            const T yb[3] = {fs[3 * b], fs[3 * b + 1], fs[3 * b + 2]};
            const T rb[3] = {yb[0] - fs[12], yb[1] - fs[13], yb[2] - fs[14]};
            cx<T> g = green_p<T>(xa[0] - yb[0], xa[1] - yb[1], xa[2] - yb[2], 0u);
            g = wgt * g;
            mo.S = mo.S + g;
            for (int d = 0; d < 3; ++d) {
                mo.A[d] = mo.A[d] + ra[d] * g;
                mo.B[d] = mo.B[d] + rb[d] * g;
            }
            mo.C = mo.C + (ra[0] * rb[0] + ra[1] * rb[1] + ra[2] * rb[2]) * g;
        }
    }
    scatter_tt<T>(m, q, Z, N, t, s, mo);
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

template <typename T>
__global__ void __launch_bounds__(128) k_near_tt(DevMesh m, DevReq q, T *Z, size_t N,
                                                 const NearPair *list, int n) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;
    const NearPair pr = list[wid];
    const int t = pr.x, s = pr.y;
    Mom<double> acc;
    acc.zero();
    if (lane < 28) {
        const bool oi = lane < 14;
        const int qi = oi ? lane : lane - 14;
        const int self = oi ? t : s, other = oi ? s : t;
        const double *r5 = m.q5 + (size_t)self * 42 + 3 * qi;
        const double w = m.vol[self] * c_w5tet[qi];
        for (int k = 0; k < 9; ++k) {
            if (!((pr.mask >> k) & 1u)) continue;
            const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
            double sp, cp;
            sincos(q.kx * R[0] + q.ky * R[1], &sp, &cp);
            const double f = 0.5 / (4.0 * M_PI);
            cx<double> ph = {f * cp, f * sp};
            // order (i): source image y - R; order (ii): test image x + R
            const double sg = oi ? -1.0 : 1.0;
            if ((pr.touch >> k) & 1u)
                static_tt_term<double>(r5, w, m.tv + 12 * (size_t)other, R, sg, m.cen + 3 * self,
                                       m.cen + 3 * other, oi, ph, acc);
            else
                static_tt_term<T>(r5, w, m.tv + 12 * (size_t)other, R, sg, m.cen + 3 * self,
                                  m.cen + 3 * other, oi, ph, acc);
        }
    }
    if (lane < 16) {
        const T *ft = m.far<T>(t);
        const T *fs = m.far<T>(s);
        const int a = lane >> 2, b = lane & 3;
        const T xa[3] = {ft[3 * a], ft[3 * a + 1], ft[3 * a + 2]};
        const T yb[3] = {fs[3 * b], fs[3 * b + 1], fs[3 * b + 2]};
        cx<T> g = green_p<T>(xa[0] - yb[0], xa[1] - yb[1], xa[2] - yb[2], pr.mask);
        const double wg = double(ft[27]) * double(fs[27]);
        cx<double> gd = {wg * double(g.re), wg * double(g.im)};
        double ra[3], rb[3];
        for (int d = 0; d < 3; ++d) {
            ra[d] = double(xa[d]) - double(ft[12 + d]);
            rb[d] = double(yb[d]) - double(fs[12 + d]);
        }
        acc.S = acc.S + gd;
        for (int d = 0; d < 3; ++d) {
            acc.A[d] = acc.A[d] + ra[d] * gd;
            acc.B[d] = acc.B[d] + rb[d] * gd;
        }
        acc.C = acc.C + (ra[0] * rb[0] + ra[1] * rb[1] + ra[2] * rb[2]) * gd;
    }
    double v[16] = {acc.S.re, acc.S.im, acc.C.re, acc.C.im,
                    acc.A[0].re, acc.A[0].im, acc.A[1].re, acc.A[1].im, acc.A[2].re, acc.A[2].im,
                    acc.B[0].re, acc.B[0].im, acc.B[1].re, acc.B[1].im, acc.B[2].re, acc.B[2].im};
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

template <typename T, int PK>
__global__ void __launch_bounds__(128) k_far_scalar(DevMesh m, DevReq q, T *Z, size_t N, int nx, int ny,
                                                    const uint32_t *bm) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (y >= ny) return;
    if (bit_set(bm, (size_t)x * ny + y)) return;
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    // a test face is addressed by its half-function index; geometry by charge-face index
    const T *fx = far_el<T, XT>(m, XT ? x : m.hf[x]);
    const T *fy = far_el<T, YT>(m, y);
    const int qx = XT ? 4 : 3, qy = YT ? 4 : 3;
    const T wgt = fx[XT ? 27 : 9] * fy[YT ? 27 : 9];
    cx<T> S = {0, 0};
    for (int a = 0; a < qx; ++a)
        for (int b = 0; b < qy; ++b) {
            cx<T> g = green_p<T>(fx[3 * a] - fy[3 * b], fx[3 * a + 1] - fy[3 * b + 1], fx[3 * a + 2] - fy[3 * b + 2], 0u);
            S = S + g;
        }
    S = wgt * S;
    scatter_scalar<T, PK>(m, q, Z, N, x, y, S);
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
__global__ void __launch_bounds__(128) k_near_scalar(DevMesh m, DevReq q, T *Z, size_t N,
                                                     const NearPair *list, int n) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;
    constexpr bool XT = PKTraits<PK>::xtet, YT = PKTraits<PK>::ytet;
    const NearPair pr = list[wid];
    const int x = pr.x, y = pr.y;
    // face elements are addressed through the charge-face index
    const int xf = XT ? x : m.hf[x];
    const int yf = y;
    const int nqx = XT ? 14 : 7, nqy = YT ? 14 : 7;
    cx<double> acc = {0, 0};
    if (lane < nqx + nqy) {
        const bool oi = lane < nqx;
        const int qi = oi ? lane : lane - nqx;
        const bool self_tet = oi ? XT : YT;
        const int self = oi ? (XT ? x : xf) : (YT ? y : yf);
        const bool other_tet = oi ? YT : XT;
        const int other = oi ? (YT ? y : yf) : (XT ? x : xf);
        const double *r5 = self_tet ? m.q5 + (size_t)self * 42 + 3 * qi : m.f5 + (size_t)self * 21 + 3 * qi;
        const double w = self_tet ? m.vol[self] * c_w5tet[qi] : m.farea[self] * c_w5tri[qi];
        const double *vo = other_tet ? m.tv + 12 * (size_t)other : m.fv + 9 * (size_t)other;
        for (int k = 0; k < 9; ++k) {
            if (!((pr.mask >> k) & 1u)) continue;
            const double R[3] = {(k / 3 - 1) * m.a, (k % 3 - 1) * m.b, 0.0};
            double sp, cp;
            sincos(q.kx * R[0] + q.ky * R[1], &sp, &cp);
            const double f = 0.5 * w / (4.0 * M_PI);
            const double sg = oi ? -1.0 : 1.0;
            double I = ((pr.touch >> k) & 1u) ? static_scalar<double>(r5, other_tet, vo, R, sg)
                                              : static_scalar<T>(r5, other_tet, vo, R, sg);
            acc.re += f * cp * I;
            acc.im += f * sp * I;
        }
    }
    const int qx = XT ? 4 : 3, qy = YT ? 4 : 3;
    if (lane < qx * qy) {
        const T *fx = far_el<T, XT>(m, xf);
        const T *fy = far_el<T, YT>(m, yf);
        const int a = lane / qy, b = lane % qy;
        cx<T> g = green_p<T>(fx[3 * a] - fy[3 * b], fx[3 * a + 1] - fy[3 * b + 1], fx[3 * a + 2] - fy[3 * b + 2], pr.mask);
        const double wg = double(fx[XT ? 27 : 9]) * double(fy[YT ? 27 : 9]);
        acc.re += wg * double(g.re);
        acc.im += wg * double(g.im);
    }
    double sr = warp_sum(acc.re), si = warp_sum(acc.im);
    if (lane == 0) scatter_scalar<T, PK>(m, q, Z, N, x, y, cx<T>{T(sr), T(si)});
}

// ---------------------------------------------------------------------------
// local (Gram) term and right-hand side, per tetrahedron
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gram(DevMesh m, DevReq q, T *Z, size_t N) {
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

__global__ void k_rhs(DevMesh m, DevReq q, double *b) {
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

template <typename T>
__global__ void k_green(const double *d, double *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cx<T> r = green_p<T>(T(d[3 * i]), T(d[3 * i + 1]), T(d[3 * i + 2]), 0u);
    out[2 * i] = double(r.re);
    out[2 * i + 1] = double(r.im);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_fill(const DevMesh &m, const DevReq &q, T *Z, size_t ld, double *b, cudaStream_t st,
                        cudaEvent_t far0, cudaEvent_t far1) {
    // Z: N rows of ld complex entries (row stride ld >= N), domain-blocked order
    const size_t N = ld;
    cudaMemsetAsync(Z, 0, sizeof(T) * 2 * ld * (size_t)m.N, st);
    if (b) cudaMemsetAsync(b, 0, sizeof(double) * 4 * (size_t)m.N, st);
    dim3 blk(128);
    k_gram<T><<<(m.nt + 127) / 128, blk, 0, st>>>(m, q, Z, N);
    if (b) k_rhs<<<(m.nt + 127) / 128, blk, 0, st>>>(m, q, b);
    if (far0) cudaEventRecord(far0, st);
    k_far_tt<T><<<dim3((m.nt + 127) / 128, m.nt), blk, 0, st>>>(m, q, Z, N);
    if (far1) cudaEventRecord(far1, st);
    if (m.n_tt) k_near_tt<T><<<(m.n_tt * 32 + 127) / 128, blk, 0, st>>>(m, q, Z, N, m.near_tt, m.n_tt);
    if (m.nf) {
        k_far_scalar<T, PK_TF><<<dim3((m.nf + 127) / 128, m.nt), blk, 0, st>>>(m, q, Z, N, m.nt, m.nf, m.bm_tf);
        if (m.n_tf) k_near_scalar<T, PK_TF><<<(m.n_tf * 32 + 127) / 128, blk, 0, st>>>(m, q, Z, N, m.near_tf, m.n_tf);
    }
    if (m.nh) {
        k_far_scalar<T, PK_FT><<<dim3((m.nt + 127) / 128, m.nh), blk, 0, st>>>(m, q, Z, N, m.nh, m.nt, m.bm_ft);
        if (m.n_ft) k_near_scalar<T, PK_FT><<<(m.n_ft * 32 + 127) / 128, blk, 0, st>>>(m, q, Z, N, m.near_ft, m.n_ft);
        k_far_scalar<T, PK_FF><<<dim3((m.nf + 127) / 128, m.nh), blk, 0, st>>>(m, q, Z, N, m.nh, m.nf, m.bm_ff);
        if (m.n_ff) k_near_scalar<T, PK_FF><<<(m.n_ff * 32 + 127) / 128, blk, 0, st>>>(m, q, Z, N, m.near_ff, m.n_ff);
    }
    return cudaGetLastError();
}

template cudaError_t launch_fill<float>(const DevMesh &, const DevReq &, float *, size_t, double *, cudaStream_t,
                                        cudaEvent_t, cudaEvent_t);
template cudaError_t launch_fill<double>(const DevMesh &, const DevReq &, double *, size_t, double *, cudaStream_t,
                                         cudaEvent_t, cudaEvent_t);

cudaError_t launch_erfcx(const double *u, double *out, int n, bool fp64, cudaStream_t st) {
    if (fp64) k_erfcx<double><<<(n + 127) / 128, 128, 0, st>>>(u, out, n);
    else k_erfcx<float><<<(n + 127) / 128, 128, 0, st>>>(u, out, n);
    return cudaGetLastError();
}

cudaError_t launch_green(const double *d, double *out, int n, bool fp64, cudaStream_t st) {
    if (fp64) k_green<double><<<(n + 127) / 128, 128, 0, st>>>(d, out, n);
    else k_green<float><<<(n + 127) / 128, 128, 0, st>>>(d, out, n);
    return cudaGetLastError();
}

}  // namespace vie
