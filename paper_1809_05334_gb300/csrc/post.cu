// Post-processing of the solved unknowns: absorbed fraction per domain
// (Eq. (7)), reflectance and transmittance from the Floquet projection of the
// equivalent current, and the gather of the unknowns into canonical order.
//
// Eq. (7), A = w int Im(eps)|E|^2 dv, is normalised to the incident power:
//   A_d = k0 int_d |Im eps_r| |E|^2 dV / (|E0|^2 a b cos theta),
// with E = d/eps_r linear in each tetrahedron, so int |E|^2 = beta^H G beta with
// the tetrahedron's second-moment matrix G_ij = V(sum_k |v_k-c|^2/20 + (v_i-c).(v_j-c)).
// A propagating order k = (k_t, +-k_z) of the field scattered by J = j w kappa D
// has amplitude E = -j k0^2/(2 a b k_z) (I - k^k^) . int kappa d e^{j k.r} dV.
#include <cuda_runtime.h>

#include "device_math.cuh"
#include "fill.h"
#include "post.h"

namespace vie {

__constant__ double c_w5tet_post[14];

cudaError_t upload_post_constants() {
    double w[14];
    tet_rule5(nullptr, w);
    return cudaMemcpyToSymbol(c_w5tet_post, w, sizeof(w));
}

__device__ __forceinline__ cx<double> ldc(const double *p) { return {p[0], p[1]}; }

// per tetrahedron: beta_i[pol] = x[row(t,i)][pol] * conj(wt) * coef  (d = sum beta_i (r - v_i))
__device__ void tet_beta(const DevMesh &m, const DevReq &q, const double *x, int t, cx<double> beta[2][4]) {
    for (int i = 0; i < 4; ++i) {
        cx<double> ws = cconj(ldc(q.wt + 2 * (4 * t + i)));
        double c = q.coef[4 * t + i];
        size_t r = (size_t)q.row[4 * t + i];
        for (int p = 0; p < 2; ++p) beta[p][i] = c * (ws * ldc(x + 4 * r + 2 * p));
    }
}

// absorbed fraction of tetrahedron t (Eq. (7), normalised), summed per domain
// into acc[p][domain]; also stored per tetrahedron in dens[p][t] if dens is set
__global__ void k_absorb(DevMesh m, DevReq q, const double *x, const int32_t *dom, double *acc,
                         int n_dom, double norm, double *dens) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nt) return;
    cx<double> beta[2][4];
    tet_beta(m, q, x, t, beta);
    const double *P = m.tv + 12 * (size_t)t;
    const double *c = m.cen + 3 * (size_t)t;
    double d[4][3], sq = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) {
            d[i][k] = P[3 * i + k] - c[k];
            sq += d[i][k] * d[i][k];
        }
    const double V = m.vol[t];
    cx<double> ie = ldc(q.ieps + 2 * t);
    // |Im eps_r| = |Im(1/ie)|
    double dd = ie.re * ie.re + ie.im * ie.im;
    double imeps = fabs(-ie.im / dd);
    for (int p = 0; p < 2; ++p) {
        double e2 = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                double G = V * (sq / 20.0 + d[i][0] * d[j][0] + d[i][1] * d[j][1] + d[i][2] * d[j][2]);
                cx<double> bi = ie * beta[p][i], bj = ie * beta[p][j];
                e2 += G * (bi.re * bj.re + bi.im * bj.im);
            }
        const double a_t = norm * imeps * e2;
        atomicAdd(acc + p * n_dom + dom[t], a_t);
        if (dens) dens[(size_t)p * m.nt + t] = a_t;
    }
}

// J[o][s][p][3] += kappa_t sum_q w_q d(x_q) exp(j k_os . x_q)
__global__ void k_project(DevMesh m, DevReq q, const double *x, const double *orders, int n_orders,
                          double *J) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nt) return;
    cx<double> beta[2][4];
    tet_beta(m, q, x, t, beta);
    cx<double> kap = ldc(q.kap + 2 * t);
    const double *P = m.tv + 12 * (size_t)t;
    const double V = m.vol[t];
    for (int o = 0; o < n_orders; ++o) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double kv[3] = {orders[4 * o], orders[4 * o + 1], (sgn == 0 ? 1.0 : -1.0) * orders[4 * o + 2]};
            cx<double> acc[2][3] = {};
            for (int k = 0; k < 14; ++k) {
                const double *xq = m.q5 + (size_t)t * 42 + 3 * k;
                double sn, cs;
                sincos(kv[0] * xq[0] + kv[1] * xq[1] + kv[2] * xq[2], &sn, &cs);
                cx<double> e = {cs * V * c_w5tet_post[k], sn * V * c_w5tet_post[k]};
                for (int p = 0; p < 2; ++p)
                    for (int i = 0; i < 4; ++i) {
                        cx<double> be = beta[p][i] * e;
                        for (int dd = 0; dd < 3; ++dd) acc[p][dd] = acc[p][dd] + (xq[dd] - P[3 * i + dd]) * be;
                    }
            }
            for (int p = 0; p < 2; ++p)
                for (int dd = 0; dd < 3; ++dd) {
                    cx<double> v = kap * acc[p][dd];
                    double *dst = J + (((size_t)o * 2 + sgn) * 2 + p) * 6 + 2 * dd;
                    atomicAdd(dst, v.re);
                    atomicAdd(dst + 1, v.im);
                }
        }
    }
}

// R, T per polarisation from the projected currents (single thread)
__global__ void k_rt(const double *orders, int n_orders, const double *J, double k0, double a, double b,
                     double kz00, const double *pol, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int p = 0; p < 2; ++p) {
        double R = 0, T = 0;
        for (int o = 0; o < n_orders; ++o) {
            const double kz = orders[4 * o + 2];
            const bool zero = orders[4 * o + 3] != 0.0;
            for (int sgn = 0; sgn < 2; ++sgn) {
                const double kv[3] = {orders[4 * o], orders[4 * o + 1], (sgn == 0 ? 1.0 : -1.0) * kz};
                const double *Jp = J + (((size_t)o * 2 + sgn) * 2 + p) * 6;
                cx<double> Jv[3] = {ldc(Jp), ldc(Jp + 2), ldc(Jp + 4)};
                cx<double> kJ = {0, 0};
                for (int d = 0; d < 3; ++d) kJ = kJ + (kv[d] / k0) * Jv[d];
                const double f = k0 * k0 / (2.0 * a * b * kz);
                double pw = 0;
                for (int d = 0; d < 3; ++d) {
                    cx<double> tr = Jv[d] - (kv[d] / k0) * kJ;
                    cx<double> E = {f * tr.im, -f * tr.re};   // -j f tr
                    if (sgn == 1 && zero) E.re += pol[3 * p + d];
                    pw += E.re * E.re + E.im * E.im;
                }
                pw *= kz / kz00;
                if (sgn == 0) R += pw; else T += pw;
            }
        }
        out[2 * p] = R;
        out[2 * p + 1] = T;
    }
}

// out[canonical n][p] = x[perm[n]][p]
__global__ void k_unpermute(const double *x, const int32_t *perm, int n, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *s = x + 4 * (size_t)perm[i];
    double *d = out + 4 * (size_t)i;
    d[0] = s[0]; d[1] = s[1]; d[2] = s[2]; d[3] = s[3];
}

cudaError_t launch_post(const DevMesh &m, const DevReq &q, const double *x, const int32_t *dom, int n_dom,
                        double norm, const double *orders, int n_orders, double a, double b, double kz00,
                        const double *pol_dev, double *acc, double *J, double *rt, double *dens, cudaStream_t st) {
    cudaMemsetAsync(acc, 0, sizeof(double) * 2 * n_dom, st);
    cudaMemsetAsync(J, 0, sizeof(double) * 24 * n_orders, st);
    k_absorb<<<(m.nt + 127) / 128, 128, 0, st>>>(m, q, x, dom, acc, n_dom, norm, dens); ++g_launches;
    k_project<<<(m.nt + 127) / 128, 128, 0, st>>>(m, q, x, orders, n_orders, J); ++g_launches;
    k_rt<<<1, 32, 0, st>>>(orders, n_orders, J, q.k0, a, b, kz00, pol_dev, rt); ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const double *x, const int32_t *perm, int n, double *out, cudaStream_t st) {
    k_unpermute<<<(n + 255) / 256, 256, 0, st>>>(x, perm, n, out); ++g_launches;
    return cudaGetLastError();
}

}  // namespace vie
