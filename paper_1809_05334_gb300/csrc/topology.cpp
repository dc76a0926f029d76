// SWG topology and near-pair lists of a periodic tetrahedral unit cell (host).
//
// Schaubert-Wilton-Glisson functions (Sec. 2.1): one unknown per face; interior
// faces carry a full function on T+ and T-, faces on the body's top/bottom carry
// a half function (T+ only), and lateral faces on x=0/x=a (y=0/y=b) are paired
// into one Bloch-periodic function (Sec. 2.2) whose T- half is the image of the
// tetrahedron at the x=a (y=b) wall shifted by (a,0,0) ((0,b,0)).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <map>
#include <tuple>

#include "vie_internal.h"

namespace vie {

namespace {

using Key = std::array<int32_t, 3>;

inline void face_local(int i, int out[3]) {
    int k = 0;
    for (int j = 0; j < 4; ++j)
        if (j != i) out[k++] = j;
}

struct GeoKey {  // rounded sorted coordinates of a lateral face, for wall matching
    std::array<long long, 9> v;
    bool operator<(const GeoKey &o) const { return v < o.v; }
};

GeoKey geo_key(const double *p0, const double *p1, const double *p2, double sx, double sy) {
    std::array<std::array<long long, 3>, 3> q;
    const double *p[3] = {p0, p1, p2};
    for (int i = 0; i < 3; ++i) {
        q[i][0] = std::llround((p[i][0] - sx) * 1e6);
        q[i][1] = std::llround((p[i][1] - sy) * 1e6);
        q[i][2] = std::llround(p[i][2] * 1e6);
    }
    std::sort(q.begin(), q.end());
    GeoKey k;
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) k.v[3 * i + d] = q[i][d];
    return k;
}

double norm3(const double *v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

}  // namespace

std::string build_topology(const double *verts, int nv, const int32_t *tets, int nt,
                           const int32_t *tet_domain, int n_dom, double a, double b,
                           int active, Topology &T) {
    T = Topology();
    T.nt = nt;
    T.nv = nv;
    T.n_dom = n_dom;
    T.a = a;
    T.b = b;
    T.active = active;
    if (nt <= 0 || nv <= 0 || n_dom <= 0 || a <= 0 || b <= 0) return "empty mesh or bad period";
    for (int t = 0; t < nt; ++t) {
        for (int j = 0; j < 4; ++j)
            if (tets[4 * t + j] < 0 || tets[4 * t + j] >= nv) return "tetrahedron vertex out of range";
        if (tet_domain[t] < 0 || tet_domain[t] >= n_dom) return "tetrahedron domain out of range";
    }
    const double tol = 1e-9 * std::max(a, b);

    // geometry
    T.tv.resize(12 * (size_t)nt);
    T.vol.resize(nt);
    T.cen.resize(3 * (size_t)nt);
    T.rad.resize(nt);
    T.area.resize(4 * (size_t)nt);
    T.dom.assign(tet_domain, tet_domain + nt);
    for (int t = 0; t < nt; ++t) {
        double *P = &T.tv[12 * (size_t)t];
        for (int j = 0; j < 4; ++j)
            for (int d = 0; d < 3; ++d) P[3 * j + d] = verts[3 * tets[4 * t + j] + d];
        double e1[3], e2[3], e3[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = P[3 + d] - P[d];
            e2[d] = P[6 + d] - P[d];
            e3[d] = P[9 + d] - P[d];
        }
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double v = (cr[0] * e3[0] + cr[1] * e3[1] + cr[2] * e3[2]) / 6.0;
        if (!(v > 0)) return "tetrahedron " + std::to_string(t) + " is not positively oriented";
        T.vol[t] = v;
        for (int d = 0; d < 3; ++d) T.cen[3 * t + d] = 0.25 * (P[d] + P[3 + d] + P[6 + d] + P[9 + d]);
        double r = 0;
        for (int j = 0; j < 4; ++j) {
            double dv[3] = {P[3 * j] - T.cen[3 * t], P[3 * j + 1] - T.cen[3 * t + 1], P[3 * j + 2] - T.cen[3 * t + 2]};
            r = std::max(r, norm3(dv));
        }
        T.rad[t] = r;
        for (int i = 0; i < 4; ++i) {
            int l[3];
            face_local(i, l);
            double f1[3], f2[3];
            for (int d = 0; d < 3; ++d) {
                f1[d] = P[3 * l[1] + d] - P[3 * l[0] + d];
                f2[d] = P[3 * l[2] + d] - P[3 * l[0] + d];
            }
            double c[3] = {f1[1] * f2[2] - f1[2] * f2[1], f1[2] * f2[0] - f1[0] * f2[2], f1[0] * f2[1] - f1[1] * f2[0]};
            T.area[4 * t + i] = 0.5 * norm3(c);
        }
    }

    // faces and owners
    std::map<Key, std::vector<std::pair<int, int>>> owners;
    for (int t = 0; t < nt; ++t)
        for (int i = 0; i < 4; ++i) {
            int l[3];
            face_local(i, l);
            Key k = {tets[4 * t + l[0]], tets[4 * t + l[1]], tets[4 * t + l[2]]};
            std::sort(k.begin(), k.end());
            owners[k].push_back({t, i});
        }
    for (auto &kv : owners)
        if (kv.second.size() > 2) return "a face is shared by more than two tetrahedra";

    auto wall = [&](const Key &k) -> int {  // 0 x0, 1 xa, 2 y0, 3 yb, -1 none
        bool all[4] = {true, true, true, true};
        for (int j = 0; j < 3; ++j) {
            const double *p = verts + 3 * k[j];
            all[0] &= std::fabs(p[0]) < tol;
            all[1] &= std::fabs(p[0] - a) < tol;
            all[2] &= std::fabs(p[1]) < tol;
            all[3] &= std::fabs(p[1] - b) < tol;
        }
        for (int w = 0; w < 4; ++w)
            if (all[w]) return w;
        return -1;
    };
    // periodic pairing: face on the low wall <-> face on the high wall
    std::map<Key, std::pair<Key, int>> partner;  // key -> (other key, axis 1=x 2=y)
    std::map<Key, bool> is_high;
    for (int axis = 0; axis < 2; ++axis) {
        std::map<GeoKey, Key> lo, hi;
        for (auto &kv : owners) {
            if (kv.second.size() != 1) continue;
            int w = wall(kv.first);
            const double *p0 = verts + 3 * kv.first[0], *p1 = verts + 3 * kv.first[1], *p2 = verts + 3 * kv.first[2];
            if (w == 2 * axis) lo[geo_key(p0, p1, p2, 0, 0)] = kv.first;
            if (w == 2 * axis + 1) hi[geo_key(p0, p1, p2, axis == 0 ? a : 0, axis == 1 ? b : 0)] = kv.first;
        }
        if (lo.size() != hi.size()) return "periodic walls do not match";
        for (auto &kv : lo) {
            auto it = hi.find(kv.first);
            if (it == hi.end()) return "periodic walls do not match";
            partner[kv.second] = {it->second, axis + 1};
            partner[it->second] = {kv.second, axis + 1};
            is_high[it->second] = true;
        }
    }

    T.basis.assign(4 * (size_t)nt, -1);
    T.sgn.assign(4 * (size_t)nt, 0);
    T.shift.assign(4 * (size_t)nt, 0);
    for (int t = 0; t < nt; ++t)
        for (int i = 0; i < 4; ++i) {
            if (T.basis[4 * t + i] >= 0) continue;
            int l[3];
            face_local(i, l);
            Key k = {tets[4 * t + l[0]], tets[4 * t + l[1]], tets[4 * t + l[2]]};
            std::sort(k.begin(), k.end());
            auto &own = owners[k];
            int n = (int)T.kind.size();
            if (own.size() == 2) {
                auto p = std::min(own[0], own[1]), m = std::max(own[0], own[1]);
                T.kind.push_back(KIND_INTERIOR);
                T.tp.push_back(p.first); T.ip.push_back(p.second);
                T.tm.push_back(m.first); T.im.push_back(m.second);
                T.basis[4 * p.first + p.second] = n; T.sgn[4 * p.first + p.second] = 1;
                T.basis[4 * m.first + m.second] = n; T.sgn[4 * m.first + m.second] = -1;
            } else if (partner.count(k)) {
                auto pr = partner[k];
                Key klo = is_high.count(k) ? pr.first : k;
                Key khi = is_high.count(k) ? k : pr.first;
                auto p = owners[klo][0], m = owners[khi][0];
                T.kind.push_back(KIND_PERIODIC);
                T.tp.push_back(p.first); T.ip.push_back(p.second);
                T.tm.push_back(m.first); T.im.push_back(m.second);
                T.basis[4 * p.first + p.second] = n; T.sgn[4 * p.first + p.second] = 1;
                T.basis[4 * m.first + m.second] = n; T.sgn[4 * m.first + m.second] = -1;
                T.shift[4 * m.first + m.second] = (int8_t)pr.second;
            } else {
                T.kind.push_back(KIND_HALF);
                T.tp.push_back(t); T.ip.push_back(i);
                T.tm.push_back(-1); T.im.push_back(-1);
                T.basis[4 * t + i] = n; T.sgn[4 * t + i] = 1;
            }
        }
    T.N = (int)T.kind.size();

    // charge-carrying faces: half functions and faces between two domains
    for (int n = 0; n < T.N; ++n) {
        bool charge = T.kind[n] == KIND_HALF || T.dom[T.tp[n]] != T.dom[T.tm[n]];
        if (!charge) continue;
        int idx = (int)T.cf.size();
        T.cf.push_back(n);
        if (T.kind[n] == KIND_HALF) T.hf.push_back(idx);
        int l[3];
        face_local(T.ip[n], l);
        const double *P = &T.tv[12 * (size_t)T.tp[n]];
        double c[3] = {0, 0, 0};
        for (int j = 0; j < 3; ++j)
            for (int d = 0; d < 3; ++d) {
                T.fv.push_back(P[3 * l[j] + d]);
                c[d] += P[3 * l[j] + d] / 3.0;
            }
        for (int d = 0; d < 3; ++d) T.fcen.push_back(c[d]);
        double r = 0;
        for (int j = 0; j < 3; ++j) {
            double dv[3] = {P[3 * l[j]] - c[0], P[3 * l[j] + 1] - c[1], P[3 * l[j] + 2] - c[2]};
            r = std::max(r, norm3(dv));
        }
        T.frad.push_back(r);
    }

    // near-pair lists: for every x and image R_k, the y whose centroid lies
    // within NEAR_FACTOR (rho_x + rho_y) of c_x + R_k, found through a uniform
    // bucket grid over the y centroids (cell size NEAR_FACTOR * 2 max rho_y)
    auto near_list = [&](int nx, const double *cx, const double *rx, const double *vx, int kvx,
                         int ny, const double *cy, const double *ry, const double *vy, int kvy,
                         std::vector<NearPair> &out) {
        double rymax = 0, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int j = 0; j < ny; ++j) {
            rymax = std::max(rymax, ry[j]);
            for (int q = 0; q < 3; ++q) {
                lo[q] = std::min(lo[q], cy[3 * j + q]);
                hi[q] = std::max(hi[q], cy[3 * j + q]);
            }
        }
        const double hcell = std::max(2.0 * NEAR_FACTOR * rymax, 1e-9);
        int nc[3];
        for (int q = 0; q < 3; ++q) nc[q] = std::max(1, std::min(512, (int)std::ceil((hi[q] - lo[q]) / hcell) + 1));
        auto cell_of = [&](double v, int q) {
            return std::min(nc[q] - 1, std::max(0, (int)std::floor((v - lo[q]) / hcell)));
        };
        // counting sort of the y into cells
        std::vector<int> start((size_t)nc[0] * nc[1] * nc[2] + 1, 0), items(ny);
        std::vector<int> cid(ny);
        for (int j = 0; j < ny; ++j) {
            cid[j] = (cell_of(cy[3 * j], 0) * nc[1] + cell_of(cy[3 * j + 1], 1)) * nc[2] + cell_of(cy[3 * j + 2], 2);
            start[cid[j] + 1]++;
        }
        for (size_t c = 1; c < start.size(); ++c) start[c] += start[c - 1];
        {
            std::vector<int> fill(start.begin(), start.end() - 1);
            for (int j = 0; j < ny; ++j) items[fill[cid[j]]++] = j;
        }
        // per-x lists, concatenated in x order (each sorted by y)
        std::vector<std::vector<NearPair>> per(nx);
        #pragma omp parallel
        {
            std::vector<uint16_t> mk(ny, 0), tc(ny, 0);
            std::vector<int> hit;
            #pragma omp for schedule(dynamic, 16)
            for (int i = 0; i < nx; ++i) {
                hit.clear();
                const double reach = NEAR_FACTOR * (rx[i] + rymax) * (1.0 + NEAR_MARGIN);
                for (int k = 0; k < 9; ++k) {
                    const double R[3] = {(k / 3 - 1) * a, (k % 3 - 1) * b, 0.0};
                    const double p[3] = {cx[3 * i] + R[0], cx[3 * i + 1] + R[1], cx[3 * i + 2]};
                    int c0[3], c1[3];
                    bool empty = false;
                    for (int q = 0; q < 3; ++q) {
                        if (p[q] + reach < lo[q] - hcell || p[q] - reach > hi[q] + hcell) empty = true;
                        c0[q] = cell_of(p[q] - reach, q);
                        c1[q] = cell_of(p[q] + reach, q);
                    }
                    if (empty) continue;
                    for (int u = c0[0]; u <= c1[0]; ++u)
                        for (int v = c0[1]; v <= c1[1]; ++v)
                            for (int w = c0[2]; w <= c1[2]; ++w) {
                                const int c = (u * nc[1] + v) * nc[2] + w;
                                for (int e = start[c]; e < start[c + 1]; ++e) {
                                    const int j = items[e];
                                    const double lim = NEAR_FACTOR * (rx[i] + ry[j]) * (1.0 + NEAR_MARGIN);
                                    double d[3];
                                    for (int q = 0; q < 3; ++q) d[q] = cx[3 * i + q] - cy[3 * j + q] + R[q];
                                    if (!(norm3(d) < lim)) continue;
                                    if (!mk[j]) hit.push_back(j);
                                    mk[j] |= (uint16_t)(1u << k);
                                    // shared vertex with the image y - R ?
                                    bool t = false;
                                    for (int pp = 0; pp < kvx && !t; ++pp)
                                        for (int s2 = 0; s2 < kvy; ++s2) {
                                            double ev[3];
                                            for (int q = 0; q < 3; ++q)
                                                ev[q] = vx[(size_t)kvx * 3 * i + 3 * pp + q] -
                                                        (vy[(size_t)kvy * 3 * j + 3 * s2 + q] - R[q]);
                                            if (norm3(ev) < tol) { t = true; break; }
                                        }
                                    if (t) tc[j] |= (uint16_t)(1u << k);
                                }
                            }
                }
                std::sort(hit.begin(), hit.end());
                per[i].reserve(hit.size());
                for (int j : hit) {
                    per[i].push_back({i, j, mk[j], tc[j]});
                    mk[j] = 0;
                    tc[j] = 0;
                }
            }
        }
        size_t tot = 0;
        for (auto &v : per) tot += v.size();
        out.clear();
        out.reserve(tot);
        for (auto &v : per) out.insert(out.end(), v.begin(), v.end());
    };
    int nf = (int)T.cf.size(), nh = (int)T.hf.size();
    std::vector<double> hcen(3 * (size_t)nh), hrad(nh), hv(9 * (size_t)nh);
    for (int h = 0; h < nh; ++h) {
        int f = T.hf[h];
        for (int d = 0; d < 3; ++d) hcen[3 * h + d] = T.fcen[3 * f + d];
        hrad[h] = T.frad[f];
        for (int d = 0; d < 9; ++d) hv[9 * h + d] = T.fv[9 * f + d];
    }
    near_list(nt, T.cen.data(), T.rad.data(), T.tv.data(), 4, nt, T.cen.data(), T.rad.data(), T.tv.data(), 4, T.near_tt);
    if (nf) near_list(nt, T.cen.data(), T.rad.data(), T.tv.data(), 4, nf, T.fcen.data(), T.frad.data(), T.fv.data(), 3, T.near_tf);
    if (nh) near_list(nh, hcen.data(), hrad.data(), hv.data(), 3, nt, T.cen.data(), T.rad.data(), T.tv.data(), 4, T.near_ft);
    if (nh && nf) near_list(nh, hcen.data(), hrad.data(), hv.data(), 3, nf, T.fcen.data(), T.frad.data(), T.fv.data(), 3, T.near_ff);
    return "";
}

}  // namespace vie
