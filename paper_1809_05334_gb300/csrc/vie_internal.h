// Internal host/device declarations of the periodic SWG VIE library.
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

namespace vie {

// Near-pair criterion of the discrete problem: a pair of elements is near when,
// for some lattice image (m, n) in {-1,0,1}^2, the distance between centroids
// |c_x - c_y + R_mn| is below NEAR_FACTOR * (rho_x + rho_y), rho = max distance
// from an element's centroid to its vertices (times 1 + NEAR_MARGIN).
constexpr double NEAR_FACTOR = 1.5;
// relative margin so that exact ties (structured meshes) classify as near
// independently of the rounding of the distance
constexpr double NEAR_MARGIN = 1e-9;

}  // namespace vie
struct vie_ctx;
namespace vie {
void release_device_memory(vie_ctx *ctx);
// A flag the solves of ctx poll between phases and at every GMRES iteration;
// once it is non-zero the solve returns VIE_CANCELLED (nullptr: none)
void set_cancel_flag(vie_ctx *ctx, const std::atomic<int> *flag);

// kernel launches issued by this host thread (every launch site increments it;
// a solve reports the difference across its own work)
extern thread_local int64_t g_launches;

enum Kind : int { KIND_INTERIOR = 0, KIND_HALF = 1, KIND_PERIODIC = 2 };

// One near pair: test element x, source element y, bit k of `mask` set when the
// image (m, n) = (k / 3 - 1, k % 3 - 1) is near; `touch` when the elements share
// a vertex through a near image (singular integrand: closed forms in FP64).
struct NearPair {
    int32_t x, y;
    uint16_t mask;
    uint16_t touch;
};

// SWG topology of one mesh (Sec. 2.1 basis, Sec. 2.2 Bloch pairing).
struct Topology {
    int nt = 0, nv = 0, N = 0, n_dom = 0, active = 0;
    double a = 0, b = 0;
    std::vector<double> tv;      // [nt][4][3] tetrahedron vertices
    std::vector<double> vol;     // [nt]
    std::vector<double> cen;     // [nt][3]
    std::vector<double> rad;     // [nt]
    std::vector<double> area;    // [nt][4] area of local face i (opposite vertex i)
    std::vector<int32_t> basis;  // [nt][4] canonical unknown of local face i
    std::vector<int8_t> sgn;     // [nt][4] +1 on T+, -1 on T-
    std::vector<int8_t> shift;   // [nt][4] 0, 1: T- half shifted by (a,0,0), 2: by (0,b,0)
    std::vector<int32_t> dom;    // [nt]
    std::vector<int32_t> kind, tp, ip, tm, im;   // per unknown
    // charge-carrying faces (interface or half functions), geometry at the T+ side
    std::vector<int32_t> cf;     // [nf] unknown id
    std::vector<double> fv;      // [nf][3][3]
    std::vector<double> fcen;    // [nf][3]
    std::vector<double> frad;    // [nf]
    std::vector<int32_t> hf;     // [nh] indices into cf of half functions (surface test)
    std::vector<NearPair> near_tt, near_tf, near_ft, near_ff;
};

// Builds the topology; returns an empty string or an error message.
std::string build_topology(const double *verts, int nv, const int32_t *tets, int nt,
                           const int32_t *tet_domain, int n_dom, double a, double b,
                           int active, Topology &out);

}  // namespace vie
