// Device-side views of the mesh and of one request, shared by the fill,
// post-processing and API translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "ewald_params.h"
#include "ewald_tables.h"
#include "vie_internal.h"

namespace vie {

// one near image k (= 3(m+1) + (n+1)) of the element pair (x, y)
struct NearEntry {
    int32_t x, y, k, pad;
};

struct DevMesh {
    int nt, N, nf, nh;
    double a, b;
    const double *tv;      // [nt][12] vertices
    const double *cen;     // [nt][3]
    const double *vol;     // [nt]
    const double *q5;      // [nt][14][3] degree-5 points
    const float *n32;      // [nt][14][4]: degree-5 point minus centroid, vol * weight
    const double *n64;
    const float *fn32;     // [nf][7][4]: degree-5 point minus face centroid, area * weight
    const double *fn64;
    const double *fcen;    // [nf][3] charge-face centroids
    const float *far32;    // [nt][28]: 4 points, centroid, v_i - c (4x3), weight vol/4
    const double *far64;
    const double *fv;      // [nf][9] charge-face vertices
    const double *f5;      // [nf][7][3] degree-5 points
    const double *farea;   // [nf]
    const float *ffar32;   // [nf][12]: 3 points, weight area/3, pad
    const double *ffar64;
    const int32_t *hf;     // [nh] charge-face index of each half function
    // per pair of elements (x-major): 9-bit mask of the near images
    const uint16_t *mk_tt, *mk_tf, *mk_ft, *mk_ff;
    // near (pair, image) entries, kinds 0 tet-tet, 1 tet-face, 2 face-tet, 3 face-face:
    // pr = elements not touching (product rule), to = touching (closed forms)
    const NearEntry *pr[4], *to[4];
    int npr[4], nto[4];
    const int32_t *touch_partner;   // [nto[0]] index of the entry (y, x, 8-k)
    // static (phase-free) integrals of the touching near images, a property of
    // the mesh alone: computed once by launch_static_cache, read by every fill
    const double *touch_half;       // [nto[0]][8] one integration order per tetrahedron entry
    const double *touch_sc[4];      // [nto[i]] (i = 1..3) summed static integral of a face entry

    template <typename T> __device__ const T *far(int t) const;
    template <typename T> __device__ const T *ffar(int f) const;
    template <typename T> __device__ const T *nrel(int t) const;
    template <typename T> __device__ const T *fnrel(int f) const;
};
template <> __device__ inline const float *DevMesh::far<float>(int t) const { return far32 + 28 * (size_t)t; }
template <> __device__ inline const double *DevMesh::far<double>(int t) const { return far64 + 28 * (size_t)t; }
template <> __device__ inline const float *DevMesh::ffar<float>(int f) const { return ffar32 + 12 * (size_t)f; }
template <> __device__ inline const double *DevMesh::ffar<double>(int f) const { return ffar64 + 12 * (size_t)f; }
template <> __device__ inline const float *DevMesh::nrel<float>(int t) const { return n32 + 56 * (size_t)t; }
template <> __device__ inline const double *DevMesh::nrel<double>(int t) const { return n64 + 56 * (size_t)t; }
template <> __device__ inline const float *DevMesh::fnrel<float>(int f) const { return fn32 + 28 * (size_t)f; }
template <> __device__ inline const double *DevMesh::fnrel<double>(int f) const { return fn64 + 28 * (size_t)f; }

struct DevReq {
    double k0, kx, ky;
    double kinc[3];        // incident wavevector (k_par, -k0 cos theta)
    double pol[6];         // TE and TM unit polarisations
    const int32_t *row;    // [nt*4] matrix row (domain-blocked order) of local face (t,i)
    const double *coef;    // [nt*4] sgn * area / (3 vol)
    const double *wt;      // [nt*4][2] test weight exp(+j k_par.s) (source weight = conjugate)
    const double *kap;     // [nt][2] kappa = 1 - 1/eps_r (exp(j w t) convention)
    const double *ieps;    // [nt][2] 1/eps_r
    const int32_t *frow;   // [nf] matrix row of each charge face's unknown
    const double *qs;      // [nf][2] surface charge kappa- - kappa+ (kappa- = 0 for half)
    double img_ph[18];     // exp(j k_par.R_k)/(4 pi) of the near images k = 0..8
    const float *stab;     // FP32 tables of the Ewald series (built per request)
    const float2 *ztab;
    const float4 *rtab;    // real parts of ztab (16 bytes per interval), read for the real tables
    const EwaldTables *ew; // Ewald parameters of the request (device memory)
    EwaldF32 ef;           // FP32 inner-loop parameters (kernel parameter space)
};

// degree-5 rules: barycentric points [14][4] / [7][3] (may be null) and weights
void tet_rule5(double (*pts)[4], double *w);
void tri_rule5(double (*pts)[3], double *w);
void tet_rule2(double (*pts)[4], double *w);
void tri_rule2(double (*pts)[3], double *w);

cudaError_t upload_constants();
// The library's constant tables (quadrature weights, Faddeeva coefficients)
// written to `device` (the current device) once per process under a lock:
// later calls return at once, so constant memory that running solves read is
// never written again.  Returns the CUDA error of the first upload, if any.
cudaError_t upload_device_constants(int device);
// build_ewald_tables: ewald_tables.h
cudaError_t upload_ewald(EwaldTables *dev, const EwaldTables &t, cudaStream_t st);
template <typename T>
cudaError_t launch_fill(const DevMesh &m, const DevReq &q, T *Z, size_t ld, double *b, cudaStream_t st,
                        cudaEvent_t far0 = nullptr, cudaEvent_t far1 = nullptr);
// the request-independent static integrals of the touching near images:
// touch_half [nto[0]][8] and touch_sc[i] [nto[i]] (i = 1..3)
cudaError_t launch_static_cache(const DevMesh &m, double *touch_half, double *const touch_sc[4], cudaStream_t st);
cudaError_t launch_erfcx(const double *u, double *out, int n, bool fp64, cudaStream_t st);
// rtab (optional): the real spectral tables; with it, normal incidence takes the fill's short form
cudaError_t launch_green(const double *d, double *out, int n, bool fp64, const float *stab, const float2 *ztab,
                         const EwaldTables *ew, const EwaldF32 &ef, cudaStream_t st, const float4 *rtab = nullptr);
cudaError_t launch_build_tables(const EwaldTables *ew, float *stab, float2 *ztab, int n_tab, cudaStream_t st,
                                float4 *rtab = nullptr);

}  // namespace vie
