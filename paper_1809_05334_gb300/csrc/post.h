// Post-processing launchers (see post.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "fill.h"

namespace vie {

cudaError_t upload_post_constants();
cudaError_t launch_post(const DevMesh &m, const DevReq &q, const double *x, const int32_t *dom, int n_dom,
                        double norm, const double *orders, int n_orders, double a, double b, double kz00,
                        const double *pol_dev, double *acc, double *J, double *rt, double *dens, cudaStream_t st);
cudaError_t launch_unpermute(const double *x, const int32_t *perm, int n, double *out, cudaStream_t st);

}  // namespace vie
