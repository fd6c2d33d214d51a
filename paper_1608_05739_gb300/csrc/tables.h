// tables.h -- host entry points of the plan-time table kernels (tables.cu).
#pragma once
#include <cuda_runtime.h>

namespace psatd {
cudaError_t launch_twiddles(void* out, int n, bool f32, cudaStream_t st);
cudaError_t launch_coefs(void* out, bool f32, int e0, int e1, int e2, int nx, int ny, int nz,
                         double rx, double ry, double rz, double g0, double c, double dt,
                         double eps0, double invN, cudaStream_t st);
}  // namespace psatd
