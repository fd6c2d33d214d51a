// tables.h -- host entry points of the plan-time table kernels (tables.cu).
#pragma once
#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace psatd {
// L: transform length of the axis (nx/2 for the R2C axis); ept: elements per
// thread of the kernels that read it; table of at most 2L entries
cudaError_t launch_twiddles(void* out, int L, int ept, bool r2c, bool f32, cudaStream_t st);
// elements per thread of the transposing passes (RowEPT in fft_core.cuh) and of the fused pass
inline int row_ept(int L) { return L >= 16 ? 16 : 8; }
inline int push_ept(int, bool tc = false) { return tc ? PushEPT<16, true>::value : PushEPT<16>::value; }
// split-FP16 radix-16 DFT matrices of both directions, tensor-core operand layout
cudaError_t launch_tc_dftmat(void* out, cudaStream_t st);
cudaError_t launch_coefs(void* out, bool f32, int e0, int e1, int e2, int nx, int ny, int nz,
                         double rx, double ry, double rz, double g0, double c, double dt,
                         double eps0, double invN, cudaStream_t st);
}  // namespace psatd
