// tables.h -- host entry points of the plan-time table kernels (tables.cu).
#pragma once
#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace psatd {
// L: transform length of the axis (nx/2 for the R2C axis); ept: elements per
// thread of the kernels that read it; table of at most 2L entries
cudaError_t launch_twiddles(void* out, int L, int ept, bool r2c, bool f32, cudaStream_t st);
// elements per thread of the transposing passes (RowEPT in fft_core.cuh) and of the fused pass
inline int row_ept(int L) { return odd_factor(L) == 3 ? 24 : odd_factor(L) == 5 ? 20 : L >= 16 ? 16 : 8; }
inline int push_ept(int L, bool tc = false) {
  return odd_factor(L) == 3 ? 12 : odd_factor(L) == 5 ? 20 : tc ? 16 : 8;
}
// split-FP16 (or split-BF16) radix-16 DFT matrices of both directions, tensor-core operand layout
cudaError_t launch_tc_dftmat(void* out, bool bf16, cudaStream_t st);
// kp: per-axis order-p wavenumber tables (units of g0, n_i/2+1 entries) of a
// staggered plan, or NULL for the collocated exact-k plan
cudaError_t launch_coefs(void* out, bool f32, int e0, int e1, int e2, int nx, int ny, int nz,
                         double rx, double ry, double rz, double g0, double c, double dt,
                         double eps0, double invN, cudaStream_t st, const double* const kp[3] = nullptr);
// order-p wavenumbers (double, units of g0) and half-cell phases (twiddle type) of one axis
cudaError_t launch_kp_tables(double* kp, void* ph, const double* C, int nl, int n, double d, double g0, bool f32,
                             cudaStream_t st);
// staggered Fornberg weights C_1..C_(p/2) of even order p (host, FP64)
void staggered_weights(int p, double* C);
// NaN / Inf scan of the n_out output arrays (PSATD_FLAG_CHECKED): `count`
// elements per patch, patches at off[0 .. npatch) (off NULL: one array each);
// sets the non-finite bit in *err.
cudaError_t launch_nonfinite(bool f32, void* const* out, int n_out, const int64_t* off, int npatch,
                             int64_t count, int* err, cudaStream_t st);

}  // namespace psatd
