// farfield.h -- launcher of the Fraunhofer far-field transform (farfield.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace psatd {

// Arguments of one far-field transform: field F [ny][nx] (row stride nx), the
// window [x0, x1) x [y0, y1) in cells, cell sizes, Hann apodisation flags, nk
// wavevectors k[2j] = kx, k[2j+1] = ky, complex results out[2j], out[2j+1].
struct FarfieldArgs {
  const void* F;
  int64_t nx;
  int64_t x0, x1, y0, y1;
  double dx, dy;
  int win_x, win_y;
  const double* k;
  double* out;
  int nk;
};

// Longest window row the kernel's shared-memory phase table takes.
constexpr int64_t kFarfieldMaxRow = 8192;

cudaError_t launch_farfield(bool f32, const FarfieldArgs& a, cudaStream_t st);

}  // namespace psatd
