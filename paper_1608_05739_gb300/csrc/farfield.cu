// farfield.cu -- the Fraunhofer far-field transform of a field snapshot, the
// diagnostic of the angularly resolved harmonic spectrum (Sec. II.B): for every
// requested wavevector k_j = (kx, ky),
//   U_j = sum over the window's cells of w(x, y) F(x, y) exp(-i (kx x + ky y)) dx dy,
// x = i dx, y = j dy, w an optional Hann apodisation (along x, or x and y).
// One CTA per wavevector: the CTA builds the x phase table w_x(i) exp(-i kx x_i)
// in shared memory (FP64 sincos, rounded once to the field's precision), each
// warp takes rows of the window, sums a row with its lanes (fixed xor-butterfly
// order), applies the row's phase and weight in FP64, and the warps' partial
// sums are added in a fixed order: the result does not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "farfield.h"

namespace psatd {

__device__ __forceinline__ double hann_w(int i, int n) {
  const double s = sinpi((i + 0.5) / (double)n);
  return s * s;
}

template <typename R>
__global__ void __launch_bounds__(256) k_farfield(FarfieldArgs a) {
  typedef typename std::conditional<sizeof(R) == 4, float2, double2>::type C2;
  extern __shared__ __align__(16) unsigned char ff_smem[];
  C2* px = reinterpret_cast<C2*>(ff_smem);
  __shared__ double red[2][8];
  const int j = blockIdx.x;
  const double kx = a.k[2 * j], ky = a.k[2 * j + 1];
  const int wx = (int)(a.x1 - a.x0), wy = (int)(a.y1 - a.y0);
  for (int i = threadIdx.x; i < wx; i += blockDim.x) {
    double s, c;
    sincos(kx * (double)(a.x0 + i) * a.dx, &s, &c);
    const double w = a.win_x ? hann_w(i, wx) : 1.0;
    px[i].x = (R)(w * c);
    px[i].y = (R)(-w * s);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const R* F = static_cast<const R*>(a.F);
  double ure = 0.0, uim = 0.0;
  for (int r = warp; r < wy; r += nwarp) {
    const R* row = F + (a.y0 + r) * a.nx + a.x0;
    R sre = R(0), sim = R(0);
    for (int i = lane; i < wx; i += 32) {
      const R f = row[i];
      sre += f * px[i].x;
      sim += f * px[i].y;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      sre += __shfl_xor_sync(0xffffffffu, sre, o);
      sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    if (lane == 0) {
      double s, c;
      sincos(ky * (double)(a.y0 + r) * a.dy, &s, &c);
      const double w = a.win_y ? hann_w(r, wy) : 1.0;
      ure += w * ((double)sre * c + (double)sim * s);
      uim += w * ((double)sim * c - (double)sre * s);
    }
  }
  if (lane == 0) {
    red[0][warp] = ure;
    red[1][warp] = uim;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < nwarp; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    a.out[2 * j] = s0 * a.dx * a.dy;
    a.out[2 * j + 1] = s1 * a.dx * a.dy;
  }
}

cudaError_t launch_farfield(bool f32, const FarfieldArgs& a, cudaStream_t st) {
  const int wx = (int)(a.x1 - a.x0);
  const size_t smem = (size_t)wx * (f32 ? sizeof(float2) : sizeof(double2));
  cudaError_t e;
  if (f32) {
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_farfield<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
    k_farfield<float><<<a.nk, 256, smem, st>>>(a);
  } else {
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_farfield<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
    k_farfield<double><<<a.nk, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace psatd
