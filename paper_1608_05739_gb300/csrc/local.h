// local.h -- host entry points of the guard-refresh copies (local.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace psatd {

constexpr int kLocalMaxComp = 11;

// Per-component arrays: the global grid (read by the gather, written by the
// scatter) and the packed extended patches (patch q at q * ex * ey).
struct LocalComps {
  const void* global[kLocalMaxComp];
  void* global_out[kLocalMaxComp];
  void* patch[kLocalMaxComp];
};

// global -> extended patches (guards included), components 0..ncomp-1
cudaError_t launch_guard_gather(bool f32, const LocalComps& c, int ncomp, int64_t nx, int64_t ny, int px, int py,
                                int g, cudaStream_t st);
// extended patches' interiors -> global, components 0..ncomp-1
cudaError_t launch_guard_scatter(bool f32, const LocalComps& c, int ncomp, int64_t nx, int64_t ny, int px, int py,
                                 int g, cudaStream_t st);

}  // namespace psatd
