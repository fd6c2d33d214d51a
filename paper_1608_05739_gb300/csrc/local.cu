// local.cu -- guard refresh of the local-FFT decomposition (Sec. II.A.3): the
// copies between a periodic global 2D grid and its patches extended by guard
// cells.  Patch (p, q) of ix x iy interior cells extended by g on every side
// holds, at (i, j), the global cell ((p ix - g + i) mod nx, (q iy - g + j) mod ny).
#include <cuda_runtime.h>
#include <stdint.h>

#include "local.h"

namespace psatd {

struct LocalGeom {
  int64_t nx, ny;  // global grid
  int px, py, g;   // patches along x, y; guard width
  int ix, iy;      // interior cells of a patch
  int ex, ey;      // extended patch: ix + 2g, iy + 2g
};

// global -> patches: one thread per extended-patch element of every component
template <typename R>
__global__ void k_guard_gather(LocalComps c, LocalGeom G, int ncomp) {
  const int64_t per_patch = (int64_t)G.ex * G.ey;
  const int64_t per_comp = per_patch * G.px * G.py;
  const int64_t total = per_comp * ncomp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int comp = (int)(e / per_comp);
    const int64_t r = e - comp * per_comp;
    const int patch = (int)(r / per_patch);
    const int64_t l = r - patch * per_patch;
    const int j = (int)(l / G.ex), i = (int)(l - (int64_t)j * G.ex);
    const int p = patch % G.px, q = patch / G.px;
    int64_t x = (int64_t)p * G.ix - G.g + i, y = (int64_t)q * G.iy - G.g + j;
    x = ((x % G.nx) + G.nx) % G.nx;
    y = ((y % G.ny) + G.ny) % G.ny;
    static_cast<R*>(c.patch[comp])[r] = static_cast<const R*>(c.global[comp])[y * G.nx + x];
  }
}

// patches -> global: one thread per interior element of every component
template <typename R>
__global__ void k_guard_scatter(LocalComps c, LocalGeom G, int ncomp) {
  const int64_t per_patch = (int64_t)G.ix * G.iy;
  const int64_t per_comp = per_patch * G.px * G.py;
  const int64_t total = per_comp * ncomp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int comp = (int)(e / per_comp);
    const int64_t r = e - comp * per_comp;
    const int patch = (int)(r / per_patch);
    const int64_t l = r - patch * per_patch;
    const int j = (int)(l / G.ix), i = (int)(l - (int64_t)j * G.ix);
    const int p = patch % G.px, q = patch / G.px;
    const int64_t src = (int64_t)patch * G.ex * G.ey + (int64_t)(j + G.g) * G.ex + (i + G.g);
    const int64_t dst = ((int64_t)q * G.iy + j) * G.nx + (int64_t)p * G.ix + i;
    static_cast<R*>(c.global_out[comp])[dst] = static_cast<const R*>(c.patch[comp])[src];
  }
}

static unsigned blocks_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

cudaError_t launch_guard_gather(bool f32, const LocalComps& c, int ncomp, int64_t nx, int64_t ny, int px, int py,
                                int g, cudaStream_t st) {
  LocalGeom G{nx, ny, px, py, g, (int)(nx / px), (int)(ny / py), (int)(nx / px) + 2 * g, (int)(ny / py) + 2 * g};
  const int64_t total = (int64_t)G.ex * G.ey * px * py * ncomp;
  if (f32) k_guard_gather<float><<<blocks_for(total), 256, 0, st>>>(c, G, ncomp);
  else k_guard_gather<double><<<blocks_for(total), 256, 0, st>>>(c, G, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_guard_scatter(bool f32, const LocalComps& c, int ncomp, int64_t nx, int64_t ny, int px, int py,
                                 int g, cudaStream_t st) {
  LocalGeom G{nx, ny, px, py, g, (int)(nx / px), (int)(ny / py), (int)(nx / px) + 2 * g, (int)(ny / py) + 2 * g};
  const int64_t total = (int64_t)G.ix * G.iy * px * py * ncomp;
  if (f32) k_guard_scatter<float><<<blocks_for(total), 256, 0, st>>>(c, G, ncomp);
  else k_guard_scatter<double><<<blocks_for(total), 256, 0, st>>>(c, G, ncomp);
  return cudaGetLastError();
}

}  // namespace psatd
