// fdtd.cu -- Yee and Cole-Karkkainen (CKC) FDTD steps on a periodic grid
// (Sec. III.A; Table 1 rows "Yee" and "CKC"), the comparators of the PSATD step.
//
// Staggering (index [k][j][i] of each component):
//   Ex (i+1/2, j, k)  Ey (i, j+1/2, k)  Ez (i, j, k+1/2)
//   Bx (i, j+1/2, k+1/2)  By (i+1/2, j, k+1/2)  Bz (i+1/2, j+1/2, k); J with E.
// A step advances co-temporal (E, B): B -= (dt/2) curl E; E += dt (c^2 curl B
// - J/eps0); B -= (dt/2) curl E.  Faraday uses forward differences of E,
// Ampere backward differences of B.  CKC (2D only, beta = 1/4): each Faraday
// difference along one axis is averaged over the transverse neighbour rows
// with weights (beta/2, 1 - beta, beta/2).  One thread per cell, x fastest
// (coalesced); an absent component (NULL) is identically zero.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace psatd {

struct FdtdGrid {
  int nx, ny, nz;
  int ndim;
};

template <typename R>
__device__ __forceinline__ R ld(const R* p, int64_t i) { return p ? p[i] : R(0); }

__device__ __forceinline__ int64_t lin(const FdtdGrid& g, int i, int j, int k) {
  return ((int64_t)k * g.ny + j) * g.nx + i;
}
__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// forward difference along x of p at cell (i, j, k), times inv_d
template <typename R>
__device__ __forceinline__ R dpx(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return p ? (p[lin(g, wrap(i + 1, g.nx), j, k)] - p[lin(g, i, j, k)]) * inv : R(0);
}
template <typename R>
__device__ __forceinline__ R dpy(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return p ? (p[lin(g, i, wrap(j + 1, g.ny), k)] - p[lin(g, i, j, k)]) * inv : R(0);
}
template <typename R>
__device__ __forceinline__ R dpz(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return (p && g.ndim == 3) ? (p[lin(g, i, j, wrap(k + 1, g.nz))] - p[lin(g, i, j, k)]) * inv : R(0);
}
template <typename R>
__device__ __forceinline__ R dmx(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return p ? (p[lin(g, i, j, k)] - p[lin(g, wrap(i - 1, g.nx), j, k)]) * inv : R(0);
}
template <typename R>
__device__ __forceinline__ R dmy(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return p ? (p[lin(g, i, j, k)] - p[lin(g, i, wrap(j - 1, g.ny), k)]) * inv : R(0);
}
template <typename R>
__device__ __forceinline__ R dmz(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  return (p && g.ndim == 3) ? (p[lin(g, i, j, k)] - p[lin(g, i, j, wrap(k - 1, g.nz))]) * inv : R(0);
}

// x-difference averaged over the y-neighbour rows (CKC) or plain (Yee)
template <typename R, bool CKC>
__device__ __forceinline__ R dpx_s(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  const R d0 = dpx(p, g, i, j, k, inv);
  if constexpr (!CKC) return d0;
  const R dm = dpx(p, g, i, wrap(j - 1, g.ny), k, inv), dp = dpx(p, g, i, wrap(j + 1, g.ny), k, inv);
  return R(0.75) * d0 + R(0.125) * (dm + dp);
}
template <typename R, bool CKC>
__device__ __forceinline__ R dpy_s(const R* p, const FdtdGrid& g, int i, int j, int k, R inv) {
  const R d0 = dpy(p, g, i, j, k, inv);
  if constexpr (!CKC) return d0;
  const R dm = dpy(p, g, wrap(i - 1, g.nx), j, k, inv), dp = dpy(p, g, wrap(i + 1, g.nx), j, k, inv);
  return R(0.75) * d0 + R(0.125) * (dm + dp);
}

template <typename R, bool CKC>
__global__ void __launch_bounds__(256) k_fdtd_faraday(FdtdGrid g, R* Bx, R* By, R* Bz, const R* Ex,
                                                      const R* Ey, const R* Ez, R h, R idx, R idy,
                                                      R idz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  const int64_t c = lin(g, i, j, k);
  if (Bx) Bx[c] = Bx[c] - h * (dpy_s<R, CKC>(Ez, g, i, j, k, idy) - dpz(Ey, g, i, j, k, idz));
  if (By) By[c] = By[c] - h * (dpz(Ex, g, i, j, k, idz) - dpx_s<R, CKC>(Ez, g, i, j, k, idx));
  if (Bz) Bz[c] = Bz[c] - h * (dpx_s<R, CKC>(Ey, g, i, j, k, idx) - dpy_s<R, CKC>(Ex, g, i, j, k, idy));
}

template <typename R>
__global__ void __launch_bounds__(256) k_fdtd_ampere(FdtdGrid g, R* Ex, R* Ey, R* Ez, const R* Bx,
                                                     const R* By, const R* Bz, const R* Jx,
                                                     const R* Jy, const R* Jz, R dt, R c2,
                                                     R dt_eps0, R idx, R idy, R idz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nx) return;
  const int64_t c = lin(g, i, j, k);
  if (Ex) {
    R e = Ex[c] + dt * (c2 * (dmy(Bz, g, i, j, k, idy) - dmz(By, g, i, j, k, idz)));
    if (Jx) e = e - dt_eps0 * Jx[c];
    Ex[c] = e;
  }
  if (Ey) {
    R e = Ey[c] + dt * (c2 * (dmz(Bx, g, i, j, k, idz) - dmx(Bz, g, i, j, k, idx)));
    if (Jy) e = e - dt_eps0 * Jy[c];
    Ey[c] = e;
  }
  if (Ez) {
    R e = Ez[c] + dt * (c2 * (dmx(By, g, i, j, k, idx) - dmy(Bx, g, i, j, k, idy)));
    if (Jz) e = e - dt_eps0 * Jz[c];
    Ez[c] = e;
  }
}

template <typename R>
cudaError_t launch_fdtd(int ndim, int scheme, int64_t nx, int64_t ny, int64_t nz, const double* d,
                        double dt, double c, double eps0, void* const E[3], void* const B[3],
                        const void* const J[3], int nsteps, cudaStream_t st) {
  FdtdGrid g{(int)nx, (int)ny, (int)nz, ndim};
  const dim3 block(nx < 256 ? (unsigned)nx : 256u);
  const dim3 grid((unsigned)((nx + block.x - 1) / block.x), (unsigned)ny, (unsigned)nz);
  R* e[3] = {static_cast<R*>(E[0]), static_cast<R*>(E[1]), static_cast<R*>(E[2])};
  R* b[3] = {static_cast<R*>(B[0]), static_cast<R*>(B[1]), static_cast<R*>(B[2])};
  const R* j[3] = {static_cast<const R*>(J[0]), static_cast<const R*>(J[1]),
                   static_cast<const R*>(J[2])};
  const R idx = R(1.0 / d[0]), idy = R(1.0 / d[1]), idz = R(ndim == 3 ? 1.0 / d[2] : 0.0);
  const R h = R(0.5 * dt);
  for (int s = 0; s < nsteps; ++s) {
    for (int half = 0; half < 2; ++half) {
      if (half == 1) {
        k_fdtd_ampere<R><<<grid, block, 0, st>>>(g, e[0], e[1], e[2], b[0], b[1], b[2], j[0], j[1], j[2],
                                                 R(dt), R(c * c), R(dt / eps0), idx, idy, idz);
      }
      if (scheme == 1)
        k_fdtd_faraday<R, true><<<grid, block, 0, st>>>(g, b[0], b[1], b[2], e[0], e[1], e[2], h, idx, idy, idz);
      else
        k_fdtd_faraday<R, false><<<grid, block, 0, st>>>(g, b[0], b[1], b[2], e[0], e[1], e[2], h, idx, idy, idz);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template cudaError_t launch_fdtd<float>(int, int, int64_t, int64_t, int64_t, const double*, double,
                                        double, double, void* const[3], void* const[3],
                                        const void* const[3], int, cudaStream_t);
template cudaError_t launch_fdtd<double>(int, int, int64_t, int64_t, int64_t, const double*, double,
                                         double, double, void* const[3], void* const[3],
                                         const void* const[3], int, cudaStream_t);

}  // namespace psatd
