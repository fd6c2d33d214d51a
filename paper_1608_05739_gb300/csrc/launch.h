// launch.h -- host-side launchers of the PSATD pass kernels, instantiated per
// precision and variant in the rows_* / push_* translation units.  L is the
// transform length along the pass axis (a power of two 8..4096, or 3 * 2^k for
// the *3 launchers); every launcher returns the launch's cudaError_t.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "persist.cuh"
#include "psatd_kernels.cuh"

namespace psatd {

struct PassGeom {
  dim3 grid;
  int log_tb;      // lines per CTA = 1 << log_tb
  size_t smem;     // dynamic shared memory bytes
};

// a0_off: optional device table of per-patch element offsets into the caller's
// arrays (input of launch_fwd_T, output of launch_inv_T); NULL: a0 * stride.
// TC = true: the tensor-core (split-FP16) variants, float data only.
template <typename R, int TC = 0>
cudaError_t launch_fwd_T(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io,
                         const void* tw, int64_t in_sa0, int64_t in_sb, int64_t out_sa0,
                         int64_t out_sk, const int64_t* a0_off = nullptr);
template <typename R, int TC = 0>
cudaError_t launch_inv_T(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io,
                         const void* tw, int64_t in_sa0, int64_t in_sk, int64_t out_sa0,
                         int64_t out_sb, const int64_t* a0_off = nullptr);
// EPT: 8 or 16 elements per thread (radix-8 / radix-16 stages); TC needs 16.
template <typename R, int TC, int EPT>
cudaError_t launch_line_push(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                             const PushArgs<R>& a, const void* tw);

// the same passes for the mixed lengths L = 3 * 2^k (48..3072; R2C / C2R up to 1536), float only
template <typename R>
cudaError_t launch_fwd_T3(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk,
                          const int64_t* a0_off = nullptr);
template <typename R>
cudaError_t launch_inv_T3(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb,
                          const int64_t* a0_off = nullptr);
template <typename R>
cudaError_t launch_line_push3(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                              const PushArgs<R>& a, const void* tw);

// the same passes for the mixed lengths L = 5 * 2^k (80..1280), float only
template <typename R>
cudaError_t launch_fwd_T5(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk,
                          const int64_t* a0_off = nullptr);
template <typename R>
cudaError_t launch_inv_T5(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb,
                          const int64_t* a0_off = nullptr);
template <typename R>
cudaError_t launch_line_push5(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                              const PushArgs<R>& a, const void* tw);

// Persistent batch passes (persist.cuh): FAM 0 power-of-two lengths, 1 the 3 * 2^k
// lengths (float, TC = 0).  `grid` CTAs of kPersistThreads threads; *occ (if not
// NULL) receives the CTAs per SM the kernel can keep resident.
template <typename R, int TC, int FAM>
cudaError_t launch_persist_x(bool fwd, int grid, cudaStream_t st, const XClassArgs* cls, const PersistQueue& q,
                             int* occ = nullptr);
template <typename R, int TC, int FAM>
cudaError_t launch_persist_push(int layout, int n_in, int grid, cudaStream_t st, const PushArgs<R>* cls,
                                const void* const* tws, const PersistQueue& q, int* occ = nullptr);

template <typename R>
cudaError_t launch_fdtd(int ndim, int scheme, int64_t nx, int64_t ny, int64_t nz, const double* d,
                        double dt, double c, double eps0, void* const E[3], void* const B[3],
                        const void* const J[3], int nsteps, cudaStream_t st);

}  // namespace psatd
