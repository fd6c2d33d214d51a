// persist_impl.cuh -- host launchers of the persistent batch passes; included by
// the persist_* translation units, which instantiate them per precision.
#pragma once
#include "launch.h"

namespace psatd {

// Opt the kernel in to its dynamic shared memory (always: its static shared
// memory, the class arguments, adds to the request), and report its occupancy.
template <typename K>
static cudaError_t persist_launch(K kern, int threads, size_t smem, int* occ) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if (occ) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R, int TC, int FAM>
cudaError_t launch_persist_x(bool fwd, int grid, cudaStream_t st, const XClassArgs* cls, const PersistQueue& q,
                             int* occ) {
  const size_t smem = persist_x_smem<R, TC, FAM>();
  auto kern = fwd ? k_persist_x<R, TC, FAM, true> : k_persist_x<R, TC, FAM, false>;
  cudaError_t e = persist_launch(kern, kPersistXThreads, smem, occ);
  if (e != cudaSuccess || grid <= 0) return e;
  kern<<<grid, kPersistXThreads, smem, st>>>(cls, q);
  return cudaGetLastError();
}

template <typename R, int TC, int FAM>
cudaError_t launch_persist_push(int layout, int n_in, int grid, cudaStream_t st, const PushArgs<R>* cls,
                                const void* const* tws, const PersistQueue& q, int* occ) {
  const size_t smem = persist_push_smem<R, TC, FAM>(n_in);
  void (*kern)(const PushArgs<R>*, const void* const*, PersistQueue) = nullptr;
  switch (layout) {
    case 1: kern = k_persist_push<R, TC, FAM, 1>; break;
    case 2: kern = k_persist_push<R, TC, FAM, 2>; break;
    case 3: kern = k_persist_push<R, TC, FAM, 3>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = persist_launch(kern, kPersistThreads, smem, occ);
  if (e != cudaSuccess || grid <= 0) return e;
  kern<<<grid, kPersistThreads, smem, st>>>(cls, tws, q);
  return cudaGetLastError();
}

}  // namespace psatd
