// persist_tcb.cu -- instantiation of the persistent passes with split-BF16 tensor-core stages (persist.cuh).
#include "persist_impl.cuh"

namespace psatd {
template cudaError_t launch_persist_x<float, 2, 0>(bool, int, cudaStream_t, const XClassArgs*, const PersistQueue&, int*);
template cudaError_t launch_persist_push<float, 2, 0>(int, int, int, cudaStream_t, const PushArgs<float>*, const void* const*, const PersistQueue&, int*);
}  // namespace psatd
