// persist_tc.cu -- instantiation of the persistent passes with split-FP16 tensor-core stages (persist.cuh).
#include "persist_impl.cuh"

namespace psatd {
template cudaError_t launch_persist_x<float, 1, 0>(bool, int, cudaStream_t, const XClassArgs*, const PersistQueue&, int*);
template cudaError_t launch_persist_push<float, 1, 0>(int, int, int, cudaStream_t, const PushArgs<float>*, const void* const*, const PersistQueue&, int*);
}  // namespace psatd
