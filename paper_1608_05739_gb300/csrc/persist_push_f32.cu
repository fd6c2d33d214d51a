// persist_push_f32.cu -- instantiation of the persistent fused pass, float, power-of-two lengths (persist.cuh).
#include "persist_impl.cuh"

namespace psatd {
template cudaError_t launch_persist_push<float, 0, 0>(int, int, int, cudaStream_t, const PushArgs<float>*, const void* const*, const PersistQueue&, int*);
}  // namespace psatd
