// persist_push3_f32.cu -- instantiation of the persistent fused pass, float, 3 * 2^k lengths (persist.cuh).
#include "persist_impl.cuh"

namespace psatd {
template cudaError_t launch_persist_push<float, 0, 1>(int, int, int, cudaStream_t, const PushArgs<float>*, const void* const*, const PersistQueue&, int*);
}  // namespace psatd
