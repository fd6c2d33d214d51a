// persist_x_f32.cu -- instantiation of the persistent transposing x passes, float, power-of-two and 3 * 2^k lengths (persist.cuh).
#include "persist_impl.cuh"

namespace psatd {
template cudaError_t launch_persist_x<float, 0, 0>(bool, int, cudaStream_t, const XClassArgs*, const PersistQueue&, int*);
template cudaError_t launch_persist_x<float, 0, 1>(bool, int, cudaStream_t, const XClassArgs*, const PersistQueue&, int*);
}  // namespace psatd
