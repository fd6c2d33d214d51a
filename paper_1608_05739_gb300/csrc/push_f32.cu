// push_f32.cu -- float instantiation of the fused last-axis FFT + PSATD push pass.
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push<float, false, 8>(int, int, dim3, int, int, size_t, cudaStream_t,
                                              const PushArgs<float>&, const void*);

}  // namespace psatd
