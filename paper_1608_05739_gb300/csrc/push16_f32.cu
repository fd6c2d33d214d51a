// push16_f32.cu -- float instantiation of the fused last-axis FFT + PSATD push
// pass with radix-16 stages (16 elements per thread), one of the autotuner's
// radix schedules.
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push<float, false, 16>(int, int, dim3, int, int, size_t, cudaStream_t,
                                                   const PushArgs<float>&, const void*);
}  // namespace psatd
