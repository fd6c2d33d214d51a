// push16_f64.cu -- double instantiation of the fused last-axis FFT + PSATD push
// pass with radix-16 stages (16 elements per thread), one of the autotuner's
// radix schedules.
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push<double, false, 16>(int, int, dim3, int, int, size_t, cudaStream_t,
                                                   const PushArgs<double>&, const void*);
}  // namespace psatd
