// push5_f32.cu -- float instantiation of the fused last-axis FFT + PSATD push
// pass for the mixed lengths 5 * 2^k (radix-5 first stage, 20 elements per thread).
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push5<float>(int, int, dim3, int, int, size_t, cudaStream_t, const PushArgs<float>&,
                                              const void*);
}  // namespace psatd
