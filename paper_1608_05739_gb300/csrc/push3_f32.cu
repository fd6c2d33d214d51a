// push3_f32.cu -- float instantiation of the fused last-axis FFT + PSATD push
// pass for the mixed lengths 3 * 2^k (radix-3 first stage, 24 elements per thread).
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push3<float>(int, int, dim3, int, int, size_t, cudaStream_t, const PushArgs<float>&,
                                              const void*);
}  // namespace psatd
