// push_tcb.cu -- tensor-core (split-BF16 radix-16) instantiation of the fused
// last-axis FFT + PSATD push pass, float data.
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_line_push<float, 2, 16>(int, int, dim3, int, int, size_t, cudaStream_t,
                                                    const PushArgs<float>&, const void*);
}  // namespace psatd
