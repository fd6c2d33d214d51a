// rows5_f32.cu -- float instantiation of the transposing line-FFT passes for the
// mixed lengths 5 * 2^k (radix-5 first stage, 20 elements per thread).
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_fwd_T5<float>(int, bool, const PassGeom&, cudaStream_t, const LineIO&, const void*,
                                          int64_t, int64_t, int64_t, int64_t, const int64_t*);
template cudaError_t launch_inv_T5<float>(int, bool, const PassGeom&, cudaStream_t, const LineIO&, const void*,
                                          int64_t, int64_t, int64_t, int64_t, const int64_t*);
}  // namespace psatd
