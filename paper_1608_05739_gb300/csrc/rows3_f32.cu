// rows3_f32.cu -- float instantiation of the transposing line-FFT passes for the
// mixed lengths 3 * 2^k (radix-3 first stage, 24 elements per thread).
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_fwd_T3<float>(int, bool, const PassGeom&, cudaStream_t, const LineIO&, const void*,
                                          int64_t, int64_t, int64_t, int64_t, const int64_t*);
template cudaError_t launch_inv_T3<float>(int, bool, const PassGeom&, cudaStream_t, const LineIO&, const void*,
                                          int64_t, int64_t, int64_t, int64_t, const int64_t*);
}  // namespace psatd
