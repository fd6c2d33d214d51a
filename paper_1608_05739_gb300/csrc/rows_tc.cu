// rows_tc.cu -- tensor-core (split-FP16 radix-16) instantiation of the
// transposing line-FFT passes, float data.
#include "launch_impl.cuh"

namespace psatd {
template cudaError_t launch_fwd_T<float, 1>(int, bool, const PassGeom&, cudaStream_t, const LineIO&,
                                                const void*, int64_t, int64_t, int64_t, int64_t,
                                                const int64_t*);
template cudaError_t launch_inv_T<float, 1>(int, bool, const PassGeom&, cudaStream_t, const LineIO&,
                                                const void*, int64_t, int64_t, int64_t, int64_t,
                                                const int64_t*);
}  // namespace psatd
