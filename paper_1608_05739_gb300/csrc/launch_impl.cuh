// launch_impl.cuh -- templated launchers with the switch over the transform
// length; included by the per-precision translation units.
#pragma once
#include "launch.h"

namespace psatd {

// Dynamic shared-memory opt-in (static shared memory adds to the request).  The
// carveout is left to the driver: a maximal shared carveout shrinks the L1 that
// holds the twiddle tables and was measured slower.
template <typename K>
static cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 32 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <typename R, int TC, int L>
static cudaError_t fwd_T_L(bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io,
                           const void* tw, int64_t a, int64_t b, int64_t c, int64_t d, const int64_t* off) {
  typedef typename Types<R>::W W;
  const dim3 block(FFTPlan<L, RowEPT<L>::value>::kT, 1u << g.log_tb);
  cudaError_t e;
  if (r2c) {
    if constexpr (L <= 2048) {
      auto kern = k_fwd_T<R, L, true, TC>;
      if ((e = set_smem(kern, g.smem)) != cudaSuccess) return e;
      kern<<<g.grid, block, g.smem, st>>>(io, static_cast<const W*>(tw), a, b, c, d, g.log_tb, off);
    } else {
      return cudaErrorInvalidValue;
    }
  } else {
    auto kern = k_fwd_T<R, L, false, TC>;
    if ((e = set_smem(kern, g.smem)) != cudaSuccess) return e;
    kern<<<g.grid, block, g.smem, st>>>(io, static_cast<const W*>(tw), a, b, c, d, g.log_tb, off);
  }
  return cudaGetLastError();
}

template <typename R, int TC, int L>
static cudaError_t inv_T_L(bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io,
                           const void* tw, int64_t a, int64_t b, int64_t c, int64_t d, const int64_t* off) {
  typedef typename Types<R>::W W;
  const dim3 block(FFTPlan<L, RowEPT<L>::value>::kT, 1u << g.log_tb);
  cudaError_t e;
  if (c2r) {
    if constexpr (L <= 2048) {
      auto kern = k_inv_T<R, L, true, TC>;
      if ((e = set_smem(kern, g.smem)) != cudaSuccess) return e;
      kern<<<g.grid, block, g.smem, st>>>(io, static_cast<const W*>(tw), a, b, c, d, g.log_tb, off);
    } else {
      return cudaErrorInvalidValue;
    }
  } else {
    auto kern = k_inv_T<R, L, false, TC>;
    if ((e = set_smem(kern, g.smem)) != cudaSuccess) return e;
    kern<<<g.grid, block, g.smem, st>>>(io, static_cast<const W*>(tw), a, b, c, d, g.log_tb, off);
  }
  return cudaGetLastError();
}

template <typename R, int TC, int EPT, int L>
static cudaError_t push_L(int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                          const PushArgs<R>& a, const void* tw) {
  typedef typename Types<R>::W W;
  if constexpr (L < EPT) {
    return cudaErrorInvalidValue;
  } else {
    const dim3 block(FFTPlan<L, EPT>::kT, tb, groups);
    // component groups: their own instantiation, for whole-warp lines in FP32 and
    // for the tensor-core pairs (the host admits groups > 1 nowhere else)
    constexpr bool kGrpOk = TC ? EPT == 16 : (sizeof(R) == 4 && FFTPlan<L, EPT>::kT % 32 == 0);
    if (groups > 1 && !kGrpOk) return cudaErrorInvalidValue;
    cudaError_t e;
#define PSATD_PUSH_LAUNCH(LAY, GRP)                                            \
  {                                                                            \
    auto kern = k_line_push<R, L, LAY, TC, EPT, GRP>;                          \
    if ((e = set_smem(kern, smem)) != cudaSuccess) return e;                   \
    kern<<<grid, block, smem, st>>>(a, static_cast<const W*>(tw));             \
  }
#define PSATD_PUSH_CASE(LAY)                                                   \
  case LAY: {                                                                  \
    if constexpr (kGrpOk) {                                                    \
      if (groups > 1) PSATD_PUSH_LAUNCH(LAY, true)                             \
      else PSATD_PUSH_LAUNCH(LAY, false)                                       \
    } else {                                                                   \
      PSATD_PUSH_LAUNCH(LAY, false)                                            \
    }                                                                          \
    break;                                                                     \
  }
    switch (layout) {
      PSATD_PUSH_CASE(0)
      PSATD_PUSH_CASE(1)
      PSATD_PUSH_CASE(2)
      PSATD_PUSH_CASE(3)
      default:
        return cudaErrorInvalidValue;
    }
#undef PSATD_PUSH_CASE
#undef PSATD_PUSH_LAUNCH
    return cudaGetLastError();
  }
}

// The tensor-core variants exist from L = 16 on (their first radix-16 stage).
#define PSATD_L_SWITCH(FN, ...)                                   \
  switch (L) {                                                    \
    case 8: if constexpr (!TC) return FN<R, TC, 8>(__VA_ARGS__);  \
            else return cudaErrorInvalidValue;                    \
    case 16: return FN<R, TC, 16>(__VA_ARGS__);                   \
    case 32: return FN<R, TC, 32>(__VA_ARGS__);                   \
    case 64: return FN<R, TC, 64>(__VA_ARGS__);                   \
    case 128: return FN<R, TC, 128>(__VA_ARGS__);                 \
    case 256: return FN<R, TC, 256>(__VA_ARGS__);                 \
    case 512: return FN<R, TC, 512>(__VA_ARGS__);                 \
    case 1024: return FN<R, TC, 1024>(__VA_ARGS__);               \
    case 2048: return FN<R, TC, 2048>(__VA_ARGS__);               \
    case 4096: return FN<R, TC, 4096>(__VA_ARGS__);               \
    default: return cudaErrorInvalidValue;                        \
  }

// Mixed lengths 3 * 2^k (FP32, no tensor-core stages).
#define PSATD_L3_SWITCH(FN, ...)                         \
  switch (L) {                                           \
    case 48: return FN<R, 0, 48>(__VA_ARGS__);           \
    case 96: return FN<R, 0, 96>(__VA_ARGS__);           \
    case 192: return FN<R, 0, 192>(__VA_ARGS__);         \
    case 384: return FN<R, 0, 384>(__VA_ARGS__);         \
    case 768: return FN<R, 0, 768>(__VA_ARGS__);         \
    case 1536: return FN<R, 0, 1536>(__VA_ARGS__);       \
    case 3072: return FN<R, 0, 3072>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;               \
  }

// Mixed lengths 5 * 2^k (FP32, no tensor-core stages).
#define PSATD_L5_SWITCH(FN, ...)                         \
  switch (L) {                                           \
    case 80: return FN<R, 0, 80>(__VA_ARGS__);           \
    case 160: return FN<R, 0, 160>(__VA_ARGS__);         \
    case 320: return FN<R, 0, 320>(__VA_ARGS__);         \
    case 640: return FN<R, 0, 640>(__VA_ARGS__);         \
    case 1280: return FN<R, 0, 1280>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;               \
  }

template <typename R>
cudaError_t launch_fwd_T5(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk, const int64_t* a0_off) {
  PSATD_L5_SWITCH(fwd_T_L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off)
}
template <typename R>
cudaError_t launch_inv_T5(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb, const int64_t* a0_off) {
  PSATD_L5_SWITCH(inv_T_L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off)
}
template <typename R>
cudaError_t launch_line_push5(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                              const PushArgs<R>& a, const void* tw) {
  switch (L) {
    case 80: return push_L<R, 0, 20, 80>(layout, grid, tb, groups, smem, st, a, tw);
    case 160: return push_L<R, 0, 20, 160>(layout, grid, tb, groups, smem, st, a, tw);
    case 320: return push_L<R, 0, 20, 320>(layout, grid, tb, groups, smem, st, a, tw);
    case 640: return push_L<R, 0, 20, 640>(layout, grid, tb, groups, smem, st, a, tw);
    case 1280: return push_L<R, 0, 20, 1280>(layout, grid, tb, groups, smem, st, a, tw);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_fwd_T3(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk, const int64_t* a0_off) {
  PSATD_L3_SWITCH(fwd_T_L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off)
}
template <typename R>
cudaError_t launch_inv_T3(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                          int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb, const int64_t* a0_off) {
  PSATD_L3_SWITCH(inv_T_L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off)
}
template <typename R>
cudaError_t launch_line_push3(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                              const PushArgs<R>& a, const void* tw) {
  switch (L) {
    case 48: return push_L<R, 0, 12, 48>(layout, grid, tb, groups, smem, st, a, tw);
    case 96: return push_L<R, 0, 12, 96>(layout, grid, tb, groups, smem, st, a, tw);
    case 192: return push_L<R, 0, 12, 192>(layout, grid, tb, groups, smem, st, a, tw);
    case 384: return push_L<R, 0, 12, 384>(layout, grid, tb, groups, smem, st, a, tw);
    case 768: return push_L<R, 0, 12, 768>(layout, grid, tb, groups, smem, st, a, tw);
    case 1536: return push_L<R, 0, 12, 1536>(layout, grid, tb, groups, smem, st, a, tw);
    case 3072: return push_L<R, 0, 12, 3072>(layout, grid, tb, groups, smem, st, a, tw);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int TC>
cudaError_t launch_fwd_T(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io,
                         const void* tw, int64_t in_sa0, int64_t in_sb, int64_t out_sa0,
                         int64_t out_sk, const int64_t* a0_off) {
  PSATD_L_SWITCH(fwd_T_L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off)
}

template <typename R, int TC>
cudaError_t launch_inv_T(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io,
                         const void* tw, int64_t in_sa0, int64_t in_sk, int64_t out_sa0,
                         int64_t out_sb, const int64_t* a0_off) {
  PSATD_L_SWITCH(inv_T_L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off)
}

template <typename R, int TC, int EPT>
static cudaError_t push_L_e(int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                            const PushArgs<R>& a, const void* tw, int L) {
#define PUSH_E(LL) push_L<R, TC, EPT, LL>
  switch (L) {
    case 8: if constexpr (!TC) return PUSH_E(8)(layout, grid, tb, groups, smem, st, a, tw);
            else return cudaErrorInvalidValue;
    case 16: return PUSH_E(16)(layout, grid, tb, groups, smem, st, a, tw);
    case 32: return PUSH_E(32)(layout, grid, tb, groups, smem, st, a, tw);
    case 64: return PUSH_E(64)(layout, grid, tb, groups, smem, st, a, tw);
    case 128: return PUSH_E(128)(layout, grid, tb, groups, smem, st, a, tw);
    case 256: return PUSH_E(256)(layout, grid, tb, groups, smem, st, a, tw);
    case 512: return PUSH_E(512)(layout, grid, tb, groups, smem, st, a, tw);
    case 1024: return PUSH_E(1024)(layout, grid, tb, groups, smem, st, a, tw);
    case 2048: return PUSH_E(2048)(layout, grid, tb, groups, smem, st, a, tw);
    case 4096: return PUSH_E(4096)(layout, grid, tb, groups, smem, st, a, tw);
    default: return cudaErrorInvalidValue;
  }
#undef PUSH_E
}

template <typename R, int TC, int EPT>
cudaError_t launch_line_push(int L, int layout, dim3 grid, int tb, int groups, size_t smem, cudaStream_t st,
                             const PushArgs<R>& a, const void* tw) {
  return push_L_e<R, TC, EPT>(layout, grid, tb, groups, smem, st, a, tw, L);
}

}  // namespace psatd
