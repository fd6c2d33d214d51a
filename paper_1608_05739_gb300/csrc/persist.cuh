// persist.cuh -- persistent batch passes: one launch per pass type runs the work
// of every size class of a batch of 2D patches (the paper's local-FFT subdomains,
// Sec. II.A.3).  Each CTA takes work items from a
// device queue (an atomic counter, kPersistChunk items per take) until it is
// empty; an item is one CTA's worth of the standalone pass (a block of rows of
// one component of one patch, or a block of lines of the fused pass), whose
// arguments come from a per-class table.  The three passes of a step run in
// stream order, which is their only dependency, so no CTA ever waits on
// another.  The last CTA to finish zeroes the queue for the next launch.
#pragma once

#include "psatd_kernels.cuh"

namespace psatd {

constexpr int kPersistThreads = 128;   // fused pass: one 128-row MMA group per CTA in the tensor-core variant
constexpr int kPersistXThreads = 256;  // transposing passes: 8 to 128 rows per item, two MMA groups
constexpr int kPersistChunk = 4;

// One work item: size class, patch within the class and component (transposing
// passes), block of rows / lines.
struct BatchItem {
  int cls;
  int a0;
  int a1;
  int blk;
};

// Per-class arguments of a transposing pass (forward: in_sa0, in_sb, out_sa0,
// out_sk; inverse: in_sa0, in_sk, out_sa0, out_sb) and its geometry.
struct XClassArgs {
  LineIO io;
  const void* tw;
  int64_t s0, s1, s2, s3;
  const int64_t* off;
  int64_t nb;  // rows per patch
  int L;       // line length
  int pad;
};

struct PersistQueue {
  const BatchItem* items;
  int n_items;
  unsigned* counter;  // [0] next item, [1] finished CTAs; both zero between launches
};

// Take the next chunk of items (thread 0), shared with the CTA; returns its
// first index (>= n_items: queue empty).
__device__ __forceinline__ int persist_take(const PersistQueue& q, int* slot) {
  __syncthreads();  // every thread is done with the previous item's shared memory
  if (threadIdx.x == 0) *slot = (int)atomicAdd(q.counter, (unsigned)kPersistChunk);
  __syncthreads();
  return *slot;
}
// After the CTA's last take: the last CTA to finish resets the queue.
__device__ __forceinline__ void persist_finish(const PersistQueue& q) {
  if (threadIdx.x == 0 && atomicAdd(q.counter + 1, 1u) == gridDim.x - 1) {
    q.counter[0] = 0u;
    q.counter[1] = 0u;
  }
}

template <class T>
__device__ __forceinline__ void copy_to_shared(T* dst, const T* src) {
  static_assert(sizeof(T) % 8 == 0, "8-byte words");
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 8); i += blockDim.x)
    reinterpret_cast<uint64_t*>(dst)[i] = reinterpret_cast<const uint64_t*>(src)[i];
}

// Lengths of the persistent passes: FAM 0 powers of two, FAM 1 the 3 * 2^k
// lengths (FP32).  Transposing passes: x lines of L = nx/2 points; fused pass:
// last-axis lines.  Lines of T = L/EPT threads, kPersistThreads / T of them per item.
#define PSATD_PERSIST_X_LENGTHS(FAM, CASE) \
  if constexpr (FAM == 0) { CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) } \
  else { CASE(48) CASE(96) CASE(192) CASE(384) }
#define PSATD_PERSIST_Y_LENGTHS(FAM, CASE) \
  if constexpr (FAM == 0) { CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) } \
  else { CASE(48) CASE(96) CASE(192) CASE(384) CASE(768) }

template <int L>
struct PersistRows {
  static constexpr int T = L / RowEPT<L>::value;
  static constexpr int TB = kPersistXThreads / T;
  static constexpr int LOG_TB = ilog2(TB);
};

// Transposing x pass (forward R2C or inverse C2R) over every class of the queue.
// Register caps of the persistent passes (CTAs that must stay resident together),
// as their standalone kernels: the SIMT transposing passes 64 registers (128 for
// the 3 * 2^k lengths, 24 elements per thread), the tensor-core ones 128 (at 64
// their 16-element rows and split pieces went to the stack); the SIMT fused pass
// 128, the tensor-core one up to 255 (two CTAs per SM, as its shared memory allows
// anyway; with every line length in one kernel it spilled at 128).
template <typename R, int TC, int FAM, bool FWD>
__global__ void __launch_bounds__(kPersistXThreads, (FAM || TC) ? 2 : 4) k_persist_x(const XClassArgs* __restrict__ cls, PersistQueue q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int slot;
  __shared__ __align__(16) XClassArgs A;
  TcCtx tc;
  if constexpr (TC) tc_setup(tc, smem_raw, cls[0].io.gmat, 0u, cls[0].io.err, TC == 2, 0u, cls[0].io.tc_ctl);
  for (;;) {
    const int i0 = persist_take(q, &slot);
    if (i0 >= q.n_items) break;
    const int i1 = i0 + kPersistChunk < q.n_items ? i0 + kPersistChunk : q.n_items;
    for (int i = i0; i < i1; ++i) {
      const BatchItem it = q.items[i];
      __syncthreads();
      copy_to_shared(&A, &cls[it.cls]);
      __syncthreads();
      typedef typename Types<R>::W W;
      bool matched = false;
#define PSATD_X_CASE(LL)                                                                                        \
  if (A.L == LL) {                                                                                              \
    matched = true;                                                                                             \
    typedef PersistRows<LL> G;                                                                                  \
    const RowCta cta{it.blk, it.a0, it.a1, (int)threadIdx.x % G::T, (int)threadIdx.x / G::T, G::LOG_TB, A.nb}; \
    if constexpr (FWD)                                                                                          \
      fwd_T_body<R, LL, true, TC, true>(A.io, static_cast<const W*>(A.tw), A.s0, A.s1, A.s2, A.s3, A.off, cta, \
                                        smem_raw, tc);                                                          \
    else                                                                                                        \
      inv_T_body<R, LL, true, TC, true>(A.io, static_cast<const W*>(A.tw), A.s0, A.s1, A.s2, A.s3, A.off, cta, \
                                        smem_raw, tc);                                                          \
  }
      PSATD_PERSIST_X_LENGTHS(FAM, PSATD_X_CASE)
#undef PSATD_X_CASE
      // a length without a case (the host admits none) is reported, not skipped silently
      if (!matched && threadIdx.x == 0 && A.io.chk_err) atomicOr(A.io.chk_err, kErrBounds);
    }
  }
  persist_finish(q);
  if constexpr (TC) tc_teardown(tc);
}

// Fused last-axis pass over every class of the queue (PushArgs per class; the
// line length is 2 (tab_row - 1)).
template <typename R, int TC, int FAM, int LAYOUT>
__global__ void __launch_bounds__(kPersistThreads, TC ? 2 : 4) k_persist_push(const PushArgs<R>* __restrict__ cls,
                                                                  const void* const* __restrict__ tws,
                                                                  PersistQueue q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int slot;
  __shared__ __align__(8) uint64_t stage_mbar;
  StageCtx sc;
  stage_init(sc, &stage_mbar, cls[0].err ? cls[0].err : cls[0].chk_err);
  TcCtx tc;
  if constexpr (TC) tc_setup(tc, smem_raw, cls[0].gmat, 0u, cls[0].err, TC == 2, 0u, cls[0].tc_ctl);
  // (the queue's first take has a block barrier before any use of the stage mbarrier)
  constexpr int EPT = FAM ? 12 : (TC ? 16 : 8);
  for (;;) {
    const int i0 = persist_take(q, &slot);
    if (i0 >= q.n_items) break;
    const int i1 = i0 + kPersistChunk < q.n_items ? i0 + kPersistChunk : q.n_items;
    for (int i = i0; i < i1; ++i) {
      const BatchItem it = q.items[i];
      const PushArgs<R>& A = cls[it.cls];
      const int Lc = 2 * (A.tab_row - 1);
      typedef typename Types<R>::W W;
      bool matched = false;
#define PSATD_Y_CASE(LL)                                                                                   \
  if (Lc == LL) {                                                                                          \
    matched = true;                                                                                        \
    constexpr int T = LL / EPT;                                                                            \
    line_push_body<R, LL, LAYOUT, TC, EPT>(A, static_cast<const W*>(tws[it.cls]), it.blk,                 \
                                           (int)threadIdx.x % T, (int)threadIdx.x / T, kPersistThreads / T, \
                                           0, 1, smem_raw, tc, sc);                                        \
  }
      PSATD_PERSIST_Y_LENGTHS(FAM, PSATD_Y_CASE)
#undef PSATD_Y_CASE
      if (!matched && threadIdx.x == 0 && A.chk_err) atomicOr(A.chk_err, kErrBounds);
    }
  }
  persist_finish(q);
  if constexpr (TC) tc_teardown(tc);
}

// Dynamic shared memory of the persistent passes (bytes, after the tensor-core
// tail for TC): the largest item of the family.
template <typename R, int TC, int FAM>
constexpr size_t persist_x_smem() {
  // TB lines of L values, plus split-BF16's third A piece (one per 128 threads)
  return (TC ? kTcTail : 0) + (size_t)kPersistXThreads * (FAM ? 24 : 16) * sizeof(typename Types<R>::C) +
         (TC == 2 ? (kPersistXThreads / 128) * TcGeom<16>::kAPiece : 0);
}
template <typename R, int TC, int FAM>
constexpr size_t persist_push_smem(int n_in) {
  return (TC ? kTcTail : 0) +
         (size_t)(n_in + 1) * kPersistThreads * (FAM ? 12 : (TC ? 16 : 8)) * sizeof(typename Types<R>::C);
}

}  // namespace psatd
