// tc_dft.cuh -- radix-R DFT stages (R = 8, 16) on the 5th-generation tensor
// cores: tcgen05.mma with split-FP16 operands and FP32 accumulators in TMEM.
//
// A radix-R stage applies the R x R DFT matrix F to every butterfly's R inputs.
// Written over the reals (element q = (re, im) -> K indices 2q, 2q+1), that is
// the contraction D[m][n] = sum_k A[m][k] G[n][k], m = one butterfly per
// thread (128 rows per MMA, M = 128), K = N = 2R, with G the real form of F:
//   G[2r][2q] = Re F_rq, G[2r][2q+1] = -Im F_rq, G[2r+1][2q] = Im F_rq,
//   G[2r+1][2q+1] = Re F_rq.
// Split operands with an exact head.  Each row is scaled by a power of two s
// that puts its largest component in [2^14, 2^15); the head A_h rounds the
// scaled row to multiples of 16 (11 bits, exact in FP16) and A_l = FP16 of the
// remainder (|A_l| <= 8).  G = G_h + G_l + G_ll with G_h on the 2^-8 grid
// (9 bits) and G_l, G_ll the FP16 roundings of the remainders.  The head
// products A_h G_h are multiples of 2^-4 below 2^15 in magnitude, so their
// 32-term sums (below 2^20) are exact in the FP32 accumulator whatever its
// rounding: the tensor core's truncating accumulation, which shrinks every
// output by a fraction of an ulp and makes a long run decay, never acts on
// them.  The corrections A_h G_l + A_l G_h + A_h G_ll + A_l G_l (2^-9 of the
// head) go to a second accumulator; the two are added in FP32 (round to
// nearest) and the row is scaled back by 1/s.  What is dropped (A_l G_ll and
// the remainders of the splits) is below 2^-24 of the row maximum.
//
// Split-BF16 (bf16 = 1; BF16 keeps 8 bits): the head A_h rounds the scaled row
// to multiples of 128 (8 bits), A_m and A_l are the BF16 roundings of the two
// remainders (a third A piece, in its own region a_tile3); G_h is on the 2^-7
// grid, G_m and G_l the BF16 remainders.  The head products are integers below
// 2^15 (32-term sums exact in FP32); the corrections A_h G_m, A_m G_h, A_h G_l,
// A_l G_h, A_m G_m go to the second accumulator; what is dropped is below 2^-24
// of the row maximum.
//
// Shared-memory operand layout (K-major, no swizzle): 8-row x 16-byte core
// matrices, the K-adjacent ones 128 B apart (LBO), the 8-row groups
// R/4 * 128 B apart (SBO).  One 16-bit K step of an MMA covers two core
// matrices along K, so the second K step of R = 16 starts 256 B further on.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace psatd {

// Status bits written to the plan's device error word.
constexpr int kErrMmaWait = 1;  // an MMA-completion wait ran out of iterations

// Bits of the passes' tensor-core control word (LineIO::tc_ctl, PushArgs::tc_ctl).
// kTcStallMma is a test hook for the failure path: the issuing thread commits
// no MMA, so every completion wait runs out (after kTestWaitIters polls).
constexpr int kTcStallMma = 1;

struct TcCtx {
  uint32_t mbar;     // shared address of the MMA-completion mbarrier
  uint32_t tmem;     // TMEM address of the CTA's accumulators (lane 0, first column)
  uint32_t a_tile;   // shared address of this CTA's A tiles (group g at + g * tile bytes)
  uint32_t a_tile3;  // split-BF16: third A piece (group g at + g * piece bytes)
  uint32_t bmat;     // shared address of the split DFT matrices, forward then adjoint
  uint32_t phase;    // parity of the next mbarrier phase (identical in every thread)
  volatile int* abort;  // CTA-shared word: nonzero once any thread's completion wait ran out
  int* err;          // device error word (may be null)
  int bf16;          // 0 split-FP16, 1 split-BF16
  int wait_iters;    // poll limit of each completion wait
  int stall;         // kTcStallMma: issue nothing (test hook)
};

// Bytes of one split piece (hi or lo) of the A tile of 128 rows / of G.
template <int RS> struct TcGeom {
  static constexpr int kSBO = RS * 32;              // 8-row group stride
  static constexpr int kAPiece = 128 * RS * 4;      // 128 rows x 2R halves
  static constexpr int kATile = 2 * kAPiece;        // A_h, A_l
  static constexpr int kGPiece = 8 * RS * RS;       // 2R rows x 2R halves
  static constexpr int kGDir = 3 * kGPiece;         // G_h, G_l, G_ll of one direction
  static constexpr int kKSteps = RS / 8;            // MMAs (K = 16) per product
  static constexpr int kCols = 2 * RS;              // columns of one accumulator (N)
  // instruction descriptor: F32 accumulate, F16 A and B, both K-major,
  // N = 2R (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4); BF16 A and B
  // set the format fields (bits 7-9, 10-12) to 1
  static constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(2 * RS / 8) << 17) | (8u << 24);
  static constexpr uint32_t kIdescBF16 = kIdesc | (1u << 7) | (1u << 10);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1 in
// bits 46-47, base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase with parity `phase` to complete, at most `iters` polls
// (each may suspend the thread briefly).  Returns false when the limit is
// reached; the caller then records the failure (tc_dft) so that the CTA stops
// using the tensor cores, finishes and frees its TMEM.
constexpr int kWaitIters = 1 << 21;
constexpr int kTestWaitIters = 256;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, int iters) {
  uint32_t done = 0;
  for (int i = 0; i < iters; ++i) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// TMEM allocation of `ncols` columns (a power of two >= 32) by one whole warp;
// the address lands in the shared word at `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x N consecutive 32-bit columns: thread i of the warp gets lane
// (lane base + i), registers = columns in order.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t b2u(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Columns of TMEM per CTA for `nthreads` threads: per group of 128 rows a
// 32-column head accumulator and a 32-column correction accumulator (a power
// of two; at most 512 per SM, which the threads per SM guarantee for any mix
// of these kernels up to 1024 threads per SM and otherwise the allocation waits).
__host__ __device__ constexpr int tc_tmem_cols(int nthreads) {
  return nthreads <= 128 ? 64 : nthreads <= 256 ? 128 : nthreads <= 512 ? 256 : 512;
}

// One radix-RS DFT (forward, or adjoint for ADJ) of the RS values a[] of every
// thread's butterfly, on the tensor cores.  Every thread of the CTA calls it
// (block barriers inside); the block's thread count is a multiple of 128.  The
// A tiles alias exchange space that holds no live data at a stage boundary.
// BF16: split-BF16 operands (else split-FP16).
// Failure path: a thread whose completion wait runs out sets the CTA's abort
// word and the error word and leaves a[] as it is (its TMEM row may still be
// written by the MMAs).  The abort word is read after the stage's first
// barrier, so every thread sees the same value: once it is set, no thread
// splits, issues, waits or reads TMEM again, and tc_teardown makes one last
// bounded wait for the outstanding commit before it frees the TMEM columns.
// act = false: the thread writes no operand (its 128-row group has no data this
// round; its rows of the MMAs read whatever the tile holds and are not used).
template <int RS, bool ADJ, bool BF16>
__device__ __forceinline__ void tc_dft(float2 (&a)[RS], TcCtx& tc, bool act = true) {
  typedef TcGeom<RS> G;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int grp = tid >> 7, row = tid & 127;
  const int ngrp = (blockDim.x * blockDim.y * blockDim.z) >> 7;

  // row scale 2^k with max |component| * 2^k in [2^14, 2^15)
  float mx = 0.f;
#pragma unroll
  for (int r = 0; r < RS; ++r) mx = fmaxf(mx, fmaxf(fabsf(a[r].x), fabsf(a[r].y)));
  const int be = (__float_as_int(mx) >> 23) & 0xff;
  int k = be ? 141 - be : 0;
  k = k > 126 ? 126 : k;
  const float s = __int_as_float((127 + k) << 23), is = __int_as_float((127 - k) << 23);
  constexpr float kRound16 = 201326592.0f;    // 1.5 * 2^27: (t + c) - c rounds t to a multiple of 16
  constexpr float kRound128 = 1610612736.0f;  // 1.5 * 2^30: to a multiple of 128

  __syncthreads();  // every exchange read of the previous stage is done
  const bool aborted = *tc.abort != 0;
  if (!aborted && act) {
    const uint32_t base = tc.a_tile + grp * G::kATile + (row >> 3) * G::kSBO + (row & 7) * 16;
    const uint32_t base3 = tc.a_tile3 + grp * G::kAPiece + (row >> 3) * G::kSBO + (row & 7) * 16;
#pragma unroll
    for (int kc = 0; kc < RS / 4; ++kc) {
      uint32_t hi[4], lo[4], l3[4];
      if constexpr (BF16) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float tx = a[4 * kc + e].x * s, ty = a[4 * kc + e].y * s;
          const float hx = __fsub_rn(__fadd_rn(tx, kRound128), kRound128);
          const float hy = __fsub_rn(__fadd_rn(ty, kRound128), kRound128);
          const float rx = __fsub_rn(tx, hx), ry = __fsub_rn(ty, hy);
          const __nv_bfloat162 m = __floats2bfloat162_rn(rx, ry);
          const float2 mf = __bfloat1622float2(m);
          hi[e] = b2u(__floats2bfloat162_rn(hx, hy));
          lo[e] = b2u(m);
          l3[e] = b2u(__floats2bfloat162_rn(__fsub_rn(rx, mf.x), __fsub_rn(ry, mf.y)));
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base3 + kc * 128), "r"(l3[0]),
                     "r"(l3[1]), "r"(l3[2]), "r"(l3[3])
                     : "memory");
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float tx = a[4 * kc + e].x * s, ty = a[4 * kc + e].y * s;
          const float hx = __fsub_rn(__fadd_rn(tx, kRound16), kRound16);
          const float hy = __fsub_rn(__fadd_rn(ty, kRound16), kRound16);
          hi[e] = h2u(__floats2half2_rn(hx, hy));
          lo[e] = h2u(__floats2half2_rn(__fsub_rn(tx, hx), __fsub_rn(ty, hy)));
        }
      }
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + kc * 128), "r"(hi[0]), "r"(hi[1]),
                   "r"(hi[2]), "r"(hi[3])
                   : "memory");
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + G::kAPiece + kc * 128), "r"(lo[0]),
                   "r"(lo[1]), "r"(lo[2]), "r"(lo[3])
                   : "memory");
    }
  }
  fence_async_smem();
  __syncthreads();
  if (aborted) return;
  if (tid == 0 && !tc.stall) {
    tc_fence_after();
    const uint32_t g0 = tc.bmat + (ADJ ? G::kGDir : 0);
    constexpr uint32_t idesc = BF16 ? G::kIdescBF16 : G::kIdesc;
    // products: p = 0 head -> columns 0..31; the others -> 32..63 (second accumulator)
    //   FP16: A_h G_l, A_l G_h, A_h G_ll, A_l G_l        (A pieces h, l; G pieces h, l, ll)
    //   BF16: A_h G_m, A_m G_h, A_h G_l, A_l G_h, A_m G_m (A pieces h, m, l; G pieces h, m, l)
    constexpr int np = BF16 ? 6 : 5;
#pragma unroll 1
    for (int gi = 0; gi < ngrp; ++gi) {
      const uint32_t a0 = tc.a_tile + gi * G::kATile;
      const uint32_t a3 = tc.a_tile3 + gi * G::kAPiece;
      const uint32_t d = tc.tmem + gi * 64;
#pragma unroll
      for (int p = 0; p < np; ++p) {
        int ai, gj;
        if constexpr (BF16) {
          ai = p == 2 || p == 5 ? 1 : p == 4 ? 2 : 0;
          gj = p == 1 || p == 5 ? 1 : p == 3 ? 2 : 0;
        } else {
          ai = (p == 2 || p == 4) ? 1 : 0;
          gj = p == 1 || p == 4 ? 1 : p == 3 ? 2 : 0;
        }
        const uint32_t ap = ai == 2 ? a3 : a0 + ai * G::kAPiece;
        const uint32_t gp = g0 + gj * G::kGPiece;
#pragma unroll
        for (int ks = 0; ks < G::kKSteps; ++ks)
          tc_mma(d + (p ? 32 : 0), tc_desc(ap + ks * 256, 128, G::kSBO), tc_desc(gp + ks * 256, 128, G::kSBO),
                 idesc, (p > 1 || ks > 0) ? 1u : 0u);
      }
    }
    tc_commit(tc.mbar);
  }
  // warp-uniform outcome: the TMEM loads below are .sync.aligned
  const bool ok = __all_sync(0xffffffffu, mbar_wait(tc.mbar, tc.phase, tc.wait_iters));
  tc.phase ^= 1u;
  if (!ok) {
    *tc.abort = 1;
    if (tc.err) atomicOr(tc.err, kErrMmaWait);
    return;
  }
  tc_fence_after();
  const uint32_t taddr = tc.tmem + ((uint32_t)((tid >> 5) & 3) << 21) + grp * 64;  // lane base 32 (warp % 4)
  // 16 columns (8 complex outputs) at a time: head, then correction added
#pragma unroll
  for (int h = 0; h < RS / 8; ++h) {
    uint32_t r[16];
    tmem_ld16(taddr + h * 16, r);
    tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 8; ++q) a[8 * h + q] = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
    tmem_ld16(taddr + 32 + h * 16, r);
    tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 8; ++q)
      a[8 * h + q] = make_float2(__fadd_rn(a[8 * h + q].x, __uint_as_float(r[2 * q])) * is,
                                 __fadd_rn(a[8 * h + q].y, __uint_as_float(r[2 * q + 1])) * is);
  }
  tc_fence_before();
}


// Shared-memory tail of a tensor-core pass kernel (at the start of its dynamic
// shared memory): the split radix-16 DFT matrices of both directions, the
// mbarrier, the TMEM address word and the abort word.
constexpr int kTcTail = 2 * TcGeom<16>::kGDir + 1024;

// Set up a tensor-core pass: copy the split DFT matrices (kTcTail image made
// by the plan, 16-byte aligned) into the tail, allocate the CTA's TMEM
// columns (warp 0), initialise the mbarrier and clear the abort word.
// ctl: the pass's control word (kTcStallMma).  Contains a block barrier.
__device__ __forceinline__ void tc_setup(TcCtx& tc, unsigned char* tail, const void* gmat, uint32_t a_tile,
                                         int* err, int bf16, uint32_t a_tile3, int ctl) {
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  constexpr int kG = 2 * TcGeom<16>::kGDir;
  for (int i = tid; i < kG / 16; i += nthr)
    reinterpret_cast<uint4*>(tail)[i] = __ldg(static_cast<const uint4*>(gmat) + i);
  uint64_t* mb = reinterpret_cast<uint64_t*>(tail + kG);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tail + kG + 8);
  int* abort_word = reinterpret_cast<int*>(tail + kG + 12);
  if (tid == 0) *abort_word = 0;
  if (tid < 32) {
    tmem_alloc(smem_u32(slot), (uint32_t)tc_tmem_cols(nthr));
    tc_fence_before();
  }
  if (tid == 0) mbar_init(smem_u32(mb), 1);
  fence_async_smem();
  __syncthreads();
  tc_fence_after();
  tc.mbar = smem_u32(mb);
  tc.tmem = *reinterpret_cast<volatile uint32_t*>(slot);
  tc.a_tile = a_tile;
  tc.a_tile3 = a_tile3;
  tc.bf16 = bf16;
  tc.bmat = smem_u32(tail);
  tc.phase = 0u;
  tc.abort = abort_word;
  tc.err = err;
  tc.stall = ctl & kTcStallMma;
  tc.wait_iters = tc.stall ? kTestWaitIters : kWaitIters;
}

// Release the TMEM columns once every thread is done with them (block barrier).
// After an expired wait (abort word set) the last commit may still be
// outstanding: warp 0 first waits for it once more (bounded), then frees.
__device__ __forceinline__ void tc_teardown(const TcCtx& tc) {
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    if (*tc.abort) mbar_wait(tc.mbar, tc.phase ^ 1u, tc.wait_iters);
    __syncwarp();
    tc_fence_after();
    tmem_free(tc.tmem, (uint32_t)tc_tmem_cols(nthr));
  }
}

}  // namespace psatd
