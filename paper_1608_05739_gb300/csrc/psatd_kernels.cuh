// psatd_kernels.cuh -- the PSATD step's pass kernels (templates; instantiated
// per precision and variant by the rows_* / push_* translation units).
//
// Data flow of one step (2D: passes 1, 3, 5; 3D: passes 1-5):
//   1  k_fwd_T<R2C>  x-rows of every input array -> R2C -> half spectrum,
//                    written with the row index b contiguous (tile transpose)
//   2  k_fwd_T<C2C>  (3D) y-lines -> C2C, written z-contiguous
//   3  k_line_push   the last axis: forward FFT of every input component,
//                    the analytic PSATD push per mode (Sec. III.B), inverse FFT
//                    of the E and B components, in place
//   4  k_inv_T<C2C>  (3D) inverse y-lines, read z-contiguous
//   5  k_inv_T<C2R>  inverse x-rows (C2R) into the caller's E and B arrays
// A CTA handles TB lines (blockDim.y) of T = L/EPT threads each (blockDim.x).
// Sources without a plan-time role (the optional NaN / Inf scan of the outputs)
// follow the passes: k_nonfinite.
#pragma once

#include "fft_core.cuh"

namespace psatd {

constexpr int kMaxComp = 11;

// Per-component base pointers of a pass (index = grid z = component slot).
struct LineIO {
  const void* in[kMaxComp];
  void* out[kMaxComp];
  const void* gmat;  // tensor-core passes: split DFT matrices (kTcTail image)
  int* err;          // tensor-core passes: device error word
  int tc_ctl;        // tensor-core passes: control word (kTcStallMma test hook)
  // checked mode (PSATD_FLAG_CHECKED): elements of every input / output array
  // (0: unchecked) and the error word that a failed index check sets
  int64_t in_ext, out_ext;
  int* chk_err;
};

// k-space coefficient table entry (one per |m|-octant point), see tables.cu.
template <typename R>
struct alignas(8 * sizeof(R)) Coef {
  R C_h, C_l;  // cos(x) / N              (hi, lo)
  R S_h, S_l;  // sin(x) / |m| / N        (hi, lo)
  R A1;        // (1 - C) / |m|^2 / N
  R A4;        // (S/(c k) - dt) / (eps0 |m|^2) / N
  R B1;        // (S/x - 1) / (eps0 g0 |m|^2) / N
  R B2;        // (S/x - C) / (eps0 g0 |m|^2) / N
};

template <typename R>
struct PushArgs {
  void* spec;        // spectral scratch, component slot c at spec + c * cs
  int64_t cs;        // component stride (complex elements)
  const Coef<R>* tab;
  int nlines;        // lines along the last axis
  int n_in, n_out;   // component slots read / written
  int form;          // 0 vacuum, 1 J, 2 rho
  int ndim;
  int nx_half;       // nx/2 (Nyquist index along x)
  int lines_per_patch;  // 2D: nx/2 + 1 lines per patch of a batch (line = patch * lpp + kx)
  int ny;            // 3D: lines are (kx, ky), ky fastest
  int tab_row;       // L/2 + 1 entries per table row
  R rx, ry, rz;      // k_i = g0 * r_i * m_i
  R c_h, c_l;        // c (hi, lo)
  R ic_h, ic_l;      // 1/c (hi, lo)
  R s_src;           // 1 / (eps0 c g0)
  R s_a6;            // 1 / (eps0 c^2 g0)
  const void* gmat;  // tensor-core pass: split DFT matrices (kTcTail image)
  int* err;          // tensor-core pass: device error word
  int tc_ctl;        // tensor-core pass: control word (kTcStallMma test hook)
  int64_t tab_ext;   // checked mode: coefficient-table entries (0: unchecked); spectra: n_in * cs
  int* chk_err;      // checked mode: error word of a failed index check
  int scheme;        // 0: PSATD (analytic in time); 1: PSTD (leapfrog, p_h / p_e / p_j / inv_n)
  R p_h, p_e, p_j, inv_n;  // PSTD: dt g0 / 2, c^2 dt g0, dt / eps0, 1/N
  int stag;          // staggered order-p plan (PSATD-p): k_p and half-cell phases below
  const double* kp[3];  // per axis, k_p / g0 for |m| = 0..n/2
  const void* ph[3];    // per axis, exp(-i pi m/n) for m = 0..n/2 (twiddle type)
};

// Error-word bits of the checked mode (PSATD_FLAG_CHECKED): the non-finite scan
// and the passes' index checks; the tensor-core passes use kErrMmaWait (tc_dft.cuh).
constexpr int kErrNonfinite = 1 << 8;
constexpr int kErrBounds = 1 << 9;

// Index check of the checked mode: every thread tests the ends of the element
// ranges it is about to touch against the extents the pass was given; the CTA
// agrees (one barrier) and, when any range falls outside, sets kErrBounds and
// the CTA touches nothing (it returns before its first access).
__device__ __forceinline__ bool cta_out_of_bounds(bool bad, int* err) {
  if (!__syncthreads_or(bad)) return false;
  if (threadIdx.x == 0 && threadIdx.y == 0 && err) atomicOr(err, kErrBounds);
  return true;
}

// Scan `n` elements of each of gridDim.y arrays (at p[y] + off[patch], patches
// along gridDim.z; off == NULL: one array from p[y]) for NaN / Inf and set
// kErrNonfinite in *err on a hit (grid-stride over x).
struct NfPtrs {
  const void* p[6];
};
template <typename R>
__global__ void k_nonfinite(NfPtrs ptrs, const int64_t* __restrict__ off, int64_t n, int* err) {
  const R* a = static_cast<const R*>(ptrs.p[blockIdx.y]) + (off ? off[blockIdx.z] : 0);
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonfinite);
}

// Threads per CTA a transposing pass of length L may use (the register budget
// of 24 elements per thread halves it for the mixed lengths).
template <typename R, int L>
struct RowThreads { static constexpr int value = RowEPT<L>::value >= 20 ? 256 : sizeof(R) == 4 ? 512 : 256; };

// XOR mask of row r's buffer in the transposed stores and reads (TB = 1 << log_tb
// rows): rows spread over the 16 eight-byte bank pairs (at most 16 rows: one row
// per pair; more: two or more rows per pair); it stays inside the line for L < 16.
__device__ __forceinline__ int row_xor(int r, int log_tb, int L) {
  return (log_tb <= 4 ? r * (16 >> log_tb) : r) & 15 & (L - 1);
}

// ---------------------------------------------------------------- pass 1 / 2
// Forward FFT along the contiguous axis of TB consecutive lines b, written out
// with b contiguous: out[a1] + a0*out_sa0 + k*out_sk + b.  R2C: the input rows
// are real (length 2L), the output has L+1 bins (half spectrum).
// TC: radix-16 stages on the tensor cores (1 split-FP16, 2 split-BF16); the
// dynamic shared memory then starts with the kTcTail block and the A tiles
// alias the line buffers.
// Work of one CTA of a transposing pass: row block bx (rows bx TB .. bx TB + TB - 1,
// TB = 1 << log_tb) of plane / patch a0 and component a1, thread (t, g) = (position
// in its line, line in the block); rows b >= nb are idle (they transform zeros and
// store nothing), so that a block may run past the rows of its patch.
struct RowCta {
  int bx, a0, a1, t, g, log_tb;
  int64_t nb;
};

template <typename R, int L, bool R2C, int TC, bool PART>
__device__ __forceinline__ void fwd_T_body(const LineIO& io, const typename Types<R>::W* __restrict__ tw,
                                           int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk,
                                           const int64_t* __restrict__ in_off, const RowCta& cta,
                                           unsigned char* smem_raw, TcCtx& tc) {
  typedef typename Types<R>::C C;
  constexpr int EPT = RowEPT<L>::value;
  typedef FFTPlan<L, EPT> P;
  constexpr int T = P::kT;
  constexpr int NK = R2C ? L + 1 : L;
  C* smem = reinterpret_cast<C*>(smem_raw + (TC ? kTcTail : 0));
  const int log_tb = cta.log_tb;
  const int TB = 1 << log_tb;
  const int t = cta.t, g = cta.g;
  const int64_t b0 = (int64_t)cta.bx * TB;
  const int64_t b = b0 + g;
  // PART: the block may run past the rows (nb) of its plane; else every row is valid
  const bool valid = !PART || b < cta.nb;
  const int rows = PART ? (int)(cta.nb - b0 < TB ? cta.nb - b0 : TB) : TB;  // valid rows of the block
  const int a0 = cta.a0, a1 = cta.a1;
  if (io.in_ext) {  // checked mode: the rows read and the transposed block written
    const int64_t o0c = in_off ? in_off[a0] : a0 * in_sa0;
    const int64_t in_end = valid ? o0c + b * in_sb + (R2C ? 2 * L : L) : 0;
    const int64_t out_end = a0 * out_sa0 + b0 + rows + (int64_t)(NK - 1) * out_sk;
    if (cta_out_of_bounds(in_end > io.in_ext || out_end > io.out_ext || o0c < 0, io.chk_err)) return;
  }
  __shared__ const void* twslot;
  if (t == 0 && g == 0) twslot = tw;
  if constexpr (TC) {  // the A tiles alias the line buffers; split-BF16's third piece follows them
    tc.a_tile = smem_u32(smem);
    tc.a_tile3 = smem_u32(smem + (R2C ? TB * L : L * (TB + 1)));
  }
  ExBuf<C> ex{{smem + g * L, smem + g * L}, 0, &twslot, true};  // one exchange buffer per line
  if constexpr (!TC && T % 32 == 0)
    if (TB <= 8) {  // each line's warps synchronise among themselves between stages
      ex.bar_id = 1 + g;
      ex.bar_n = T;
    }

  C v[EPT];
  {
    const C* row;
    const int64_t o0 = in_off ? in_off[a0] : a0 * in_sa0;  // per-patch offsets of a batch
    if constexpr (R2C)
      row = reinterpret_cast<const C*>(static_cast<const R*>(io.in[a1]) + o0 + b * in_sb);
    else
      row = static_cast<const C*>(io.in[a1]) + o0 + b * in_sb;
#pragma unroll
    for (int m = 0; m < EPT; ++m) v[m] = (!PART || valid) ? row[t + T * m] : mkc(R(0), R(0));
  }
  // twslot visible to every line (else the first exchange barrier publishes it, when it spans the CTA)
  if (P::kStages == 1 || ex.bar_n) __syncthreads();
  block_fft_fwd<R, L, EPT, TC>(v, ex, tw, t, &tc);

  if constexpr (R2C) {
    // X[k] = Fe[k] + W_N^k Fo[k], Fe = (Z[k] + Z*[L-k])/2, Fo = (Z[k] - Z*[L-k])/(2i), k = 0..L,
    // computed straight into the transposed store: Z of row g goes to this line's buffer
    // (XOR-ed by a row-dependent mask so that the column-wise reads hit distinct banks),
    // then each thread produces whole output elements (k, row) and stores them.
    C* zb = ex.next();
    const int xg = row_xor(g, log_tb, L);  // stays inside the line for L < 16
#pragma unroll
    for (int m = 0; m < EPT; ++m) zb[(t + T * m) ^ xg] = v[m];
    __syncthreads();
    // Thread (k0, gg) produces bins k = k0 + j T, j < EPT (all below L), and thread
    // k0 = 0 also bin L; twiddles are loaded in groups of four before their use.
    const typename Types<R>::W* wn = tw + P::kTwEntries;  // W_N^k, N = 2L
    const int tid = g * T + t;
    const int gg = tid & (TB - 1);
    const int k0 = tid >> log_tb;  // in [0, T)
    const int xgg = row_xor(gg, log_tb, L);
    const C* zr = smem + gg * L;
    C* o = static_cast<C*>(io.out[a1]) + a0 * out_sa0 + b0 + (int64_t)k0 * out_sk + gg;
    const int64_t ostep = (int64_t)T * out_sk;
    if (!PART || gg < rows) {
#pragma unroll
    for (int j0 = 0; j0 < EPT; j0 += 4) {
      typename Types<R>::W w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = __ldg(&wn[k0 + (j0 + j) * T]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + (j0 + j) * T;
        const C zk = zr[k ^ xgg];
        const C zm = cconj(zr[(is_pow2(L) ? ((L - k) & (L - 1)) : (k == 0 ? 0 : L - k)) ^ xgg]);
        const C fe = mkc(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y + zm.y));
        const C fo = mkc(R(0.5) * (zk.y - zm.y), R(-0.5) * (zk.x - zm.x));
        o[(j0 + j) * ostep] = cadd(fe, twmul(fo, w[j]));
      }
    }
    if (k0 == 0) {  // k = L: X[L] = Fe[0] - Fo[0]
      const C z0 = zr[0 ^ xgg];
      const C zm = cconj(z0);
      const C fe = mkc(R(0.5) * (z0.x + zm.x), R(0.5) * (z0.y + zm.y));
      const C fo = mkc(R(0.5) * (z0.y - zm.y), R(-0.5) * (z0.x - zm.x));
      o[EPT * ostep] = csub(fe, fo);
    }
    }
  } else {
    C* tile = smem;  // [NK][TB + 1], aliases the exchange buffers
    const int tp = TB + 1;
    __syncthreads();
#pragma unroll
    for (int m = 0; m < EPT; ++m) tile[(t + T * m) * tp + g] = v[m];
    __syncthreads();
    C* ob = static_cast<C*>(io.out[a1]) + a0 * out_sa0 + b0;
    const int nthr = T * TB;
    for (int idx = g * T + t; idx < NK * TB; idx += nthr) {
      const int k = idx >> log_tb, gg = idx & (TB - 1);
      if (!PART || gg < rows) ob[(int64_t)k * out_sk + gg] = tile[k * tp + gg];
    }
  }
}

// Launch bounds: two CTAs of the largest block per SM (at most 64 registers a
// thread).  The tensor-core variants then keep part of each row on the stack,
// but measured faster so than with 128 registers and half the resident warps.
template <typename R, int L, bool R2C, int TC = 0>
__global__ void __launch_bounds__(RowThreads<R, L>::value, 2) k_fwd_T(LineIO io, const typename Types<R>::W* __restrict__ tw,
                                               int64_t in_sa0, int64_t in_sb, int64_t out_sa0,
                                               int64_t out_sk, int log_tb, const int64_t* __restrict__ in_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcCtx tc;
  if constexpr (TC) tc_setup(tc, smem_raw, io.gmat, 0u, io.err, TC == 2, 0u, io.tc_ctl);
  const RowCta cta{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)threadIdx.x, (int)threadIdx.y, log_tb,
                   (int64_t)gridDim.x << log_tb};
  fwd_T_body<R, L, R2C, TC, false>(io, tw, in_sa0, in_sb, out_sa0, out_sk, in_off, cta, smem_raw, tc);
  if constexpr (TC) tc_teardown(tc);
}

// ---------------------------------------------------------------- pass 4 / 5
// Adjoint data movement of k_fwd_T: read TB consecutive b of every bin k from
// in[a1] + a0*in_sa0 + k*in_sk + b, inverse FFT along k, write the lines
// contiguously to out[a1] + a0*out_sa0 + b*out_sb.  C2R: L+1 Hermitian bins
// in, real rows of length 2L out (unnormalised).
template <typename R, int L, bool C2R, int TC, bool PART>
__device__ __forceinline__ void inv_T_body(const LineIO& io, const typename Types<R>::W* __restrict__ tw,
                                           int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb,
                                           const int64_t* __restrict__ out_off, const RowCta& cta,
                                           unsigned char* smem_raw, TcCtx& tc) {
  typedef typename Types<R>::C C;
  constexpr int EPT = RowEPT<L>::value;
  typedef FFTPlan<L, EPT> P;
  constexpr int T = P::kT;
  constexpr int NK = C2R ? L + 1 : L;
  C* smem = reinterpret_cast<C*>(smem_raw + (TC ? kTcTail : 0));
  const int log_tb = cta.log_tb;
  const int TB = 1 << log_tb;
  const int t = cta.t, g = cta.g;
  const int64_t b0 = (int64_t)cta.bx * TB;
  const int64_t b = b0 + g;
  // PART: the block may run past the rows (nb) of its plane; else every row is valid
  const bool valid = !PART || b < cta.nb;
  const int rows = PART ? (int)(cta.nb - b0 < TB ? cta.nb - b0 : TB) : TB;  // valid rows of the block
  const int a0 = cta.a0, a1 = cta.a1;
  if (io.in_ext) {  // checked mode: the transposed block read and the rows written
    const int64_t o0c = out_off ? out_off[a0] : a0 * out_sa0;
    const int64_t in_end = a0 * in_sa0 + b0 + rows + (int64_t)(NK - 1) * in_sk;
    const int64_t out_end = valid ? o0c + b * out_sb + (C2R ? 2 * L : L) : 0;
    if (cta_out_of_bounds(in_end > io.in_ext || out_end > io.out_ext || o0c < 0, io.chk_err)) return;
  }
  __shared__ const void* twslot;
  if (t == 0 && g == 0) twslot = tw;
  if constexpr (TC) {
    tc.a_tile = smem_u32(smem);
    tc.a_tile3 = smem_u32(smem + (C2R ? TB * L : L * (TB + 1)));
  }
  C v[EPT];
  if constexpr (C2R) {
    // Z[k] = Fe + i Fo, Fe = X[k] + X*[L-k], Fo = (X[k] - X*[L-k]) conj(W_N^k), read straight
    // from the transposed spectrum: each thread takes a bin pair (k, L-k) of one line, which
    // also gives Z[L-k] = Fe* + i Fo* (as W_N^(L-k) = -conj(W_N^k)), and writes both into the
    // line's buffer under the row-dependent XOR mask of the forward pass.
    // Thread (p0, gg) takes the pairs pp = p0 + j T, j < EPT/2 (all below L/2), and
    // thread p0 = 0 also the self-paired bin L/2; every load is issued before the first use.
    const typename Types<R>::W* wn = tw + P::kTwEntries;
    const int tid = g * T + t;
    const int gg = tid & (TB - 1);
    const int p0 = tid >> log_tb;  // in [0, T)
    const int xgg = row_xor(gg, log_tb, L);
    C* zr = smem + gg * L;
    const bool gvalid = !PART || gg < rows;
    const C* ib = static_cast<const C*>(io.in[a1]) + a0 * in_sa0 + b0 + gg;
    constexpr int NP = EPT / 2;  // 4 to 12 pairs, taken four (or two) at a time
    constexpr int GP = NP % 4 == 0 ? 4 : 2;
    const C zero = mkc(R(0), R(0));
#pragma unroll
    for (int j0 = 0; j0 < NP; j0 += GP) {
      C xk[GP], xm[GP];
      typename Types<R>::W w[GP];
#pragma unroll
      for (int j = 0; j < GP; ++j) {
        const int pp = p0 + (j0 + j) * T;
        xk[j] = gvalid ? ib[(int64_t)pp * in_sk] : zero;
        xm[j] = gvalid ? ib[(int64_t)(L - pp) * in_sk] : zero;
        w[j] = __ldg(&wn[pp]);
      }
#pragma unroll
      for (int j = 0; j < GP; ++j) {
        const int pp = p0 + (j0 + j) * T;
        const C xmc = cconj(xm[j]);
        const C fe = cadd(xk[j], xmc);
        const C d = csub(xk[j], xmc);
        const C fo = (pp == 0) ? d : twmul_conj(d, w[j]);
        zr[pp ^ xgg] = cadd(fe, cmul_pi(fo));
        if (pp > 0) zr[(L - pp) ^ xgg] = cadd(cconj(fe), cmul_pi(cconj(fo)));
      }
    }
    if (p0 == 0) {  // pp = L/2: X[L/2] pairs with itself
      const C x = gvalid ? ib[(int64_t)(L / 2) * in_sk] : zero;
      const C fe = cadd(x, cconj(x));
      const C fo = twmul_conj(csub(x, cconj(x)), __ldg(&wn[L / 2]));
      zr[(L / 2) ^ xgg] = cadd(fe, cmul_pi(fo));
    }
    __syncthreads();
    const int xg = row_xor(g, log_tb, L);
    const C* zb = smem + g * L;
#pragma unroll
    for (int m = 0; m < EPT; ++m) v[m] = zb[(t + T * m) ^ xg];
  } else {
    C* tile = smem;
    const int tp = TB + 1;
    {
      // L * TB values over T * TB threads: EPT each, all loads issued before the stores
      const C* ib = static_cast<const C*>(io.in[a1]) + a0 * in_sa0 + b0;
      const int nthr = T * TB;
      C tv[EPT];
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const int idx = g * T + t + j * nthr;
        tv[j] = (!PART || (idx & (TB - 1)) < rows) ? ib[(int64_t)(idx >> log_tb) * in_sk + (idx & (TB - 1))]
                                                   : mkc(R(0), R(0));
      }
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const int idx = g * T + t + j * nthr;
        tile[(idx >> log_tb) * tp + (idx & (TB - 1))] = tv[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < EPT; ++m) v[m] = tile[(t + T * m) * tp + g];
    __syncthreads();
  }
  ExBuf<C> ex{{smem + g * L, smem + g * L}, 0, &twslot, true};  // one exchange buffer per line
  if constexpr (!TC && T % 32 == 0)
    if (TB <= 8) {  // line-private stages: the line's own warps synchronise
      ex.bar_id = 1 + g;
      ex.bar_n = T;
    }
  block_fft_inv<R, L, EPT, TC>(v, ex, tw, t, &tc);
  if (PART && !valid) return;
  C* row;
  const int64_t o0 = out_off ? out_off[a0] : a0 * out_sa0;  // per-patch offsets of a batch
  if constexpr (C2R)
    row = reinterpret_cast<C*>(static_cast<R*>(io.out[a1]) + o0 + b * out_sb);
  else
    row = static_cast<C*>(io.out[a1]) + o0 + b * out_sb;
#pragma unroll
  for (int m = 0; m < EPT; ++m) row[t + T * m] = v[m];
}

template <typename R, int L, bool C2R, int TC = 0>
__global__ void __launch_bounds__(RowThreads<R, L>::value, 2) k_inv_T(LineIO io, const typename Types<R>::W* __restrict__ tw,
                                               int64_t in_sa0, int64_t in_sk, int64_t out_sa0,
                                               int64_t out_sb, int log_tb, const int64_t* __restrict__ out_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcCtx tc;
  if constexpr (TC) tc_setup(tc, smem_raw, io.gmat, 0u, io.err, TC == 2, 0u, io.tc_ctl);
  const RowCta cta{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)threadIdx.x, (int)threadIdx.y, log_tb,
                   (int64_t)gridDim.x << log_tb};
  inv_T_body<R, L, C2R, TC, false>(io, tw, in_sa0, in_sk, out_sa0, out_sb, out_off, cta, smem_raw, tc);
  if constexpr (TC) tc_teardown(tc);
}

// ---------------------------------------------------------------- the push
template <typename R>
struct CoefReg {
  R C_h, C_l, S_h, S_l, A1, A4, B1, B2;
};

template <class C, typename R>
__device__ __forceinline__ C rmul(R a, C z) { return mkc(a * z.x, a * z.y); }
// z * (h + l), compensated in float
template <class C, typename R>
__device__ __forceinline__ C rmul2(R h, R l, C z) {
  if constexpr (Types<R>::kComp) return mkc(fmaf(z.x, h, z.x * l), fmaf(z.y, h, z.y * l));
  else return mkc(z.x * h, z.y * h);
}
template <class C> __device__ __forceinline__ C iz(C z) { return cmul_pi(z); }

// (h, l) of a*b for hi/lo pairs a = (ah, al), b = (bh, bl)
template <typename R>
__device__ __forceinline__ void prod2(R ah, R al, R bh, R bl, R& h, R& l) {
  h = ah * bh;
  if constexpr (Types<R>::kComp) l = fmaf(ah, bh, -h) + (ah * bl + al * bh);
  else l = R(0);
}

// TE part (Ex, Ey, Bz; Jx, Jy; rho) of a mode with m = (mx, my, 0).
template <typename R, class C>
__device__ __forceinline__ void push_te(C& E0, C& E1, C& B2, C J0, C J1, C r0, C r1, R mx, R my,
                                        const CoefReg<R>& f, R cS_h, R cS_l, R Sc_h, R Sc_l,
                                        const PushArgs<R>& a, int form) {
  const C mE = cadd(rmul(mx, E0), rmul(my, E1));
  const C mxEz = csub(rmul(mx, E1), rmul(my, E0));
  C e0 = cadd(rmul2(f.C_h, f.C_l, E0), iz(rmul2(cS_h, cS_l, rmul(my, B2))));
  C e1 = csub(rmul2(f.C_h, f.C_l, E1), iz(rmul2(cS_h, cS_l, rmul(mx, B2))));
  C b2 = csub(rmul2(f.C_h, f.C_l, B2), iz(rmul2(Sc_h, Sc_l, mxEz)));
  if (form == 0) {
    const C l = rmul(f.A1, mE);
    e0 = cadd(e0, rmul(mx, l));
    e1 = cadd(e1, rmul(my, l));
  } else {
    const R ss = a.s_src * f.S_h;
    e0 = csub(e0, rmul(ss, J0));
    e1 = csub(e1, rmul(ss, J1));
    const C mxJz = csub(rmul(mx, J1), rmul(my, J0));
    b2 = cadd(b2, iz(rmul(a.s_a6 * f.A1, mxJz)));
    if (form == 1) {
      const C mJ = cadd(rmul(mx, J0), rmul(my, J1));
      const C l = cadd(rmul(f.A1, mE), rmul(f.A4, mJ));
      e0 = cadd(e0, rmul(mx, l));
      e1 = cadd(e1, rmul(my, l));
    } else {
      const C q = iz(csub(rmul(f.B1, r1), rmul(f.B2, r0)));
      e0 = cadd(e0, rmul(mx, q));
      e1 = cadd(e1, rmul(my, q));
    }
  }
  E0 = e0;
  E1 = e1;
  B2 = b2;
}

// TM part (Ez, Bx, By; Jz) of a mode with m = (mx, my, 0); k.E = 0 here.
template <typename R, class C>
__device__ __forceinline__ void push_tm(C& E2, C& B0, C& B1, C J2, R mx, R my, const CoefReg<R>& f,
                                        R cS_h, R cS_l, R Sc_h, R Sc_l, const PushArgs<R>& a,
                                        int form) {
  const C mB = cadd(rmul(mx, B0), rmul(my, B1));
  const C mxBz = csub(rmul(mx, B1), rmul(my, B0));
  C e2 = cadd(rmul2(f.C_h, f.C_l, E2), iz(rmul2(cS_h, cS_l, mxBz)));
  const C lb = rmul(f.A1, mB);
  C b0 = csub(cadd(rmul2(f.C_h, f.C_l, B0), rmul(mx, lb)), iz(rmul2(Sc_h, Sc_l, rmul(my, E2))));
  C b1 = cadd(cadd(rmul2(f.C_h, f.C_l, B1), rmul(my, lb)), iz(rmul2(Sc_h, Sc_l, rmul(mx, E2))));
  if (form != 0) {
    e2 = csub(e2, rmul(a.s_src * f.S_h, J2));
    const R a6 = a.s_a6 * f.A1;
    b0 = cadd(b0, iz(rmul(a6, rmul(my, J2))));
    b1 = csub(b1, iz(rmul(a6, rmul(mx, J2))));
  }
  E2 = e2;
  B0 = b0;
  B1 = b1;
}

// Full 3D mode.
template <typename R, class C>
__device__ __forceinline__ void push_3d(C (&E)[3], C (&B)[3], const C (&J)[3], C r0, C r1, R mx,
                                        R my, R mz, const CoefReg<R>& f, R cS_h, R cS_l, R Sc_h,
                                        R Sc_l, const PushArgs<R>& a, int form) {
  const R m[3] = {mx, my, mz};
  const C mE = cadd(cadd(rmul(mx, E[0]), rmul(my, E[1])), rmul(mz, E[2]));
  const C mB = cadd(cadd(rmul(mx, B[0]), rmul(my, B[1])), rmul(mz, B[2]));
  C mxB[3], mxE[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    mxB[i] = csub(rmul(m[i1], B[i2]), rmul(m[i2], B[i1]));
    mxE[i] = csub(rmul(m[i1], E[i2]), rmul(m[i2], E[i1]));
  }
  C e[3], bb[3];
  const C lb = rmul(f.A1, mB);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    e[i] = cadd(rmul2(f.C_h, f.C_l, E[i]), iz(rmul2(cS_h, cS_l, mxB[i])));
    bb[i] = csub(cadd(rmul2(f.C_h, f.C_l, B[i]), rmul(m[i], lb)), iz(rmul2(Sc_h, Sc_l, mxE[i])));
  }
  if (form == 0) {
    const C l = rmul(f.A1, mE);
#pragma unroll
    for (int i = 0; i < 3; ++i) e[i] = cadd(e[i], rmul(m[i], l));
  } else {
    const R ss = a.s_src * f.S_h;
    const R a6 = a.s_a6 * f.A1;
    C l;
    if (form == 1) {
      const C mJ = cadd(cadd(rmul(mx, J[0]), rmul(my, J[1])), rmul(mz, J[2]));
      l = cadd(rmul(f.A1, mE), rmul(f.A4, mJ));
    } else {
      l = iz(csub(rmul(f.B1, r1), rmul(f.B2, r0)));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      const C mxJ = csub(rmul(m[i1], J[i2]), rmul(m[i2], J[i1]));
      e[i] = cadd(csub(e[i], rmul(ss, J[i])), rmul(m[i], l));
      bb[i] = cadd(bb[i], iz(rmul(a6, mxJ)));
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    E[i] = e[i];
    B[i] = bb[i];
  }
}

// PSTD (Table 1): the leapfrog of the FDTD schemes with spectral derivatives, for
// co-temporal E, B: B -= (dt/2) i k x E; E += c^2 dt i k x B - dt J/eps0;
// B -= (dt/2) i k x E; then the 1/N of the inverse transform.  k = g0 m.
template <typename R, class C>
__device__ __forceinline__ void pstd_modes(C (&E)[3], C (&B)[3], const C (&J)[3], R mx, R my, R mz,
                                           const PushArgs<R>& a) {
  const R m[3] = {mx, my, mz};
  auto curl = [&](const C (&F)[3], C (&out)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      out[i] = csub(rmul(m[i1], F[i2]), rmul(m[i2], F[i1]));
    }
  };
  C t[3];
  curl(E, t);
#pragma unroll
  for (int i = 0; i < 3; ++i) B[i] = csub(B[i], iz(rmul(a.p_h, t[i])));
  curl(B, t);
#pragma unroll
  for (int i = 0; i < 3; ++i) E[i] = csub(cadd(E[i], iz(rmul(a.p_e, t[i]))), rmul(a.p_j, J[i]));
  curl(E, t);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    B[i] = rmul(a.inv_n, csub(B[i], iz(rmul(a.p_h, t[i]))));
    E[i] = rmul(a.inv_n, E[i]);
  }
}

// Layout codes (psatd_layout): 0 3D6, 1 2D6, 2 TE, 3 TM.
// Slot order: 3D6/2D6: E0 E1 E2 B0 B1 B2 [J0 J1 J2] [rho_n rho_np1]
//             TE: E0 E1 B2 [J0 J1] [rho_n rho_np1];  TM: E2 B0 B1 [J2]
// Staggered axes of each slot (bit 0 x, 1 y, 2 z): the Yee positions Ex(x),
// Ey(y), Ez(z), Bx(y,z), By(x,z), Bz(x,y), J as E, rho on the nodes.
template <int LAYOUT>
__device__ __forceinline__ int slot_stagger(int c) {
  if constexpr (LAYOUT == 2) return c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 3 : c == 3 ? 1 : c == 4 ? 2 : 0;
  else if constexpr (LAYOUT == 3) return c == 0 ? 4 : c == 1 ? 6 : c == 2 ? 5 : 4;
  else return c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 4 : c == 3 ? 6 : c == 4 ? 5 : c == 5 ? 3 : c == 6 ? 1 : c == 7 ? 2 : c == 8 ? 4 : 0;
}

template <typename R, int LAYOUT, bool PSTD>
__device__ __forceinline__ void push_slots(typename Types<R>::C* st, int ss, int l, const CoefReg<R>& f,
                                           R mx, R my, R mz, const PushArgs<R>& a,
                                           const typename Types<R>::W* P) {
  typedef typename Types<R>::C C;
  const C Z = mkc(R(0), R(0));
  const int form = a.form;
  R cS_h, cS_l, Sc_h, Sc_l;
  prod2(a.c_h, a.c_l, f.S_h, f.S_l, cS_h, cS_l);
  prod2(a.ic_h, a.ic_l, f.S_h, f.S_l, Sc_h, Sc_l);
  // staggered plans (P != NULL): slot values to true positions on the way in, back on the way out
  const int zmask = a.ndim == 3 ? 7 : 3;
  struct Ref {
    C* p;
    int m;
    const typename Types<R>::W* P;
    __device__ __forceinline__ operator C() const {
      C v = *p;
      if (P) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
          if (m & (1 << ax)) v = twmul(v, P[ax]);
      }
      return v;
    }
    __device__ __forceinline__ Ref& operator=(C v) {
      if (P) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
          if (m & (1 << ax)) v = twmul_conj(v, P[ax]);
      }
      *p = v;
      return *this;
    }
  };
  auto S = [&](int c) -> Ref { return Ref{&st[c * ss + l], slot_stagger<LAYOUT>(c) & zmask, P}; };
  if constexpr (PSTD) {  // J-form or vacuum
    C E[3] = {Z, Z, Z}, B[3] = {Z, Z, Z}, J[3] = {Z, Z, Z};
    if constexpr (LAYOUT == 2) {
      E[0] = S(0); E[1] = S(1); B[2] = S(2);
      if (form) { J[0] = S(3); J[1] = S(4); }
    } else if constexpr (LAYOUT == 3) {
      E[2] = S(0); B[0] = S(1); B[1] = S(2);
      if (form) J[2] = S(3);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        E[i] = S(i);
        B[i] = S(3 + i);
        if (form) J[i] = S(6 + i);
      }
    }
    pstd_modes<R>(E, B, J, mx, my, mz, a);
    if constexpr (LAYOUT == 2) {
      S(0) = E[0]; S(1) = E[1]; S(2) = B[2];
    } else if constexpr (LAYOUT == 3) {
      S(0) = E[2]; S(1) = B[0]; S(2) = B[1];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        S(i) = E[i];
        S(3 + i) = B[i];
      }
    }
    return;
  }
  if constexpr (LAYOUT == 2) {
    C E0 = S(0), E1 = S(1), B2 = S(2);
    const C J0 = form ? S(3) : Z, J1 = form ? S(4) : Z;
    const C r0 = form == 2 ? S(5) : Z, r1 = form == 2 ? S(6) : Z;
    push_te<R>(E0, E1, B2, J0, J1, r0, r1, mx, my, f, cS_h, cS_l, Sc_h, Sc_l, a, form);
    S(0) = E0; S(1) = E1; S(2) = B2;
  } else if constexpr (LAYOUT == 3) {
    C E2 = S(0), B0 = S(1), B1 = S(2);
    const C J2 = form ? S(3) : Z;
    push_tm<R>(E2, B0, B1, J2, mx, my, f, cS_h, cS_l, Sc_h, Sc_l, a, form);
    S(0) = E2; S(1) = B0; S(2) = B1;
  } else if constexpr (LAYOUT == 1) {
    C E0 = S(0), E1 = S(1), E2 = S(2), B0 = S(3), B1 = S(4), B2 = S(5);
    const C J0 = form ? S(6) : Z, J1 = form ? S(7) : Z, J2 = form ? S(8) : Z;
    const C r0 = form == 2 ? S(9) : Z, r1 = form == 2 ? S(10) : Z;
    push_te<R>(E0, E1, B2, J0, J1, r0, r1, mx, my, f, cS_h, cS_l, Sc_h, Sc_l, a, form);
    push_tm<R>(E2, B0, B1, J2, mx, my, f, cS_h, cS_l, Sc_h, Sc_l, a, form);
    S(0) = E0; S(1) = E1; S(2) = E2; S(3) = B0; S(4) = B1; S(5) = B2;
  } else {
    C E[3] = {S(0), S(1), S(2)}, B[3] = {S(3), S(4), S(5)};
    const C J[3] = {form ? S(6) : Z, form ? S(7) : Z, form ? S(8) : Z};
    const C r0 = form == 2 ? S(9) : Z, r1 = form == 2 ? S(10) : Z;
    push_3d<R>(E, B, J, r0, r1, mx, my, mz, f, cS_h, cS_l, Sc_h, Sc_l, a, form);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S(i) = E[i];
      S(3 + i) = B[i];
    }
  }
}

// Signed integer modes (Nyquist -> 0) of a last-axis line's fixed axes and its
// coefficient-table row: 2D lines are kx, 3D lines are (kx, ky), ky fastest.
// Staggered plans keep the Nyquist index (+nx/2 on the half axis, -ny/2 on a full one).
template <typename R>
__device__ __forceinline__ void line_modes(const PushArgs<R>& a, int line, int& mxi, int& myi, int& rowi) {
  if (a.ndim == 2) {
    const int kx = line % a.lines_per_patch;
    mxi = (kx == a.nx_half && !a.stag) ? 0 : kx;
    myi = 0;
    rowi = kx;
  } else {
    const int kx = line / a.ny, ky = line - kx * a.ny;
    mxi = (kx == a.nx_half && !a.stag) ? 0 : kx;
    const int nyh = a.ny >> 1;
    myi = (ky == nyh && !a.stag) ? 0 : (ky < nyh ? ky : ky - a.ny);
    rowi = kx * (nyh + 1) + (ky <= nyh ? ky : a.ny - ky);
  }
}

template <class W> __device__ __forceinline__ W wconj(W w);
template <> __device__ __forceinline__ float4 wconj(float4 w) { return make_float4(w.x, -w.y, w.z, -w.w); }
template <> __device__ __forceinline__ double2 wconj(double2 w) { return make_double2(w.x, -w.y); }
// k_p / g0 and phase of signed mode m along axis ax of a staggered plan (k_p odd, phase conjugate for m < 0)
template <typename R>
__device__ __forceinline__ void stag_axis(const PushArgs<R>& a, int ax, int m, R& k, typename Types<R>::W& w) {
  typedef typename Types<R>::W W;
  const int am = m < 0 ? -m : m;
  const R v = (R)__ldg(&a.kp[ax][am]);
  const W p = __ldg(&static_cast<const W*>(a.ph[ax])[am]);
  k = m < 0 ? -v : v;
  w = m < 0 ? wconj(p) : p;
}

// Bulk asynchronous copy global -> this CTA's shared memory (16-byte aligned
// addresses, a multiple of 16 bytes) completing on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Error-word bit of an expired wait for the fused pass's staged inputs.
constexpr int kErrStageWait = 2;

// Staging state of the fused pass: the mbarrier its bulk copies complete on and
// the parity of that mbarrier's next phase (one phase per line block).
struct StageCtx {
  uint32_t mbar;
  uint32_t phase;
  int* err;
};
// Set up by one thread of the kernel before its first barrier.
__device__ __forceinline__ void stage_init(StageCtx& sc, uint64_t* mbar_word, int* err) {
  sc.mbar = smem_u32(mbar_word);
  sc.phase = 0u;
  sc.err = err;
  if (threadIdx.x == 0 && threadIdx.y == 0) mbar_init(sc.mbar, 1);
}

// The push of the EPT modes l = t + T m of one line, in the slots at positions
// sw<kLastCX>(l): PSATD reads the coefficient table (two modes per iteration,
// both loads issued together), PSTD none; staggered plans rotate every slot
// value to its Yee position and back around the update.
// With G component groups (grp < G) the thread takes the modes m = grp + G i
// (EPT / G of them, an even count) and the other groups' threads t the rest.
template <typename R, int L, int LAYOUT, int EPT, bool STAG, bool PSTD>
__device__ __forceinline__ void push_line_modes(typename Types<R>::C* st, int ss, const PushArgs<R>& a,
                                                const Coef<R>* trow, int t, int grp, int G, int mxi, int myi,
                                                R kpx, R kpy, typename Types<R>::W phx, typename Types<R>::W phy) {
  typedef typename Types<R>::W Wt;
  typedef FFTPlan<L, EPT> P;
  constexpr int T = P::kT;
  constexpr int CXL = P::kLastCX;
  // coefficient pairs software-pipelined: the next pair's loads are issued
  // before the current pair's update
  auto coef = [&](int l) -> Coef<R> {
    if constexpr (!PSTD) return trow[(l <= L / 2) ? l : L - l];  // |m| along the line axis
    else return Coef<R>{};
  };
  const int nm = EPT / G;
  Coef<R> qn[2] = {coef(t + T * grp), coef(t + T * (grp + G))};
#pragma unroll 1
  for (int m0 = 0; m0 < nm; m0 += 2) {
    const Coef<R> q[2] = {qn[0], qn[1]};
    if (m0 + 2 < nm) {
      qn[0] = coef(t + T * (grp + G * (m0 + 2)));
      qn[1] = coef(t + T * (grp + G * (m0 + 3)));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = t + T * (grp + G * (m0 + h));
      CoefReg<R> f;
      f.C_h = q[h].C_h; f.C_l = q[h].C_l; f.S_h = q[h].S_h; f.S_l = q[h].S_l;
      f.A1 = q[h].A1; f.A4 = q[h].A4; f.B1 = q[h].B1; f.B2 = q[h].B2;
      R mx, my, mz;
      if constexpr (STAG) {
        const int ml = l < L / 2 ? l : l - L;
        R kl;
        Wt pl;
        stag_axis(a, a.ndim == 2 ? 1 : 2, ml, kl, pl);
        Wt Ph[3];
        Ph[0] = phx;
        if (a.ndim == 2) {
          mx = kpx; my = kl; mz = R(0);
          Ph[1] = pl;
          Ph[2] = phy;
        } else {
          mx = kpx; my = kpy; mz = kl;
          Ph[1] = phy;
          Ph[2] = pl;
        }
        push_slots<R, LAYOUT, PSTD>(st, ss, sw<CXL>(l), f, mx, my, mz, a, Ph);
      } else {
        const int ml = (l == L / 2) ? 0 : (l < L / 2 ? l : l - L);
        if (a.ndim == 2) {
          mx = a.rx * R(mxi); my = a.ry * R(ml); mz = R(0);
        } else {
          mx = a.rx * R(mxi); my = a.ry * R(myi); mz = a.rz * R(ml);
        }
        push_slots<R, LAYOUT, PSTD>(st, ss, sw<CXL>(l), f, mx, my, mz, a, nullptr);
      }
    }
  }
}

// Fused last-axis pass: for TB lines (kx in 2D, (kx, ky) in 3D), forward FFT
// of every input slot, per-mode push, inverse FFT of the n_out field slots,
// written back in place.  Shared memory, component-major: slot c of the TB
// lines (TB x L values, line g at offset g L), c < n_in, then one extra
// exchange buffer per line (contiguous, so that in the tensor-core variant TC
// they hold the A tiles of the CTA's 128-row groups); a slot doubles as the
// other exchange buffer of its own transforms, and in split-BF16 the TB lines'
// slot c of the component being transformed holds the third A piece (no line
// keeps live data there at a tensor-core stage boundary), so the pass needs no
// further region.  After its forward FFT a slot holds the spectrum at positions
// sw<kLastCX>(t + T m), so the push and the inverse FFT's first exchange only
// touch each thread's own positions.
// EPT: elements per thread, 8 (radix-8 stages) or 16 (radix-16 stages; the
// only choice of the tensor-core variant).
// Component groups (G > 1, T a multiple of 32, no tensor-core stages): each
// line has G x T threads; group grp transforms the input components c = grp,
// grp + G, ... and the output components c = G - 1 - grp, 2G - 1 - grp, ...
// (the groups with an extra forward transform get one fewer inverse one), with
// its own second exchange buffer per line and its own named barrier (id
// 1 + g G + grp over its T threads), so that the groups run side by side; the
// whole CTA meets at a block barrier before and after the push, in which the
// groups split each thread position's modes.  G = 1 is the plain pass (block
// barriers throughout, as the tensor-core stages need).
// Body of one CTA of the fused pass: line block bx (lines bx tb .. bx tb + tb - 1,
// line g of the block handled by the threads g T .. g T + T - 1 of each
// component group, t their position).
// GRP: the component-group variant (a kernel of its own, so that the plain pass
// compiles with G = 1 as a constant).
template <typename R, int L, int LAYOUT, int TC, int EPT, bool GRP = false>
__device__ __forceinline__ void line_push_body(const PushArgs<R>& a_in, const typename Types<R>::W* __restrict__ tw,
                                               int bx, int t, int g, int tb, int grp, int G, unsigned char* smem_raw,
                                               TcCtx& tc, StageCtx& sc) {
  // a private copy: its scalars stay in registers through the shared-memory stores of the transforms
  const PushArgs<R> a = a_in;
  typedef typename Types<R>::C C;
  static_assert(!TC || EPT == 16, "tensor-core stages are radix 16");
  typedef FFTPlan<L, EPT> P;
  constexpr int T = P::kT;
  constexpr int CXL = P::kLastCX;
  static_assert(!GRP || TC || T % 32 == 0, "SIMT component groups need whole-warp lines");
  if constexpr (!GRP) {  // the plain pass
    grp = 0;
    G = 1;
  }
  const int line = bx * tb + g;
  const bool valid = line < a.nlines;
  if (a.tab_ext) {  // checked mode: the line's columns of every slot and its coefficient row
    int mx_c, my_c, row_c;
    line_modes(a, valid ? line : 0, mx_c, my_c, row_c);
    const bool bad = (valid && (int64_t)(line + 1) * L > a.cs) ||
                     (int64_t)(row_c + 1) * a.tab_row > a.tab_ext || row_c < 0;
    if (cta_out_of_bounds(bad, a.chk_err)) return;
  }
  C* base = reinterpret_cast<C*>(smem_raw + (TC ? kTcTail : 0));
  const int ss = tb * L;               // slot stride (component-major)
  C* st = base + g * L;                // this line's slot 0; slot c at st + c * ss
  C* bufB = base + a.n_in * ss + (grp * tb + g) * L;  // this group's second exchange buffer
  C* spec = static_cast<C*>(a.spec);
  __shared__ const void* twslot;
  if (t == 0 && g == 0 && grp == 0) twslot = tw;
  // exchange barrier of this line's group: the block's (G = 1), else a named one.
  // Only kernels whose lines have whole warps (T a multiple of 32) contain the
  // named barrier at all: its thread count must be a multiple of the warp size.
  int bar_id = 0, bar_n = 0;
  if constexpr (GRP && !TC) {
    bar_id = 1 + g * G + grp;
    bar_n = T;
  }
  if constexpr (TC) tc.a_tile = smem_u32(base + a.n_in * ss);  // split-BF16's third A piece: per component below

  int mxi, myi, rowi;
  line_modes(a, valid ? line : 0, mxi, myi, rowi);
  typedef typename Types<R>::W Wt;
  R kpx = R(0), kpy = R(0);
  Wt phx{}, phy{};
  if (a.stag) {
    stag_axis(a, 0, mxi, kpx, phx);
    if (a.ndim == 3) stag_axis(a, 1, myi, kpy, phy);
  }
  const Coef<R>* trow = a.tab + (int64_t)rowi * a.tab_row;
  // the push needs EPT coefficient entries per thread: start bringing them
  // into L2 now, so that its loads do not wait on DRAM one mode after another
#pragma unroll
  for (int m = grp; m < EPT; m += G) {
    const int l = t + T * m;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(trow + ((l <= L / 2) ? l : L - l)));
  }
  // stage every input slot of the block's lines: one bulk copy per line and
  // slot, issued by one thread, completing on the stage mbarrier; lines past
  // the last are zero-filled.  The barrier before the issue orders every earlier
  // access to this shared memory (the previous line block's, in a persistent
  // CTA) before the copies, the proxy fence the generic stores among them.
  {
    if (!valid) {
      constexpr int CH = (L * (int)sizeof(C)) / 16;  // 16-byte chunks per slot
      for (int c = 0; c < a.n_in; ++c) {
        float4* dst = reinterpret_cast<float4*>(st + c * ss);
        for (int i = t + grp * T; i < CH; i += G * T) dst[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const int line0 = bx * tb;
    const int nv = a.nlines - line0 < tb ? a.nlines - line0 : tb;  // valid lines of the block
    __syncthreads();
    if (t == 0 && g == 0 && grp == 0) {
      constexpr uint32_t bytes = (uint32_t)(L * sizeof(C));
      fence_async_smem();
      mbar_arrive_expect_tx(sc.mbar, (uint32_t)(nv * a.n_in) * bytes);
      for (int gl = 0; gl < nv; ++gl)
        for (int c = 0; c < a.n_in; ++c)
          bulk_copy_g2s(smem_u32(base + c * ss + gl * L), spec + c * a.cs + (int64_t)(line0 + gl) * L, bytes,
                        sc.mbar);
    }
    // bounded wait; on expiry the error word is set and one more bounded wait
    // lets copies still in flight land before the buffers are used
    if (!mbar_wait(sc.mbar, sc.phase, kWaitIters)) {
      if (sc.err) atomicOr(sc.err, kErrStageWait);
      mbar_wait(sc.mbar, sc.phase, kWaitIters);
    }
    sc.phase ^= 1u;
  }
  C v[EPT];
  if constexpr (TC && GRP) {
    // Tensor-core component pairs: the two groups (128 rows each) transform the
    // components c0 and c0 + 1 in lockstep, so that every tensor-core round (block
    // barriers, one issuing thread, one commit) serves both; a group with no
    // component in the last pair only takes part in the barriers and rounds.  Each
    // component exchanges in its own slot (one buffer), its A_h / A_m tiles sit in
    // that slot at the round (group j's at tc.a_tile + j x tile size = slot c0 + j:
    // the slot stride of 128 rows of 16 complex values equals the tile size) and
    // both third pieces in the spare region; the shared memory is the one-group
    // pass's, with twice its threads.
    tc.a_tile3 = smem_u32(base + a.n_in * ss);
    for (int c0 = 0; c0 < a.n_in; c0 += 2) {
      const int c = c0 + grp;
      const bool act = c < a.n_in;
      C* sl = st + (act ? c : c0) * ss;
#pragma unroll
      for (int m = 0; m < EPT; ++m) v[m] = act ? sl[t + T * m] : mkc(R(0), R(0));
      ExBuf<C> ex{{sl, sl}, 0, &twslot, true};
      tc.a_tile = smem_u32(base + c0 * ss);
      block_fft_fwd<R, L, EPT, TC>(v, ex, tw, t, &tc, act);
      if (act) {
#pragma unroll
        for (int m = 0; m < EPT; ++m) sl[sw<CXL>(t + T * m)] = v[m];
      }
    }
  } else {
    for (int c = grp; c < a.n_in; c += G) {
      C* sl = st + c * ss;
#pragma unroll
      for (int m = 0; m < EPT; ++m) v[m] = sl[t + T * m];
      ExBuf<C> ex{{sl, bufB}, 0, &twslot, false, bar_id, bar_n};
      ex.sync();  // the slot becomes an exchange buffer
      if constexpr (TC) tc.a_tile3 = smem_u32(base + c * ss);
      if constexpr (TC == 0 && (EPT == 8 || EPT == 12))
        block_fft_fwd_pf<R, L, EPT>(v, ex, t);
      else
        block_fft_fwd<R, L, EPT, TC>(v, ex, tw, t, &tc);
#pragma unroll
      for (int m = 0; m < EPT; ++m) sl[sw<CXL>(t + T * m)] = v[m];
    }
  }
  if (G > 1) __syncthreads();  // every group's spectra are in their slots

  // push every mode of the line (each thread its own positions); one loop per
  // (staggered?, PSTD?) combination, chosen once per CTA
  if (a.scheme == 0) {
    if (a.stag)
      push_line_modes<R, L, LAYOUT, EPT, true, false>(st, ss, a, trow, t, grp, G, mxi, myi, kpx, kpy, phx, phy);
    else
      push_line_modes<R, L, LAYOUT, EPT, false, false>(st, ss, a, trow, t, grp, G, mxi, myi, kpx, kpy, phx, phy);
  } else {
    if (a.stag)
      push_line_modes<R, L, LAYOUT, EPT, true, true>(st, ss, a, trow, t, grp, G, mxi, myi, kpx, kpy, phx, phy);
    else
      push_line_modes<R, L, LAYOUT, EPT, false, true>(st, ss, a, trow, t, grp, G, mxi, myi, kpx, kpy, phx, phy);
  }
  if (G > 1) __syncthreads();  // every mode is pushed

  if constexpr (TC && GRP) {  // output pairs in lockstep, as the input pairs above
    for (int c0 = 0; c0 < a.n_out; c0 += 2) {
      const int c = c0 + grp;
      const bool act = c < a.n_out;
      C* sl = st + (act ? c : c0) * ss;
#pragma unroll
      for (int m = 0; m < EPT; ++m) v[m] = act ? sl[sw<CXL>(t + T * m)] : mkc(R(0), R(0));
      ExBuf<C> ex{{sl, sl}, 0, &twslot, true};
      tc.a_tile = smem_u32(base + c0 * ss);
      block_fft_inv<R, L, EPT, TC>(v, ex, tw, t, &tc, act);
      if (act && valid) {
        C* dst = spec + c * a.cs + (int64_t)line * L;
#pragma unroll
        for (int m = 0; m < EPT; ++m) dst[t + T * m] = v[m];
      }
    }
    return;
  }
  for (int c = G - 1 - grp; c < a.n_out; c += G) {
    C* sl = st + c * ss;
#pragma unroll
    for (int m = 0; m < EPT; ++m) v[m] = sl[sw<CXL>(t + T * m)];
    ExBuf<C> ex{{sl, bufB}, 0, &twslot, false, bar_id, bar_n};
    if constexpr (TC) tc.a_tile3 = smem_u32(base + c * ss);
    if constexpr (TC == 0 && (EPT == 8 || EPT == 12))
      block_fft_inv_pf<R, L, EPT>(v, ex, t);
    else
      block_fft_inv<R, L, EPT, TC>(v, ex, tw, t, &tc);
    if (valid) {
      C* dst = spec + c * a.cs + (int64_t)line * L;
#pragma unroll
      for (int m = 0; m < EPT; ++m) dst[t + T * m] = v[m];
    }
  }
}

// Block (T, lines per CTA, component groups); the group variant (GRP) takes up
// to 512 threads (the tensor-core pairs 256), the plain pass 256 (or T).
template <typename R, int L, int LAYOUT, int TC = 0, int EPT = PushEPT<L, TC>::value, bool GRP = false>
__global__ void __launch_bounds__(GRP ? 512 : (FFTPlan<L, EPT>::kT > 256 ? FFTPlan<L, EPT>::kT : 256))
k_line_push(PushArgs<R> a, const typename Types<R>::W* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t stage_mbar;
  StageCtx sc;
  stage_init(sc, &stage_mbar, a.err ? a.err : a.chk_err);
  TcCtx tc;
  if constexpr (TC) tc_setup(tc, smem_raw, a.gmat, 0u, a.err, TC == 2, 0u, a.tc_ctl);  // has a block barrier
  else __syncthreads();  // the stage mbarrier is initialised
  line_push_body<R, L, LAYOUT, TC, EPT, GRP>(a, tw, (int)blockIdx.x, (int)threadIdx.x, (int)threadIdx.y,
                                             (int)blockDim.y, (int)threadIdx.z, (int)blockDim.z, smem_raw, tc, sc);
  if constexpr (TC) tc_teardown(tc);
}


}  // namespace psatd
