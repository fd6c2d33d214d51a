// fft_core.cuh -- register/shared-memory Stockham FFT building blocks for sm_103a.
//
// A length-L transform is computed by T = L/EPT threads; thread t holds the EPT
// elements x[t + T*m], m < EPT, in registers before and after the transform
// (natural order in both domains).  Lengths: powers of two 8..4096 with 8 or
// 16 elements per thread (a radix-2/4/8 first stage, then radix-EPT stages),
// 3 * 2^k, 48..3072, with 24 (radix 3, then 2/4, then 8) or 12 (prime-factor
// radix 12, then 2, then 4), or 5 * 2^k, 80..1280, with 20 (radix 5, then 2,
// then 4) -- FFTPlan below.  Between stages the data go
// through shared memory in rows of 16 elements whose columns are XOR-swizzled
// per exchange (free of bank conflicts for each stage's write pattern).
//
// Forward = Stockham decimation in time: stage (radix R, span Ns) multiplies
// input r of butterfly j by w^(r*k), w = exp(-2 pi i/(Ns R)), k = j mod Ns,
// applies the radix-R DFT and writes output r to (j - k) R + k + r Ns.
// Inverse = the exact adjoint of the forward (stages in reverse order, adjoint
// butterflies, conjugated twiddles), i.e. the unnormalised inverse DFT.  With
// the adjoint, a forward/inverse round trip deviates from N*I only through
// |w| != 1; in FP32 the twiddles and the sqrt(1/2) constant are therefore
// applied in compensated form (hi + lo parts, FMA), which keeps the round
// trip free of systematic gain over thousands of steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "tc_dft.cuh"

namespace psatd {

template <typename R> struct Types;
template <> struct Types<float> {
  typedef float2 C;   // complex value
  typedef float4 W;   // twiddle: (re_hi, im_hi, re_lo, im_lo)
  static constexpr bool kComp = true;
};
template <> struct Types<double> {
  typedef double2 C;
  typedef double2 W;  // twiddle: (re, im)
  static constexpr bool kComp = false;
};

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul_mi(C a) { return mkc(a.y, -a.x); }  // * (-i)
template <class C> __device__ __forceinline__ C cmul_pi(C a) { return mkc(-a.y, a.x); }  // * (+i)
template <class C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }

// x * w, compensated: the low parts enter first, the leading product last.
__device__ __forceinline__ float2 twmul(float2 x, float4 w) {
  float re = fmaf(x.x, w.z, -x.y * w.w);
  float im = fmaf(x.x, w.w, x.y * w.z);
  re = fmaf(-x.y, w.y, re);
  im = fmaf(x.y, w.x, im);
  re = fmaf(x.x, w.x, re);
  im = fmaf(x.x, w.y, im);
  return make_float2(re, im);
}
// x * conj(w), compensated.
__device__ __forceinline__ float2 twmul_conj(float2 x, float4 w) {
  float re = fmaf(x.x, w.z, x.y * w.w);
  float im = fmaf(x.y, w.z, -x.x * w.w);
  re = fmaf(x.y, w.y, re);
  im = fmaf(-x.x, w.y, im);
  re = fmaf(x.x, w.x, re);
  im = fmaf(x.y, w.x, im);
  return make_float2(re, im);
}
__device__ __forceinline__ double2 twmul(double2 x, double2 w) {
  return make_double2(fma(x.x, w.x, -x.y * w.y), fma(x.x, w.y, x.y * w.x));
}
__device__ __forceinline__ double2 twmul_conj(double2 x, double2 w) {
  return make_double2(fma(x.x, w.x, x.y * w.y), fma(x.y, w.x, -x.x * w.y));
}

// v * sqrt(1/2); in float as hi + lo (0.70710677f + 1.2101617e-8f).
__device__ __forceinline__ float rsqrt2_mul(float v) { return fmaf(v, 0.70710677f, v * 1.2101617e-08f); }
__device__ __forceinline__ double rsqrt2_mul(double v) { return v * 0.70710678118654752440; }

// ---------------------------------------------------------------- butterflies
// Radix-4 DFT in place (forward: exp(-2 pi i/4) = -i; adjoint: +i).  Exact
// operations apart from the additions, so the adjoint is exact.
template <bool ADJ, class C>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C s0 = cadd(x0, x2), d0 = csub(x0, x2), s1 = cadd(x1, x3), t = csub(x1, x3);
  C d1 = ADJ ? cmul_pi(t) : cmul_mi(t);
  x0 = cadd(s0, s1);
  x1 = cadd(d0, d1);
  x2 = csub(s0, s1);
  x3 = csub(d0, d1);
}

// Radix-8 forward DFT, natural order in and out: split a_r +- a_(r+4), rotate
// the difference half by w8^r, two radix-4 DFTs interleaved.
template <class C>
__device__ __forceinline__ void dft8_fwd(C* a) {
  C b0 = cadd(a[0], a[4]), b1 = cadd(a[1], a[5]), b2 = cadd(a[2], a[6]), b3 = cadd(a[3], a[7]);
  C c0 = csub(a[0], a[4]), c1 = csub(a[1], a[5]), c2 = csub(a[2], a[6]), c3 = csub(a[3], a[7]);
  // c1 *= s(1 - i); c2 *= -i; c3 *= s(-1 - i)
  c1 = mkc(rsqrt2_mul(c1.x + c1.y), rsqrt2_mul(c1.y - c1.x));
  c2 = cmul_mi(c2);
  c3 = mkc(rsqrt2_mul(c3.y - c3.x), rsqrt2_mul(-(c3.x + c3.y)));
  dft4<false>(b0, b1, b2, b3);
  dft4<false>(c0, c1, c2, c3);
  a[0] = b0; a[1] = c0; a[2] = b1; a[3] = c1;
  a[4] = b2; a[5] = c2; a[6] = b3; a[7] = c3;
}

// Exact adjoint of dft8_fwd (reverse order of its steps, conjugate constants).
template <class C>
__device__ __forceinline__ void dft8_adj(C* a) {
  C b0 = a[0], b1 = a[2], b2 = a[4], b3 = a[6];
  C c0 = a[1], c1 = a[3], c2 = a[5], c3 = a[7];
  dft4<true>(b0, b1, b2, b3);
  dft4<true>(c0, c1, c2, c3);
  // c1 *= s(1 + i); c2 *= +i; c3 *= s(-1 + i)
  c1 = mkc(rsqrt2_mul(c1.x - c1.y), rsqrt2_mul(c1.x + c1.y));
  c2 = cmul_pi(c2);
  c3 = mkc(rsqrt2_mul(-(c3.x + c3.y)), rsqrt2_mul(c3.x - c3.y));
  a[0] = cadd(b0, c0); a[1] = cadd(b1, c1); a[2] = cadd(b2, c2); a[3] = cadd(b3, c3);
  a[4] = csub(b0, c0); a[5] = csub(b1, c1); a[6] = csub(b2, c2); a[7] = csub(b3, c3);
}

// Multiplication by constants of the radix-16 DFT: z (p + i q) with p, q the
// double-precision values, applied as hi + lo pairs in float.
template <class C> struct KMul;
template <> struct KMul<float2> {
  template <int P_NUM>
  static __device__ __forceinline__ float2 mul(float2 z, double p, double q) {
    const float ph = (float)p, pl = (float)(p - (double)ph), qh = (float)q, ql = (float)(q - (double)qh);
    float re = z.x * pl;
    re = fmaf(-z.y, ql, re);
    re = fmaf(-z.y, qh, re);
    re = fmaf(z.x, ph, re);
    float im = z.x * ql;
    im = fmaf(z.y, pl, im);
    im = fmaf(z.y, ph, im);
    im = fmaf(z.x, qh, im);
    return make_float2(re, im);
  }
};
template <> struct KMul<double2> {
  template <int P_NUM>
  static __device__ __forceinline__ double2 mul(double2 z, double p, double q) {
    return make_double2(fma(z.x, p, -z.y * q), fma(z.x, q, z.y * p));
  }
};
constexpr double kCos8 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kSin8 = 0.38268343236508977173;  // sin(pi/8)

// z * w16^e (forward, w16 = exp(-2 pi i/16)) or z * conj(w16^e) (adjoint), e in {1,2,3,4,6,9}
template <int E, bool ADJ, class C>
__device__ __forceinline__ C w16mul(C z) {
  constexpr double sg = ADJ ? 1.0 : -1.0;  // sign of the imaginary part of the constant
  if constexpr (E == 1) return KMul<C>::template mul<1>(z, kCos8, sg * kSin8);
  else if constexpr (E == 3) return KMul<C>::template mul<3>(z, kSin8, sg * kCos8);
  else if constexpr (E == 9) { const C u = KMul<C>::template mul<1>(z, kCos8, sg * kSin8); return mkc(-u.x, -u.y); }
  else if constexpr (E == 4) return ADJ ? cmul_pi(z) : cmul_mi(z);
  else if constexpr (E == 2) {
    if constexpr (ADJ) return mkc(rsqrt2_mul(z.x - z.y), rsqrt2_mul(z.x + z.y));
    else return mkc(rsqrt2_mul(z.x + z.y), rsqrt2_mul(z.y - z.x));
  } else {  // E == 6
    if constexpr (ADJ) return mkc(rsqrt2_mul(-(z.x + z.y)), rsqrt2_mul(z.x - z.y));
    else return mkc(rsqrt2_mul(z.y - z.x), rsqrt2_mul(-(z.x + z.y)));
  }
}

// Radix-16 forward DFT, natural order in and out: 4 x 4 decomposition
// (radix-4 DFTs over the stride-4 columns, twiddles w16^(r1 k2), radix-4 DFTs
// over the rows, transposed read-out).
template <class C>
__device__ __forceinline__ void dft16_fwd(C* a) {
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) dft4<false>(a[r1], a[r1 + 4], a[r1 + 8], a[r1 + 12]);
  a[5] = w16mul<1, false>(a[5]);
  a[9] = w16mul<2, false>(a[9]);
  a[13] = w16mul<3, false>(a[13]);
  a[6] = w16mul<2, false>(a[6]);
  a[10] = w16mul<4, false>(a[10]);
  a[14] = w16mul<6, false>(a[14]);
  a[7] = w16mul<3, false>(a[7]);
  a[11] = w16mul<6, false>(a[11]);
  a[15] = w16mul<9, false>(a[15]);
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) dft4<false>(a[4 * k2], a[4 * k2 + 1], a[4 * k2 + 2], a[4 * k2 + 3]);
  C y[16];
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[k2 + 4 * k1] = a[4 * k2 + k1];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = y[i];
}

// Exact adjoint of dft16_fwd.
template <class C>
__device__ __forceinline__ void dft16_adj(C* a) {
  C x[16];
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) x[4 * k2 + k1] = a[k2 + 4 * k1];
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) dft4<true>(x[4 * k2], x[4 * k2 + 1], x[4 * k2 + 2], x[4 * k2 + 3]);
  x[5] = w16mul<1, true>(x[5]);
  x[9] = w16mul<2, true>(x[9]);
  x[13] = w16mul<3, true>(x[13]);
  x[6] = w16mul<2, true>(x[6]);
  x[10] = w16mul<4, true>(x[10]);
  x[14] = w16mul<6, true>(x[14]);
  x[7] = w16mul<3, true>(x[7]);
  x[11] = w16mul<6, true>(x[11]);
  x[15] = w16mul<9, true>(x[15]);
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) dft4<true>(x[r1], x[r1 + 4], x[r1 + 8], x[r1 + 12]);
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = x[i];
}

// v * sqrt(3)/2; in float as hi + lo
constexpr double kHalfSqrt3 = 0.86602540378443864676;
__device__ __forceinline__ float r3_mul(float v) {
  constexpr float h = (float)kHalfSqrt3, l = (float)(kHalfSqrt3 - (double)(float)kHalfSqrt3);
  return fmaf(v, h, v * l);
}
__device__ __forceinline__ double r3_mul(double v) { return v * kHalfSqrt3; }

// Radix-3 DFT in place (forward: exp(-2 pi i/3) = -1/2 - i sqrt3/2; adjoint:
// the conjugate constant): X0 = a0 + (a1 + a2), X1,2 = a0 - (a1 + a2)/2 -+ i
// sqrt3/2 (a1 - a2) (forward), +- (adjoint).
template <bool ADJ, class C>
__device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  const C t = cadd(a1, a2), d = csub(a1, a2);
  const C m = mkc(a0.x - 0.5f * t.x, a0.y - 0.5f * t.y);
  const C sd = mkc(r3_mul(d.x), r3_mul(d.y));
  const C s = ADJ ? cmul_pi(sd) : cmul_mi(sd);
  a0 = cadd(a0, t);
  a1 = cadd(m, s);
  a2 = csub(m, s);
}

// Radix-5 DFT in place.  With t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4,
// t4 = a2 - a3 and c_j = cos(2 pi j/5), s_j = sin(2 pi j/5):
//   X0 = a0 + t1 + t2,  m1 = a0 + c1 t1 + c2 t2,  m2 = a0 + c2 t1 + c1 t2,
//   n1 = s1 t3 + s2 t4,  n2 = s2 t3 - s1 t4,
//   forward (W = exp(-2 pi i/5)): X1,4 = m1 -+ i n1, X2,3 = m2 -+ i n2;
//   adjoint (the conjugate constants): X1,4 = m1 +- i n1, X2,3 = m2 +- i n2.
// The four constants multiply as hi + lo pairs in float.
constexpr double kC51 = 0.30901699437494742410;   // cos(2 pi/5)
constexpr double kC52 = -0.80901699437494742410;  // cos(4 pi/5)
constexpr double kS51 = 0.95105651629515357212;   // sin(2 pi/5)
constexpr double kS52 = 0.58778525229247312917;   // sin(4 pi/5)
template <int K> __device__ __forceinline__ float k5_mul(float v) {
  constexpr double c = K == 0 ? kC51 : K == 1 ? kC52 : K == 2 ? kS51 : kS52;
  constexpr float h = (float)c, l = (float)(c - (double)(float)c);
  return fmaf(v, h, v * l);
}
template <int K> __device__ __forceinline__ double k5_mul(double v) {
  return v * (K == 0 ? kC51 : K == 1 ? kC52 : K == 2 ? kS51 : kS52);
}
template <bool ADJ, class C>
__device__ __forceinline__ void dft5(C* a) {
  const C t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]), t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  const C m1 = mkc(a[0].x + k5_mul<0>(t1.x) + k5_mul<1>(t2.x), a[0].y + k5_mul<0>(t1.y) + k5_mul<1>(t2.y));
  const C m2 = mkc(a[0].x + k5_mul<1>(t1.x) + k5_mul<0>(t2.x), a[0].y + k5_mul<1>(t1.y) + k5_mul<0>(t2.y));
  const C n1 = mkc(k5_mul<2>(t3.x) + k5_mul<3>(t4.x), k5_mul<2>(t3.y) + k5_mul<3>(t4.y));
  const C n2 = mkc(k5_mul<3>(t3.x) - k5_mul<2>(t4.x), k5_mul<3>(t3.y) - k5_mul<2>(t4.y));
  const C in1 = ADJ ? cmul_pi(n1) : cmul_mi(n1), in2 = ADJ ? cmul_pi(n2) : cmul_mi(n2);
  a[0] = cadd(a[0], cadd(t1, t2));
  a[1] = cadd(m1, in1);
  a[4] = csub(m1, in1);
  a[2] = cadd(m2, in2);
  a[3] = csub(m2, in2);
}

// Radix-12 DFT in place, natural order in and out, as the prime-factor
// (Good-Thomas) split 12 = 3 x 4: with n = (4 n1 + 3 n2) mod 12 and
// k = (4 k1 + 9 k2) mod 12, W12^(n k) = W3^(n1 k1) W4^(n2 k2), so radix-3 DFTs
// over n1 and radix-4 DFTs over n2 need no twiddles between them.  The adjoint
// runs the same steps in reverse order with the conjugate DFTs.
template <bool ADJ, class C>
__device__ __forceinline__ void dft12(C* a) {
  C y[12];
  if constexpr (!ADJ) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C c0 = a[(3 * n2) % 12], c1 = a[(4 + 3 * n2) % 12], c2 = a[(8 + 3 * n2) % 12];
      dft3<false>(c0, c1, c2);
      y[3 * n2] = c0;
      y[3 * n2 + 1] = c1;
      y[3 * n2 + 2] = c2;
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      C d0 = y[k1], d1 = y[3 + k1], d2 = y[6 + k1], d3 = y[9 + k1];
      dft4<false>(d0, d1, d2, d3);
      a[(4 * k1) % 12] = d0;
      a[(4 * k1 + 9) % 12] = d1;
      a[(4 * k1 + 18) % 12] = d2;
      a[(4 * k1 + 27) % 12] = d3;
    }
  } else {
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
      C d0 = a[(4 * k1) % 12], d1 = a[(4 * k1 + 9) % 12], d2 = a[(4 * k1 + 18) % 12], d3 = a[(4 * k1 + 27) % 12];
      dft4<true>(d0, d1, d2, d3);
      y[k1] = d0;
      y[3 + k1] = d1;
      y[6 + k1] = d2;
      y[9 + k1] = d3;
    }
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C c0 = y[3 * n2], c1 = y[3 * n2 + 1], c2 = y[3 * n2 + 2];
      dft3<true>(c0, c1, c2);
      a[(3 * n2) % 12] = c0;
      a[(4 + 3 * n2) % 12] = c1;
      a[(8 + 3 * n2) % 12] = c2;
    }
  }
}

template <int RS, bool ADJ, class C>
__device__ __forceinline__ void butterfly(C* a) {
  if constexpr (RS == 3) {
    dft3<ADJ>(a[0], a[1], a[2]);
  } else if constexpr (RS == 5) {
    dft5<ADJ>(a);
  } else if constexpr (RS == 12) {
    dft12<ADJ>(a);
  } else if constexpr (RS == 2) {
    C s = cadd(a[0], a[1]), d = csub(a[0], a[1]);
    a[0] = s;
    a[1] = d;
  } else if constexpr (RS == 4) {
    dft4<ADJ>(a[0], a[1], a[2], a[3]);
  } else if constexpr (RS == 8) {
    if constexpr (ADJ) dft8_adj(a); else dft8_fwd(a);
  } else {
    if constexpr (ADJ) dft16_adj(a); else dft16_fwd(a);
  }
}

// ---------------------------------------------------------------- stage plan
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Elements per thread of the transposing row/line passes (16 from L = 16 on)
// and of the fused last-axis pass (8).
__host__ __device__ constexpr bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Lengths 3 * 2^k (k >= 4) are mixed-radix: 24 elements per thread in the
// transposing passes, 12 in the fused pass (whose shared memory per line is
// fixed, so that fewer elements per thread keep more threads on an SM).
// Lengths 5 * 2^k (k >= 4): 20 elements per thread in every pass.
__host__ __device__ constexpr int odd_factor(int v) { return is_pow2(v) ? 1 : (v % 3 == 0 ? 3 : 5); }
template <int L>
struct RowEPT { static constexpr int value = odd_factor(L) == 3 ? 24 : odd_factor(L) == 5 ? 20 : L >= 16 ? 16 : 8; };
// The fused pass keeps 8 elements per thread: with 16 a 2048-point line has
// half the threads and, its shared memory being fixed per line, the SM half
// the warps (measured slower).  The tensor-core variant (TC) takes 16, so that
// its stages are radix-16 DFT-matrix contractions.
template <int L, int TC = 0>
struct PushEPT { static constexpr int value = odd_factor(L) == 3 ? 12 : odd_factor(L) == 5 ? 20 : TC ? 16 : 8; };

// Power-of-two L: a radix-2/4/8 first stage when log2 L is not a multiple of
// log2 EPT, then radix-EPT stages.  Mixed L = 3 * 2^k: with EPT = 24 a radix-3
// first stage, a radix-2 or radix-4 stage when k is not a multiple of 3, then
// radix-8 stages; with EPT = 12 a radix-12 first stage (prime-factor 3 x 4),
// a radix-2 stage when k is odd, then radix-4 stages.  Mixed L = 5 * 2^k
// (EPT = 20): a radix-5 first stage, a radix-2 stage when k is odd, then
// radix-4 stages.  Every radix divides EPT.
template <int L, int EPT = 8>
struct FFTPlan {
  static constexpr int kEPT = EPT;
  static constexpr int kF = odd_factor(L);  // 1, 3 or 5
  static constexpr bool kMixed = kF > 1;
  static constexpr int kLog = ilog2(L / kF);  // log2 of the power-of-two part
  static constexpr int kHeadLog = (kF == 3 && EPT == 12) ? 2 : 0;  // power of two taken by the first stage
  static constexpr int kB = kF == 5 ? 2 : kMixed ? (EPT == 12 ? 2 : 3) : ilog2(EPT);
  static constexpr int kRem = (kLog - kHeadLog) % kB;
  static constexpr int kR0 = kMixed ? kF << kHeadLog : kRem ? (1 << kRem) : EPT;
  static constexpr int kStages = kMixed ? 1 + (kRem ? 1 : 0) + (kLog - kHeadLog) / kB
                                        : kRem ? kLog / kB + 1 : kLog / kB;
  static constexpr int kT = L / EPT;
  static constexpr int kBuf = L;  // exchange buffer (XOR-swizzled, no padding)
  __host__ __device__ static constexpr int radix(int s) {
    if (kMixed) return s == 0 ? kR0 : (s == 1 && kRem) ? (1 << kRem) : (1 << kB);
    return s == 0 ? kR0 : EPT;
  }
  __host__ __device__ static constexpr int span(int s) {  // Ns of stage s
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= radix(i);
    return ns;
  }
  // offset of stage s's twiddle block in the stage table (stages s >= 1)
  __host__ __device__ static constexpr int tw_off(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += (radix(i) - 1) * span(i);
    return o;
  }
  // entries of the stage table: sum over s >= 1 of (R_s - 1) Ns_s = L - R_0
  static constexpr int kTwEntries = L - kR0;
  // XOR multiplier of the exchange written by stage s (bank-conflict free for
  // the Stockham write pattern of that stage and the contiguous reads after it)
  __host__ __device__ static constexpr int swz(int s) {
    return (kMixed || EPT == 16) ? 1 : (span(s) == 1 ? 1 : 10);
  }
  // swizzle of the last exchange: forward output / inverse input positions
  // sw<kLastCX>(t + T m) are each touched by their own thread only
  static constexpr int kLastCX = (kStages >= 2) ? swz(kStages - 2) : 0;
  static_assert(kF == 3   ? (L == 3 * (1 << kLog) && (EPT == 24 || EPT == 12) && kLog >= 4)
                : kF == 5 ? (L == 5 * (1 << kLog) && EPT == 20 && kLog >= 4)
                          : (L >= EPT && EPT != 24 && EPT != 12 && EPT != 20),
                "L must be a power of two >= EPT, 3 * 2^k (k >= 4) with EPT = 12 or 24, or 5 * 2^k with EPT 20");
};

// element i of an exchange buffer, rows of 16 elements (128 B) XOR-swizzled
template <int CX>
__device__ __forceinline__ int sw(int i) { return i ^ (((i >> 4) * CX) & 15); }

// Two exchange buffers used alternately: consecutive exchanges never share a
// buffer, so one barrier per exchange suffices.  `twslot` is a shared-memory
// word holding the twiddle table's address (written before the kernel's first
// barrier): each stage reads it back, which ties that stage's twiddle loads to
// the stage (the compiler cannot prefetch every stage's twiddles of every
// transform in a kernel into registers).
// With b[0] == b[1] (one buffer, `single`), next() adds the barrier that lets
// the previous exchange's reads finish before the buffer is overwritten.
// The exchange barrier: the whole CTA (bar_n == 0), or, when each line's
// transform is private to its own warps, the named barrier bar_id over the
// line's bar_n threads (a multiple of 32), so that lines do not wait for one
// another between stages.
template <class C>
struct ExBuf {
  C* b[2];
  int cur;
  const void* const* twslot;
  bool single;
  int bar_id = 0;
  int bar_n = 0;
  __device__ __forceinline__ void sync() const {
    if (bar_n) asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(bar_n) : "memory");
    else __syncthreads();
  }
  __device__ __forceinline__ C* next() {
    C* p = b[cur];
    cur ^= 1;
    if (single) sync();
    return p;
  }
};

template <typename R, class C>
__device__ __forceinline__ const typename Types<R>::W* stage_tw(const ExBuf<C>& ex) {
  return reinterpret_cast<const typename Types<R>::W*>(
      const_cast<const void*>(*reinterpret_cast<const void* const volatile*>(ex.twslot)));
}

// Twiddle tables of a length-L transform (built in tables.cu): stage s >= 1
// keeps W_L^(r k L/(Ns R)) at [tw_off(s) + (r-1) Ns + k], k < Ns, 1 <= r < R,
// so the threads of a warp read consecutive entries.

// One forward stage.  act = false: the thread only takes part in the stage's
// barriers (and tensor-core rounds), touching no exchange memory (a component
// group with no component to transform while the other group has one).
template <typename R, int L, int EPT, int S, int TC>
__device__ __forceinline__ void fwd_stage(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                          const typename Types<R>::W* __restrict__ tw, int t, TcCtx* tc,
                                          bool act = true) {
  typedef typename Types<R>::C C;
  typedef FFTPlan<L, EPT> P;
  constexpr int RS = P::radix(S), NS = P::span(S), Q = EPT / RS, T = P::kT;
  constexpr bool LAST = (S == P::kStages - 1);
  constexpr int CX = P::swz(S);
  C* buf = nullptr;
  if constexpr (!LAST) buf = ex.next();
  asm volatile("" : "+r"(t)::"memory");  // stage boundary for the front end
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = is_pow2(NS) ? (j & (NS - 1)) : (int)((unsigned)j % (unsigned)NS);
    C a[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) a[r] = v[q + r * Q];
    if constexpr (NS > 1) {
      if (act) {
        const typename Types<R>::W* tws = stage_tw<R>(ex) + P::tw_off(S) + k;
#pragma unroll
        for (int r = 1; r < RS; ++r) a[r] = twmul(a[r], __ldg(&tws[(r - 1) * NS]));
      }
    }
    if constexpr (TC && RS == 16) tc_dft<16, false, TC == 2>(a, *tc, act);
    else if (act) butterfly<RS, false>(a);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < RS; ++r) v[q + r * Q] = a[r];
    } else if (act) {
      const int base = (j - k) * RS + k;
#pragma unroll
      for (int r = 0; r < RS; ++r) buf[sw<CX>(base + r * NS)] = a[r];
    }
  }
  if constexpr (!LAST) {
    ex.sync();
    if (act) {
#pragma unroll
      for (int m = 0; m < EPT; ++m) v[m] = buf[sw<CX>(t + T * m)];
    }
  }
}

// Adjoint of fwd_stage<S>.
template <typename R, int L, int EPT, int S, int TC>
__device__ __forceinline__ void inv_stage(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                          const typename Types<R>::W* __restrict__ tw, int t, TcCtx* tc,
                                          bool act = true) {
  typedef typename Types<R>::C C;
  typedef FFTPlan<L, EPT> P;
  constexpr int RS = P::radix(S), NS = P::span(S), Q = EPT / RS, T = P::kT;
  constexpr bool FIRST = (S == P::kStages - 1);
  constexpr int CX = P::swz(S);
  C* buf = nullptr;
  if constexpr (!FIRST) {
    buf = ex.next();
    if (act) {
#pragma unroll
      for (int m = 0; m < EPT; ++m) buf[sw<CX>(t + T * m)] = v[m];
    }
    ex.sync();
  }
  asm volatile("" : "+r"(t)::"memory");  // stage boundary (see fwd_stage)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = is_pow2(NS) ? (j & (NS - 1)) : (int)((unsigned)j % (unsigned)NS);
    C a[RS];
    if constexpr (FIRST) {
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = v[q + r * Q];
    } else if (act) {
      const int base = (j - k) * RS + k;
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = buf[sw<CX>(base + r * NS)];
    } else {
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = v[q + r * Q];
    }
    if constexpr (TC && RS == 16) tc_dft<16, true, TC == 2>(a, *tc, act);
    else if (act) butterfly<RS, true>(a);
    if constexpr (NS > 1) {
      if (act) {
        const typename Types<R>::W* tws = stage_tw<R>(ex) + P::tw_off(S) + k;
#pragma unroll
        for (int r = 1; r < RS; ++r) a[r] = twmul_conj(a[r], __ldg(&tws[(r - 1) * NS]));
      }
    }
#pragma unroll
    for (int r = 0; r < RS; ++r) v[q + r * Q] = a[r];
  }
}

// Forward transform with the twiddles of stage s + 1 loaded before stage s's
// exchange barrier (the barrier and the exchange hide their latency; plain
// fwd_stage issues them right before the multiply that needs them).  Holds one
// stage's twiddles in registers (kPF per thread), for kernels with registers to
// spare (the fused pass at 8 elements per thread).
template <int L, int EPT>
struct PFCount {
  typedef FFTPlan<L, EPT> P;
  static constexpr int at(int s) { return s >= 1 && s < P::kStages ? (EPT / P::radix(s)) * (P::radix(s) - 1) : 0; }
  static constexpr int max_from(int s) { return s >= P::kStages ? 1 : (at(s) > max_from(s + 1) ? at(s) : max_from(s + 1)); }
  static constexpr int value = max_from(1);
};

template <typename R, int L, int EPT, int S>
__device__ __forceinline__ void load_stage_tw(typename Types<R>::W (&pf)[PFCount<L, EPT>::value],
                                              const typename Types<R>::W* __restrict__ base, int t) {
  typedef FFTPlan<L, EPT> P;
  if constexpr (S >= 1 && S < P::kStages) {
    constexpr int RS = P::radix(S), NS = P::span(S), Q = EPT / RS, T = P::kT;
    if constexpr (NS > 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = t + q * T;
        const int k = is_pow2(NS) ? (j & (NS - 1)) : (int)((unsigned)j % (unsigned)NS);
        const typename Types<R>::W* tws = base + P::tw_off(S) + k;
#pragma unroll
        for (int r = 1; r < RS; ++r) pf[q * (RS - 1) + r - 1] = __ldg(&tws[(r - 1) * NS]);
      }
    }
  }
}

template <typename R, int L, int EPT, int S>
__device__ __forceinline__ void fwd_stage_pf(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                             typename Types<R>::W (&pf)[PFCount<L, EPT>::value], int t) {
  typedef typename Types<R>::C C;
  typedef FFTPlan<L, EPT> P;
  constexpr int RS = P::radix(S), NS = P::span(S), Q = EPT / RS, T = P::kT;
  constexpr bool LAST = (S == P::kStages - 1);
  constexpr int CX = P::swz(S);
  C* buf = nullptr;
  if constexpr (!LAST) buf = ex.next();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = is_pow2(NS) ? (j & (NS - 1)) : (int)((unsigned)j % (unsigned)NS);
    C a[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) a[r] = v[q + r * Q];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < RS; ++r) a[r] = twmul(a[r], pf[q * (RS - 1) + r - 1]);
    }
    butterfly<RS, false>(a);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < RS; ++r) v[q + r * Q] = a[r];
    } else {
      const int base = (j - k) * RS + k;
#pragma unroll
      for (int r = 0; r < RS; ++r) buf[sw<CX>(base + r * NS)] = a[r];
    }
  }
  if constexpr (!LAST) {
    load_stage_tw<R, L, EPT, S + 1>(pf, stage_tw<R>(ex), t);
    ex.sync();
#pragma unroll
    for (int m = 0; m < EPT; ++m) v[m] = buf[sw<CX>(t + T * m)];
  }
}

template <typename R, int L, int EPT, int... S>
__device__ __forceinline__ void fft_fwd_pf_seq(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                               int t, std::integer_sequence<int, S...>) {
  typename Types<R>::W pf[PFCount<L, EPT>::value];
  load_stage_tw<R, L, EPT, 1>(pf, stage_tw<R>(ex), t);
  (fwd_stage_pf<R, L, EPT, S>(v, ex, pf, t), ...);
}

template <typename R, int L, int EPT, int TC, int... S>
__device__ __forceinline__ void fft_fwd_seq(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                            const typename Types<R>::W* tw, int t, TcCtx* tc, bool act,
                                            std::integer_sequence<int, S...>) {
  (fwd_stage<R, L, EPT, S, TC>(v, ex, tw, t, tc, act), ...);
}
template <typename R, int L, int EPT, int TC, int... S>
__device__ __forceinline__ void fft_inv_seq(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                            const typename Types<R>::W* tw, int t, TcCtx* tc, bool act,
                                            std::integer_sequence<int, S...>) {
  (inv_stage<R, L, EPT, FFTPlan<L, EPT>::kStages - 1 - S, TC>(v, ex, tw, t, tc, act), ...);
}

// Forward DFT of length L: v holds x[t + T m] on entry, X[t + T m] on exit
// (T = L/EPT, m < EPT).  Every thread of the block must call it (block-wide
// barriers inside); the exchanges alternate between the two buffers of `ex`.
// TC: the radix-16 stages run on the tensor cores (tc_dft.cuh, context *tc):
// 1 split-FP16, 2 split-BF16.  act = false: barriers and tensor-core rounds
// only (see fwd_stage).
template <typename R, int L, int EPT, int TC = 0>
__device__ __forceinline__ void block_fft_fwd(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                              const typename Types<R>::W* tw, int t, TcCtx* tc = nullptr,
                                              bool act = true) {
  static_assert(!TC || sizeof(R) == 4, "tensor-core stages take float data");
  fft_fwd_seq<R, L, EPT, TC>(v, ex, tw, t, tc, act, std::make_integer_sequence<int, FFTPlan<L, EPT>::kStages>{});
}
// Adjoint of fwd_stage_pf's stage S: the stage's twiddles are loaded before its
// exchange barrier (they are applied after the butterfly).
template <typename R, int L, int EPT, int S>
__device__ __forceinline__ void inv_stage_pf(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                             typename Types<R>::W (&pf)[PFCount<L, EPT>::value], int t) {
  typedef typename Types<R>::C C;
  typedef FFTPlan<L, EPT> P;
  constexpr int RS = P::radix(S), NS = P::span(S), Q = EPT / RS, T = P::kT;
  constexpr bool FIRST = (S == P::kStages - 1);
  constexpr int CX = P::swz(S);
  C* buf = nullptr;
  if constexpr (!FIRST) {
    buf = ex.next();
#pragma unroll
    for (int m = 0; m < EPT; ++m) buf[sw<CX>(t + T * m)] = v[m];
  }
  load_stage_tw<R, L, EPT, S>(pf, stage_tw<R>(ex), t);
  if constexpr (!FIRST) ex.sync();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = is_pow2(NS) ? (j & (NS - 1)) : (int)((unsigned)j % (unsigned)NS);
    C a[RS];
    if constexpr (FIRST) {
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = v[q + r * Q];
    } else {
      const int base = (j - k) * RS + k;
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = buf[sw<CX>(base + r * NS)];
    }
    butterfly<RS, true>(a);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < RS; ++r) a[r] = twmul_conj(a[r], pf[q * (RS - 1) + r - 1]);
    }
#pragma unroll
    for (int r = 0; r < RS; ++r) v[q + r * Q] = a[r];
  }
}

template <typename R, int L, int EPT, int... S>
__device__ __forceinline__ void fft_inv_pf_seq(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                               int t, std::integer_sequence<int, S...>) {
  typename Types<R>::W pf[PFCount<L, EPT>::value];
  (inv_stage_pf<R, L, EPT, FFTPlan<L, EPT>::kStages - 1 - S>(v, ex, pf, t), ...);
}

// block_fft_inv with each stage's twiddles loaded before its exchange barrier.
template <typename R, int L, int EPT>
__device__ __forceinline__ void block_fft_inv_pf(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                                 int t) {
  fft_inv_pf_seq<R, L, EPT>(v, ex, t, std::make_integer_sequence<int, FFTPlan<L, EPT>::kStages>{});
}

// block_fft_fwd with next-stage twiddle prefetch (no tensor-core stages); the
// twiddle table is read through ex.twslot, which must be visible before the call.
template <typename R, int L, int EPT>
__device__ __forceinline__ void block_fft_fwd_pf(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                                 int t) {
  fft_fwd_pf_seq<R, L, EPT>(v, ex, t, std::make_integer_sequence<int, FFTPlan<L, EPT>::kStages>{});
}

// Unnormalised inverse DFT (adjoint of block_fft_fwd).
template <typename R, int L, int EPT, int TC = 0>
__device__ __forceinline__ void block_fft_inv(typename Types<R>::C (&v)[EPT], ExBuf<typename Types<R>::C>& ex,
                                              const typename Types<R>::W* tw, int t, TcCtx* tc = nullptr,
                                              bool act = true) {
  static_assert(!TC || sizeof(R) == 4, "tensor-core stages take float data");
  fft_inv_seq<R, L, EPT, TC>(v, ex, tw, t, tc, act, std::make_integer_sequence<int, FFTPlan<L, EPT>::kStages>{});
}

}  // namespace psatd
