// tables.cu -- plan-time tables, computed in FP64 on the GPU and rounded once
// to the step precision (FP32 keeps hi/lo pairs of the values that multiply
// the field state every step).
//
// Twiddles of a length-L transform with EPT elements per thread, in the order
// the FFT stages read them (fft_core.cuh): for each stage s >= 1 (radix R_s,
// span Ns), entry (r-1) Ns + k holds W_L^(r k L/(R_s Ns)); an R2C/C2R axis
// (N = 2L real points) appends W_N^k, k < L, for the even/odd split.
//
// Coefficient octant: one entry per (|mx|, |my|, |mz|), |m_i| <= n_i/2, with
// the Nyquist index of each axis taken as m_i = 0.  With the integer-mode
// vector mt = (rx mx, ry my, rz mz), k = g0 mt, x = c |k| dt (Sec. III.B: the
// analytic integration over dt with sources constant):
//   C  = cos x                          S_m = sin x / |mt|       (-> c g0 dt)
//   A1 = (1 - C) / |mt|^2              (-> (c g0 dt)^2 / 2)
//   A4 = (S/(c k) - dt) / (eps0 |mt|^2) = dt (c g0 dt)^2 f1(x) / eps0
//   B1 = (S/x - 1) / (eps0 g0 |mt|^2)   = c^2 g0 dt^2 f1(x) / eps0
//   B2 = (S/x - C) / (eps0 g0 |mt|^2)   = c^2 g0 dt^2 f2(x) / eps0
// f1 = (sin x/x - 1)/x^2, f2 = (sin x/x - cos x)/x^2 (Taylor series below 0.5),
// every entry multiplied by 1/N (the inverse-FFT normalisation).
#include <cuda_runtime.h>
#include <stdint.h>

#include "psatd_kernels.cuh"
#include "tables.h"

namespace psatd {

// Stage radices of a length-L transform with ept elements per thread, in stage
// order (the rules of FFTPlan in fft_core.cuh).
struct Radices {
  int n;
  int r[16];
};
static Radices plan_radices(int L, int ept) {
  Radices R{};
  auto lg = [](int v) { int k = 0; while ((1 << k) < v) ++k; return k; };
  if (L & (L - 1)) {  // 3 * 2^k: radix 3, (2|4), 8, ... (ept 24) or radix 12, (2), 4, ... (ept 12);
                      // 5 * 2^k: radix 5, (2), 4, ... (ept 20)
    const int f = L % 3 == 0 ? 3 : 5;
    const int head = (f == 3 && ept == 12) ? 2 : 0, b = (f == 5 || ept == 12) ? 2 : 3;
    const int k = lg(L / f) - head, rem = k % b;
    R.r[R.n++] = f << head;
    if (rem) R.r[R.n++] = 1 << rem;
    for (int i = 0; i < k / b; ++i) R.r[R.n++] = 1 << b;
  } else {
    const int k = lg(L), b = lg(ept), rem = k % b;
    R.r[R.n++] = rem ? (1 << rem) : ept;
    for (int i = 0; i < k / b - (rem ? 0 : 1); ++i) R.r[R.n++] = ept;
  }
  return R;
}

__global__ void k_twiddles(void* out, int L, Radices rad, int r2c, int f32) {
  const int nstage = L - rad.r[0];
  const int total = nstage + (r2c ? L : 0);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  double num, den;  // W = exp(-2 pi i num/den)
  if (e < nstage) {
    int off = 0, ns = rad.r[0];
    num = 0.0;
    den = (double)L;
    for (int st = 1; st < rad.n; ++st) {
      const int R = rad.r[st];
      const int size = (R - 1) * ns;
      if (e < off + size) {
        const int r = (e - off) / ns + 1, k = (e - off) % ns;
        num = (double)((long long)r * k * (L / (R * ns)));
        break;
      }
      off += size;
      ns *= R;
    }
  } else {
    num = (double)(e - nstage);
    den = 2.0 * (double)L;
  }
  double s, c;
  sincospi(-2.0 * num / den, &s, &c);
  if (f32) {
    const float ch = (float)c, sh = (float)s;
    static_cast<float4*>(out)[e] = make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
  } else {
    static_cast<double2*>(out)[e] = make_double2(c, s);
  }
}

__device__ double f1_series(double x) {  // sum_{n>=1} (-1)^n x^(2n-2) / (2n+1)!
  const double x2 = x * x;
  double t = -1.0 / 6.0, s = t;
  for (int n = 2; n <= 12; ++n) {
    t *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
    s += t;
  }
  return s;
}
__device__ double f2_series(double x) {  // sum_{n>=1} (-1)^(n+1) 2n x^(2n-2) / (2n+1)!
  const double x2 = x * x;
  double u = 1.0 / 6.0, s = 2.0 * u;
  for (int n = 2; n <= 12; ++n) {
    u *= x2 / ((2.0 * n) * (2.0 * n + 1.0));
    s += ((n & 1) ? 1.0 : -1.0) * 2.0 * n * u;
  }
  return s;
}

// Order-p staggered wavenumbers and half-cell phases of one axis of n cells of
// size d (PSATD-p, Table 1): for m = 0..n/2,
//   kp[m] = (2/d) sum_{l=1}^{p/2} C_l sin((2l-1) pi m/n) / g0   (in units of g0),
//   ph[m] = exp(-i pi m/n) (the shift of a component sitting half a cell along
//   the axis; negative m take the conjugate), rounded to the step precision
//   (FP32: hi/lo pairs).  The Nyquist entry m = n/2 is kept (k = pi/d).
__global__ void k_kp_tables(double* kp, void* ph, const double* C, int nl, int n, double d, double g0, int f32) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > n / 2) return;
  double acc = 0.0;
  for (int l = 1; l <= nl; ++l) {
    const long long num = ((long long)(2 * l - 1) * m) % (2LL * n);  // (2l-1) m/n mod 2, exactly
    acc += C[l - 1] * sinpi((double)num / (double)n);
  }
  kp[m] = 2.0 / d * acc / g0;
  double sn, cs;
  sincospi(-(double)m / (double)n, &sn, &cs);
  if (f32) {
    const float ch = (float)cs, sh = (float)sn;
    static_cast<float4*>(ph)[m] = make_float4(ch, sh, (float)(cs - (double)ch), (float)(sn - (double)sh));
  } else {
    static_cast<double2*>(ph)[m] = make_double2(cs, sn);
  }
}

__global__ void k_coefs(void* out, int f32, int e0, int e1, int e2, int nx, int ny, int nz,
                        double rx, double ry, double rz, double g0, double c, double dt,
                        double eps0, double invN, const double* kpx, const double* kpy, const double* kpz) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)e0 * e1 * e2;
  if (idx >= total) return;
  const int iz = (int)(idx % e2);
  const int iy = (int)((idx / e2) % e1);
  const int ix = (int)(idx / ((int64_t)e1 * e2));
  double mm;
  if (kpx) {  // staggered order p: |k_p| / g0 from the per-axis tables (Nyquist kept)
    const double a = kpx[ix], b = kpy[iy], z = kpz ? kpz[iz] : 0.0;
    mm = sqrt(a * a + b * b + z * z);
  } else {
    const double mx = (2 * ix == nx) ? 0.0 : ix;
    const double my = (2 * iy == ny) ? 0.0 : iy;
    const double mz = (nz > 1 && 2 * iz == nz) ? 0.0 : iz;
    mm = sqrt((rx * mx) * (rx * mx) + (ry * my) * (ry * my) + (rz * mz) * (rz * mz));
  }
  const double q = c * g0 * dt;  // x = q |mt|
  const double x = q * mm;
  double sx, cx;
  sincos(x, &sx, &cx);
  double sinc = 1.0, sinc_h = 1.0;
  if (x > 0.0) {
    sinc = sx / x;
    sinc_h = sin(0.5 * x) / (0.5 * x);
  }
  double f1, f2;
  if (x < 0.5) {
    f1 = f1_series(x);
    f2 = f2_series(x);
  } else {
    f1 = (sinc - 1.0) / (x * x);
    f2 = (sinc - cx) / (x * x);
  }
  const double C = cx * invN;
  const double Sm = q * sinc * invN;
  const double A1 = 0.5 * q * q * sinc_h * sinc_h * invN;
  const double A4 = dt * q * q * f1 / eps0 * invN;
  const double B1 = c * c * g0 * dt * dt * f1 / eps0 * invN;
  const double B2 = c * c * g0 * dt * dt * f2 / eps0 * invN;
  if (f32) {
    Coef<float> e;
    e.C_h = (float)C;
    e.C_l = (float)(C - (double)e.C_h);
    e.S_h = (float)Sm;
    e.S_l = (float)(Sm - (double)e.S_h);
    e.A1 = (float)A1;
    e.A4 = (float)A4;
    e.B1 = (float)B1;
    e.B2 = (float)B2;
    static_cast<Coef<float>*>(out)[idx] = e;
  } else {
    Coef<double> e;
    e.C_h = C;
    e.C_l = 0.0;
    e.S_h = Sm;
    e.S_l = 0.0;
    e.A1 = A1;
    e.A4 = A4;
    e.B1 = B1;
    e.B2 = B2;
    static_cast<Coef<double>*>(out)[idx] = e;
  }
}

// Split radix-16 DFT matrices for the tensor-core stages (tc_dft.cuh): for
// direction dir (0: F_rq = exp(-2 pi i rq/16), 1: its conjugate) the real
// 32 x 32 form G[n][k], n = 2r + d, k = 2q + c, as G = G_h + G_l + G_ll:
// G_h = G rounded to the 2^-8 grid (exact in FP16), G_l = FP16 of G - G_h,
// G_ll = FP16 of G - G_h - G_l (all from the FP64 value); each piece stored as
// 8-row x 16-byte core matrices (LBO 128 B, SBO 512 B).
__global__ void k_tc_dftmat(unsigned short* out, int bf16) {
  typedef TcGeom<16> G;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * 32 * 32) return;
  const int dir = e >> 10, n = (e >> 5) & 31, k = e & 31;
  const int r = n >> 1, d = n & 1, q = k >> 1, c = k & 1;
  double sn, cs;
  sincospi((dir ? 2.0 : -2.0) * (double)((r * q) & 15) / 16.0, &sn, &cs);
  const double v = d == 0 ? (c == 0 ? cs : -sn) : (c == 0 ? sn : cs);
  const int off = (n >> 3) * G::kSBO + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
  unsigned short u0, u1, u2;
  if (bf16) {  // G_h on the 2^-7 grid, G_m and G_l the BF16 remainders
    const double vh = rint(v * 128.0) / 128.0;
    const __nv_bfloat16 m = __float2bfloat16_rn((float)(v - vh));
    const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - vh - (double)__bfloat162float(m)));
    u0 = __bfloat16_as_ushort(__float2bfloat16_rn((float)vh));
    u1 = __bfloat16_as_ushort(m);
    u2 = __bfloat16_as_ushort(l);
  } else {     // G_h on the 2^-8 grid, G_l and G_ll the FP16 remainders
    const double vh = rint(v * 256.0) / 256.0;
    const __half l = __float2half_rn((float)(v - vh));
    const __half ll = __float2half_rn((float)(v - vh - (double)__half2float(l)));
    u0 = __half_as_ushort(__float2half_rn((float)vh));
    u1 = __half_as_ushort(l);
    u2 = __half_as_ushort(ll);
  }
  out[(dir * G::kGDir + off) / 2] = u0;
  out[(dir * G::kGDir + G::kGPiece + off) / 2] = u1;
  out[(dir * G::kGDir + 2 * G::kGPiece + off) / 2] = u2;
}

cudaError_t launch_tc_dftmat(void* out, bool bf16, cudaStream_t st) {
  k_tc_dftmat<<<8, 256, 0, st>>>(static_cast<unsigned short*>(out), bf16 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(void* out, int L, int ept, bool r2c, bool f32, cudaStream_t st) {
  const int total = 2 * L;
  k_twiddles<<<(total + 255) / 256, 256, 0, st>>>(out, L, plan_radices(L, ept), r2c ? 1 : 0, f32 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_coefs(void* out, bool f32, int e0, int e1, int e2, int nx, int ny, int nz,
                         double rx, double ry, double rz, double g0, double c, double dt,
                         double eps0, double invN, cudaStream_t st, const double* const kp[3]) {
  const int64_t total = (int64_t)e0 * e1 * e2;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  k_coefs<<<blocks, 256, 0, st>>>(out, f32 ? 1 : 0, e0, e1, e2, nx, ny, nz, rx, ry, rz, g0, c, dt,
                                  eps0, invN, kp ? kp[0] : nullptr, kp ? kp[1] : nullptr, kp ? kp[2] : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_kp_tables(double* kp, void* ph, const double* C, int nl, int n, double d, double g0, bool f32,
                             cudaStream_t st) {
  k_kp_tables<<<(n / 2 + 1 + 127) / 128, 128, 0, st>>>(kp, ph, C, nl, n, d, g0, f32 ? 1 : 0);
  return cudaGetLastError();
}

// Staggered first-derivative weights of order p (f'(0) ~ (1/h) sum_l C_l
// [f((l-1/2)h) - f(-(l-1/2)h)]): the ratio of consecutive weights,
// C_l / C_(l-1) = -(2l-3)^2 (h-l+1) / ((2l-1)^2 (h+l-1)), h = p/2, fixes them up
// to one factor, which the consistency condition sum_l (2l-1) C_l = 1 (exact
// derivative of a linear function) sets.
void staggered_weights(int p, double* C) {
  const int h = p / 2;
  C[0] = 1.0;
  for (int l = 2; l <= h; ++l)
    C[l - 1] = C[l - 2] * -((double)(2 * l - 3) * (2 * l - 3) * (h - l + 1)) / ((double)(2 * l - 1) * (2 * l - 1) * (h + l - 1));
  double s = 0.0;
  for (int l = 1; l <= h; ++l) s += (2 * l - 1) * C[l - 1];
  for (int l = 1; l <= h; ++l) C[l - 1] /= s;
}

cudaError_t launch_nonfinite(bool f32, void* const* out, int n_out, const int64_t* off, int npatch,
                             int64_t count, int* err, cudaStream_t st) {
  NfPtrs ptrs{};
  for (int c = 0; c < n_out && c < 6; ++c) ptrs.p[c] = out[c];
  const int64_t want = (count + 255) / 256;
  const dim3 grid((unsigned)(want < 1216 ? (want < 1 ? 1 : want) : 1216), (unsigned)n_out, (unsigned)npatch);
  if (f32) k_nonfinite<float><<<grid, 256, 0, st>>>(ptrs, off, count, err);
  else k_nonfinite<double><<<grid, 256, 0, st>>>(ptrs, off, count, err);
  return cudaGetLastError();
}

}  // namespace psatd
