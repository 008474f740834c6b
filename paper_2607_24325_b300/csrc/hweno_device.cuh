// hweno_device.cuh -- device building blocks of the unified-stencil HWENO
// operator (arxiv 2607.24325) for sm_103a: Appendix A coefficient maps,
// smoothness indicators and nonlinear weights (Steps 1-3 of Sec. 2.1 and
// 2.2), Euler physics (closed-form eigenvectors, fluxes and flux directional
// derivatives), and the ghost-cell index map used by the fused halo loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno_types.h"

#define HW_FULL_MASK 0xffffffffu

namespace hw {

// ---------------------------------------------------------------------------
// Checked build (compiled with -DHWENO_CHECKED into libhweno_checked.so): the
// shared- and global-memory indices of the stage kernels are tested against
// their buffers' extents; a bad one is counted, the first is recorded (site,
// index, extent) in this translation unit's check word, and the access is
// skipped (a load gives 0).  No trap, no assert: the context stays usable and
// the host reads the word (hweno_check_*).  In the normal build HW_IN is
// `true` and costs nothing.
// ---------------------------------------------------------------------------
#ifdef HWENO_CHECKED
static __device__ unsigned int hw_check[4];  // bad accesses, first site, its index, its extent
__device__ __forceinline__ bool hw_in(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&hw_check[0], 1u) == 0u) {
    hw_check[1] = (unsigned)site;
    hw_check[2] = (unsigned)i;
    hw_check[3] = (unsigned)n;
  }
  return false;
}
#define HW_IN(i, n, site) ::hw::hw_in((long long)(i), (long long)(n), (site))
// host side: copy (and optionally clear) this translation unit's check word
#define HW_CHECK_READER(name)                                                        \
  extern "C" int name(unsigned int* out4, int reset) {                               \
    cudaError_t e = cudaMemcpyFromSymbol(out4, ::hw::hw_check, sizeof(unsigned) * 4); \
    if (e == cudaSuccess && reset) {                                                 \
      const unsigned z[4] = {0u, 0u, 0u, 0u};                                        \
      e = cudaMemcpyToSymbol(::hw::hw_check, z, sizeof z);                           \
    }                                                                                \
    return (int)e;                                                                   \
  }
#else
#define HW_IN(i, n, site) true
#define HW_CHECK_READER(name)
#endif

// ---------------------------------------------------------------------------
// Scheme parameters in the arithmetic type T.
// ---------------------------------------------------------------------------
template <typename T>
struct WeightsT {
  T g[5];        // linear weights gamma_m
  T inv_g0;      // 1 / gamma_0
  T eps;         // epsilon of the nonlinear weights
  int pow2;      // 1: beta^2 + eps in the denominator, 0: beta + eps
  int linear;    // 1: omega = gamma (pure p0)
  int typical;   // 1: Jiang-Shu integral indicator for p0
  int screen_off;  // 1: the FP32 screens clear nothing (verification)
};

template <typename T>
__host__ __device__ inline WeightsT<T> make_weights(const WeightParams& w) {
  WeightsT<T> o;
  if constexpr (sizeof(T) == 4) {
    for (int m = 0; m < 5; ++m) o.g[m] = w.gf[m];
    o.inv_g0 = w.inv_g0f;
    o.eps = w.epsf;
  } else {
    for (int m = 0; m < 5; ++m) o.g[m] = (T)w.g[m];
    o.inv_g0 = (T)(1.0 / w.g[0]);
    o.eps = (T)w.eps;
  }
  o.pow2 = w.pow2;
  o.linear = w.linear;
  o.typical = w.typical;
  o.screen_off = w.screen_off;
  return o;
}

// Jiang-Shu indicator of a quartic in the cell's scaled coordinate,
// Eq. (smoothness-indicator-typical): sum_{l=1..4} int_{-1/2}^{1/2}
// (d^l p / dxi^l)^2 dxi as the closed quadratic form in c_1..c_4 (the odd
// monomial moments vanish).  For a linear polynomial it is c_1^2, the same
// as the moment form.
template <typename T>
__device__ __forceinline__ T beta_typical_1d(T c1, T c2, T c3, T c4) {
  return c1 * (c1 + T(0.5) * c3) + c2 * (T(13.0 / 3.0) * c2 + T(4.2) * c4) + T(3129.0 / 80.0) * c3 * c3 +
         T(87617.0 / 140.0) * c4 * c4;
}

// |x| by clearing the sign bit (a free operand modifier of the consuming
// add; a compare-and-negate would issue on the FP64 pipe in FP64).
__device__ __forceinline__ double fabs_t(double x) { return fabs(x); }
__device__ __forceinline__ float fabs_t(float x) { return fabsf(x); }

// Reciprocal and quotient.  FP64: the reciprocal by Newton-Raphson from an
// FP32 seed (rcp64 below, faithful), the quotient IEEE.  FP32: the fast
// approximate forms (a few ulp), far below the FP32 stencil's own
// conditioning -- the hardware approximate reciprocal (PTX
// rcp.approx.ftz.f32, about 1 ulp) and a quotient as a times it.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The value itself, hidden from the optimiser: an expression that produced
// it is rounded to a register value and never fused into its readers
// (so every reader, in any code context, sees the same bits).
__device__ __forceinline__ float opaque(float x) {
  asm("" : "+f"(x));
  return x;
}
__device__ __forceinline__ double opaque(double x) {
  asm("" : "+d"(x));
  return x;
}

// Square root to within a few units of 2^-23 relative (PTX sqrt.approx,
// subnormal inputs kept): for bounds that carry their own margin.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double div_t(double a, double b) { return a / b; }
__device__ __forceinline__ float div_t(float a, float b) { return a * rcp_approx(b); }
// Square root in the argument's own precision (an unqualified sqrt of a
// float would promote to the FP64 pipe).
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }

// Exact FP32 -> FP64 widening on the integer ALU, from the IEEE 754
// binary32 / binary64 encodings: the exponent is re-biased by 1023 - 127 =
// 896 and the 23 fraction bits move to the top of the 52-bit fraction.
// Zero keeps its sign; subnormals, infinities and NaN (exponent field 0 with
// a nonzero fraction, or 255) take the hardware conversion.
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned mag = u & 0x7fffffffu;
  if ((mag >> 23) - 1u >= 254u) {
    if (mag == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)x;
  }
  const unsigned hi = (u & 0x80000000u) | ((mag >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}

// FP64 -> FP32 with round-to-nearest-even on the integer ALU: the 29 dropped
// fraction bits decide the rounding, a carry out of the fraction moves into
// the exponent.  Values whose binary32 image is not a normal number
// (exponent field outside 897..1150) take the hardware conversion.
__device__ __forceinline__ float narrow_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u > 253u) return (float)x;
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned bits = (hi & 0x80000000u) | ((e - 896u) << 23) | frac;
  bits += (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;
  return __uint_as_float(bits);
}

// As narrow_f64, but magnitudes below the smallest normal FP32 number
// become zero (no FP64-pipe fallback for them).
__device__ __forceinline__ float narrow_f64_ftz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  if (((hi >> 20) & 0x7ffu) < 897u) return __uint_as_float(hi & 0x80000000u);
  return narrow_f64(x);
}

// 1/s for a positive normal double: an FP32 seed (the approximate reciprocal
// of s's significand, exponent handled on the integer ALU) and one Newton
// step y <- y + y (1 - s y) in FP64, relative error about 2^-46 -- two FP64
// operations instead of an IEEE division.  Exponents near the ends of the
// range take the division.
__device__ __forceinline__ double rcp_newton(double s) {
  const unsigned hi = (unsigned)__double2hiint(s), lo = (unsigned)__double2loint(s);
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e < 2 || e > 2044) return 1.0 / s;
  const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));  // in [1, 2)
  const double y0 = widen_f32(rcp_approx(m));                                         // in (0.5, 1]
  const unsigned yh = (unsigned)__double2hiint(y0) - ((unsigned)(e - 1023) << 20);
  const double y = __hiloint2double((int)yh, __double2loint(y0));
  return fma(y, fma(-s, y, 1.0), y);
}

// 1/s in FP64, faithful (within one unit in the last place) wherever s and
// 1/s are normal numbers: Newton-Raphson for the reciprocal,
// y <- y + y (1 - s y) with the residual formed by one fused multiply-add
// (Markstein), twice from the hardware's approximate FP64 reciprocal (PTX
// rcp.approx.ftz.f64, about the leading 20 bits); each step squares the
// relative error, so the second leaves only the rounding of its last
// operation.  Four FP64 operations, no branch.  Zeros, infinities and NaN
// keep the approximation's IEEE results (+-inf, +-0, NaN); subnormal
// arguments and results are flushed (1/s = +-inf, 0), as the approximation
// does.
__device__ __forceinline__ double rcp64(double s) {
  double y0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(s));
  const unsigned e = ((unsigned)__double2hiint(s) >> 20) & 0x7ffu;
  double y = fma(y0, fma(-s, y0, 1.0), y0);
  y = fma(y, fma(-s, y, 1.0), y);
  return e - 1u < 2045u ? y : y0;
}
__device__ __forceinline__ double rcp_t(double x) { return rcp64(x); }
__device__ __forceinline__ float rcp_t(float x) { return rcp_approx(x); }

// Input conversion of the coefficient maps: identity, or the exact widening.
template <typename TC, typename TQ>
__device__ __forceinline__ TC to_tc(TQ x) {
  if constexpr (sizeof(TC) == 8 && sizeof(TQ) == 4) return widen_f32(x);
  else return (TC)x;
}

// Nonlinear weights of Eq. (nonlinear-weights) / (nonlinear-weights-2D) for
// one target polynomial and NL linear ones: given beta_0..beta_NL and tau,
// returns r = omega_0 / gamma_0 and omega_1..omega_NL (om[0] unused).
// w~_m = gamma_m (1 + tau^2/d_m), d_m = beta_m^{1|2} + eps, omega = w~ / sum w~.
// FP64 scales every w~_m by P = prod_k d_k: with Q_m = prod_{k!=m} d_k
// (prefix times suffix products), w~_m P = gamma_m f_m, f_m = P + tau^2 Q_m
// (one fused multiply-add, nl_numerators), so the weights need one
// reciprocal instead of NL+2 (FP64 division is costly on B300) and
// r = f_0 / sum_m gamma_m f_m; FP32 keeps the quotients (products of d could
// overflow its range).
template <typename T, int NL>
__device__ __forceinline__ void nl_numerators(const T* beta, T tau, const WeightsT<T>& w, T* f) {
  const T t2 = tau * tau;
  T d[NL + 1];
#pragma unroll
  for (int m = 0; m <= NL; ++m) d[m] = (w.pow2 ? beta[m] * beta[m] : beta[m]) + w.eps;
  T pre[NL + 1], suf[NL + 1];
  pre[1] = d[0];
#pragma unroll
  for (int m = 2; m <= NL; ++m) pre[m] = pre[m - 1] * d[m - 1];
  suf[NL - 1] = d[NL];
#pragma unroll
  for (int m = NL - 2; m >= 0; --m) suf[m] = suf[m + 1] * d[m + 1];
  const T P = d[0] * suf[0];
#pragma unroll
  for (int m = 0; m <= NL; ++m) {
    const T q = m == 0 ? suf[0] : (m == NL ? pre[NL] : pre[m] * suf[m]);
    f[m] = fma(t2, q, P);
  }
}

template <typename T, int NL>
__device__ __forceinline__ void nl_weights(const T* beta, T tau, const WeightsT<T>& w, T& r, T* om) {
  if constexpr (sizeof(T) == 8) {
    T f[NL + 1];
    nl_numerators<T, NL>(beta, tau, w, f);
    T s = w.g[0] * f[0];
#pragma unroll
    for (int m = 1; m <= NL; ++m) s = fma(w.g[m], f[m], s);
    const T inv = rcp_t(s);
    r = f[0] * inv;
#pragma unroll
    for (int m = 1; m <= NL; ++m) om[m] = (w.g[m] * f[m]) * inv;
  } else {
    const T t2 = tau * tau;
    T e[NL + 1];
#pragma unroll
    for (int m = 0; m <= NL; ++m) e[m] = w.g[m] * (T(1) + div_t(t2, (w.pow2 ? beta[m] * beta[m] : beta[m]) + w.eps));
    T s = e[0];
#pragma unroll
    for (int m = 1; m <= NL; ++m) s += e[m];
    const T inv = rcp_t(s);
    r = e[0] * inv * w.inv_g0;
#pragma unroll
    for (int m = 1; m <= NL; ++m) om[m] = e[m] * inv;
  }
}

// ---------------------------------------------------------------------------
// 1D reconstruction of one scalar field (Sec. 2.1 Steps 1-3).
// Inputs u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1} (the target cell's own
// derivative is never used).  Outputs u_i(x_{i-1/2}), u_i(x_{i+1/2}),
// u_i'(x_{i-1/2}), u_i'(x_{i+1/2}) and v-hat = (u_i(x_{i+1/2}) - u_i(x_{i-1/2}))/dx.
// ---------------------------------------------------------------------------
template <typename T>
struct Rec1 { T uL, uR, dL, dR, vh; };

// Mixed precision, 1D, the FP32 screen: true where every a_m = tau^2 /
// (beta_m^p + eps) of Step 3 is provably at most 2^-24.  The argument of the
// 2D screen on the 1D maps: the coefficients from centre-shifted FP32
// differences (dm = u_{i-1} - u_i, dp = u_{i+1} - u_i, a = dx v_{i-1},
// b = dx v_{i+1}; every map constant exact in binary) err by a few u S at
// most (S the largest of |dm|, |dp|, |a|, |b|, u = 2^-24), bounded here by
// E = 2^-16 S; beta_0 = sum_l w_l c_l^2 (w = 1, 4, 36, 576, sum 617) then errs
// by at most 2^-18 beta~_0 + E (2 sum_l w_l |c~_l| + 617 E), and
// 2 sum_l w_l |c~_l| <= 2 sqrt(617 beta~_0) <= 50 sqrt(beta~_0) (Cauchy-Schwarz);
// beta_1 = dm^2 and beta_2 = dp^2 err by 2^-20 of themselves.  tau is at
// most tau~ (1 + 2^-20) + D_0 + (D_1 + D_2)/2, every beta_m at least its
// value less its bound, and ut^2 < 2^-25 dlo leaves room for the screen's
// own rounding below 2^-24.  The Jiang-Shu form always takes the FP64 path.
__device__ __forceinline__ bool screen1(float um, float u0, float up, float a, float b, const WeightsT<float>& wf) {
  // the verification build (libhweno_noscreen.so) sets screen_off on the host:
  // every lane then takes the FP64 indicator
  if (wf.typical || wf.screen_off) return false;
  const float dm = um - u0, dp = up - u0;
  const float S = fmaxf(fmaxf(fabsf(dm), fabsf(dp)), fmaxf(fabsf(a), fabsf(b)));
  const float E = S * 0x1p-16f;
  const float sd = dm + dp, df = dp - dm, ab = a + b, ba = b - a;
  const float c1 = 0.8125f * df - 0.3125f * ab;
  const float c2 = 1.25f * sd - 0.375f * ba;
  const float c3 = 0.25f * (ab - df);
  const float c4 = 0.25f * ba - 0.5f * sd;
  const float b0 = c1 * c1 + 4.0f * (c2 * c2) + 36.0f * (c3 * c3) + 576.0f * (c4 * c4);
  const float b1 = dm * dm, b2 = dp * dp;
  const float D0 = 0x1p-18f * b0 + E * (50.0f * sqrt_approx(b0) + 617.0f * E);
  const float D1 = 0x1p-20f * b1, D2 = 0x1p-20f * b2;
  const float tau = 0.5f * (fabsf(b0 - b1) + fabsf(b0 - b2));
  const float ut = tau * (1.0f + 0x1p-20f) + D0 + 0.5f * (D1 + D2);
  const float L = fmaxf(fminf(fminf(b0 - D0, b1 - D1), b2 - D2), 0.0f);
  const float dlo = (wf.pow2 ? L * L : L) + wf.eps;
  return ut * ut < 0x1p-25f * dlo;
}

template <typename T, bool W64 = false>
__device__ __forceinline__ Rec1<T> recon1(T um, T u0, T up, T vm, T vp, T dx, T idx,
                                          const WeightsT<T>& w, const WeightsT<double>* w64 = nullptr) {
  const T a = dx * vm, b = dx * vp;
  const T s = um + up, dd = up - um, ab = a + b, ba = b - a;
  // Appendix A: p0 = sum_l c_l xi^l, xi = (x - x_i)/dx
  const T c0 = T(287.0 / 240.0) * u0 - T(47.0 / 480.0) * s + T(9.0 / 320.0) * ba;
  const T c1 = T(13.0 / 16.0) * dd - T(5.0 / 16.0) * ab;
  const T c2 = T(5.0 / 4.0) * s - T(5.0 / 2.0) * u0 - T(3.0 / 8.0) * ba;
  const T c3 = T(0.25) * (ab - dd);
  const T c4 = u0 - T(0.5) * s + T(0.25) * ba;
  // p1 = u_i + d1 xi, p2 = u_i + d2 xi
  const T d1 = u0 - um, d2 = up - u0;
  T r, w1, w2;  // r = omega_0 / gamma_0
  if (w.linear) {
    r = T(1); w1 = w.g[1]; w2 = w.g[2];
  } else if constexpr (W64) {
    // mixed precision (the same rule as in 2D): a_m = tau^2 / (beta_m^p + eps)
    // from FP64 indicators, rounded to FP32, wherever the FP32 screen cannot
    // show that every a_m is at most 2^-24 for the whole warp (then 1 + a_m
    // rounds to 1 in FP32 and a_m = 0 gives the same weights bit for bit);
    // the weights w~_m = gamma_m (1 + a_m) and their normalisation in FP32.
    float am[3] = {0.0f, 0.0f, 0.0f};
    if (!__all_sync(HW_FULL_MASK, screen1(um, u0, up, a, b, w))) {
      const double Um = to_tc<double>(um), U0 = to_tc<double>(u0), Up = to_tc<double>(up), Dx = to_tc<double>(dx);
      const double A = Dx * to_tc<double>(vm), Bv = Dx * to_tc<double>(vp);  // exact products
      const double S = Um + Up, D = Up - Um, AB = A + Bv, BA = Bv - A;
      const double e1 = 13.0 / 16.0 * D - 5.0 / 16.0 * AB;
      const double e2 = 5.0 / 4.0 * S - 5.0 / 2.0 * U0 - 3.0 / 8.0 * BA;
      const double e3 = 0.25 * (AB - D);
      const double e4 = U0 - 0.5 * S + 0.25 * BA;
      const double f1 = U0 - Um, f2 = Up - U0;
      const double beta[3] = {w.typical ? beta_typical_1d(e1, e2, e3, e4)
                                        : e1 * e1 + 4.0 * e2 * e2 + 36.0 * e3 * e3 + 576.0 * e4 * e4,
                              f1 * f1, f2 * f2};
      const double tau = 0.5 * (fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]));
      const double t2 = tau * tau;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double d = (w64->pow2 ? beta[m] * beta[m] : beta[m]) + w64->eps;
        am[m] = narrow_f64_ftz(t2 * rcp_newton(d));
      }
    }
    const float e0 = opaque(w.g[0] * (1.0f + am[0])), ew1 = opaque(w.g[1] * (1.0f + am[1]));
    const float ew2 = opaque(w.g[2] * (1.0f + am[2]));
    const float inv = rcp_approx((e0 + ew1) + ew2);
    r = opaque((1.0f + am[0]) * inv);
    w1 = opaque(ew1 * inv);
    w2 = opaque(ew2 * inv);
  } else {
    // Step 2: beta = sum_l (l! c_l)^2
    T beta[3];
    beta[0] = w.typical ? beta_typical_1d(c1, c2, c3, c4)
                        : c1 * c1 + T(4) * c2 * c2 + T(36) * c3 * c3 + T(576) * c4 * c4;
    beta[1] = d1 * d1;
    beta[2] = d2 * d2;
    // Step 3
    const T tau = T(0.5) * (fabs_t(beta[0] - beta[1]) + fabs_t(beta[0] - beta[2]));
    T om[3];
    nl_weights<T, 2>(beta, tau, w, r, om);
    w1 = om[1]; w2 = om[2];
  }
  // Eq. (hweno-reconstruction-1D): u_i = r (p0 - g1 p1 - g2 p2) + w1 p1 + w2 p2
  const T k0 = r * (c0 - (w.g[1] + w.g[2]) * u0) + (w1 + w2) * u0;
  const T k1 = r * (c1 - w.g[1] * d1 - w.g[2] * d2) + w1 * d1 + w2 * d2;
  const T k2 = r * c2, k3 = r * c3, k4 = r * c4;
  const T ev = k0 + T(0.25) * k2 + T(0.0625) * k4;
  const T od = T(0.5) * k1 + T(0.125) * k3;
  const T evd = k1 + T(0.75) * k3;
  const T odd = k2 + T(0.5) * k4;
  Rec1<T> o;
  o.uR = ev + od;
  o.uL = ev - od;
  o.dR = (evd + odd) * idx;
  o.dL = (evd - odd) * idx;
  o.vh = T(2) * od * idx;
  return o;
}

// ---------------------------------------------------------------------------
// Euler physics (Examples 2, 4-9; gamma-law gas).
// ---------------------------------------------------------------------------
template <typename T>
struct Eig {
  T u, v, c, H, q2h, hb1, hic;  // q2h = (u^2+v^2)/2, hb1 = (g-1)/(2c^2), hic = 1/(2c)
  T qH;                         // q2h - H
};

template <typename T>
__device__ __forceinline__ Eig<T> eig1(T r, T m, T E, T g) {
  Eig<T> e;
  const T ir = rcp_t(r);
  e.u = m * ir;
  e.v = T(0);
  e.q2h = T(0.5) * e.u * e.u;
  const T p = (g - T(1)) * (E - m * e.u * T(0.5));
  const T c2 = g * p * ir;
  e.c = sqrt_t(c2);
  const T ic = rcp_t(e.c);
  e.hic = T(0.5) * ic;
  e.H = (E + p) * ir;
  e.hb1 = (T(0.5) * (g - T(1))) * ic * ic;
  e.qH = e.q2h - e.H;
  return e;
}

template <typename T>
__device__ __forceinline__ Eig<T> eig2(T r, T mx, T my, T E, T g) {
  Eig<T> e;
  const T ir = rcp_t(r);
  e.u = mx * ir;
  e.v = my * ir;
  e.q2h = T(0.5) * (e.u * e.u + e.v * e.v);
  const T p = (g - T(1)) * (E - r * e.q2h);
  const T c2 = g * p * ir;
  e.c = sqrt_t(c2);
  const T ic = rcp_t(e.c);
  e.hic = T(0.5) * ic;
  e.H = (E + p) * ir;
  e.hb1 = (T(0.5) * (g - T(1))) * ic * ic;
  e.qH = e.q2h - e.H;
  return e;
}

// 1D: left eigenvectors applied to x (characteristic variables w = L x).
template <typename T>
__device__ __forceinline__ void l1_apply(const Eig<T>& e, const T* x, T* w) {
  // sh, th: half the usual s, t (the halves of L's first and last rows
  // folded into the per-cell scales; exact, powers of two)
  const T sh = e.hb1 * (e.q2h * x[0] - e.u * x[1] + x[2]);
  const T th = (e.u * x[0] - x[1]) * e.hic;
  w[0] = sh + th;
  w[1] = x[0] - T(2) * sh;
  w[2] = sh - th;
}
// 1D: right eigenvectors, y = R w.
template <typename T>
__device__ __forceinline__ void r1_apply(const Eig<T>& e, const T* w, T* y) {
  const T sum = w[0] + w[1] + w[2];
  const T dif = w[2] - w[0];
  y[0] = sum;
  y[1] = e.u * sum + e.c * dif;
  y[2] = e.H * sum + e.qH * w[1] + e.u * e.c * dif;  // H (w0 + w2) + q2h w1
}

// 2D, direction D (0: x, 1: y): w = L_D x.  With s = E + q2h rho - u m_x -
// v m_y (three fused multiply-adds) and t = u_n rho - m_n:
// w = (hb1 s + hic t, rho - 2 hb1 s, m_t - u_t rho, hb1 s - hic t).
template <int D, typename T>
__device__ __forceinline__ void l2_apply(const Eig<T>& e, const T* x, T* w) {
  const T sh = e.hb1 * (x[3] + e.q2h * x[0] - e.u * x[1] - e.v * x[2]);  // half of s
  const T un = D == 0 ? e.u : e.v;
  const T t = un * x[0] - x[1 + D];
  w[0] = sh + e.hic * t;
  w[1] = x[0] - T(2) * sh;
  w[2] = D == 0 ? x[2] - e.v * x[0] : x[1] - e.u * x[0];
  w[3] = sh - e.hic * t;
}
// 2D, direction D: y = R_D w.
template <int D, typename T>
__device__ __forceinline__ void r2_apply(const Eig<T>& e, const T* w, T* y) {
  const T sum = w[0] + w[1] + w[3];
  const T dif = w[3] - w[0];
  const T un = D == 0 ? e.u : e.v;
  const T ut = D == 0 ? e.v : e.u;   // tangential velocity
  y[0] = sum;
  if (D == 0) {
    y[1] = e.u * sum + e.c * dif;
    y[2] = e.v * sum + w[2];
  } else {
    y[1] = e.u * sum + w[2];
    y[2] = e.v * sum + e.c * dif;
  }
  // H (w0 + w3) + q2h w1 = H sum + (q2h - H) w1
  y[3] = e.H * sum + e.qH * w[1] + ut * w[2] + un * e.c * dif;
}

// Flux f(U) and its directional derivative f'(U) V, 1D Euler.  With
// u = m / rho, H = (E + p) / rho and t = V_m - u V_rho (so that rho du = t):
//   f'(U) V = (V_m,  u (V_m + t) + dp,  H t + u (V_E + dp)),
//   dp = (g - 1) (V_E - u V_m + u^2/2 V_rho);
// no division by rho beyond the one reciprocal.
template <typename T>
__device__ __forceinline__ void euler1_flux(const T* U, const T* V, T g, T* F, T* H) {
  const T ir = rcp_t(U[0]);
  const T u = U[1] * ir;
  const T gm = g - T(1);
  const T ek = T(0.5) * (u * u);
  const T p = gm * (U[2] - U[0] * ek);
  const T Ep = U[2] + p;
  F[0] = U[1];
  F[1] = U[1] * u + p;
  F[2] = u * Ep;
  const T h = Ep * ir;
  const T t = V[1] - u * V[0];
  const T dp = gm * (V[2] - u * V[1] + ek * V[0]);
  H[0] = V[1];
  H[1] = u * (V[1] + t) + dp;
  H[2] = h * t + u * (V[2] + dp);
}

// 2D Euler, direction D: flux and directional derivatives along V and W.
// With u_n the normal velocity, H = (E + p) / rho and t = V_{m_n} - u_n V_rho
// (rho d(u_n) = t, rho d(u_t) = V_{m_t} - u_t V_rho):
//   d(m_n u_n + p) = u_n (V_{m_n} + t) + dp,  d(m_n u_t) = u_t t + u_n V_{m_t},
//   d(u_n (E + p)) = H t + u_n (V_E + dp),
//   dp = (g - 1) (V_E - u V_{m_x} - v V_{m_y} + |u|^2/2 V_rho).
template <int D, typename T>
__device__ __forceinline__ void euler2_flux(const T* U, const T* V, const T* Wv, T g, T* F, T* HV,
                                            T* HW) {
  const T ir = rcp_t(U[0]);
  const T u = U[1] * ir, v = U[2] * ir;
  const T gm = g - T(1);
  const T ek = T(0.5) * (u * u + v * v);
  const T p = gm * (U[3] - U[0] * ek);
  const T Ep = U[3] + p;
  const T un = D == 0 ? u : v;
  const T ut = D == 0 ? v : u;
  const T mn = U[1 + D];
  F[0] = mn;
  F[1] = D == 0 ? mn * u + p : mn * u;
  F[2] = D == 1 ? mn * v + p : mn * v;
  F[3] = un * Ep;
  const T h = Ep * ir;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* X = s == 0 ? V : Wv;
    T* Hh = s == 0 ? HV : HW;
    const T dmn = X[1 + D], dmt = X[2 - D];
    const T t = dmn - un * X[0];
    const T dp = gm * (X[3] - u * X[1] - v * X[2] + ek * X[0]);
    const T hn = un * (dmn + t) + dp;  // normal momentum flux
    const T ht = ut * t + un * dmt;    // tangential momentum flux
    Hh[0] = dmn;
    Hh[1 + D] = hn;
    Hh[2 - D] = ht;
    Hh[3] = h * t + un * (X[3] + dp);
  }
}

// Spectral radius |u_n| + c (Euler) at a cell average, in the state's own
// precision (it only sets alpha and dt); NaN if non-physical.
template <typename T>
__device__ __forceinline__ double euler_radius(T r, T mn, T ekin2, T E, T g) {
  // ekin2 = |m|^2 (sum of squared momenta)
  const T p = (g - T(1)) * (E - T(0.5) * ekin2 / r);
  if (!(r > T(0)) || !(p > T(0))) return __longlong_as_double(0x7ff8000000000000LL);
  return (double)(fabs_t(mn / r) + sqrt_t(g * p / r));
}

// Asynchronous 4- or 8-byte global -> shared copy (cp.async, no register
// staging): a whole halo box can be in flight at once.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
// Waits until every cp.async this thread issued has landed.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// Running max of non-negative doubles through their bit patterns (exact,
// order independent); NaN bit patterns exceed every finite one.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(HW_FULL_MASK, v, o);
    // NaN wins: compare bit patterns of non-negative values
    v = (unsigned long long)__double_as_longlong(t) > (unsigned long long)__double_as_longlong(v) ? t : v;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Ghost cells (2 deep) for the fused halo loads.  The map reproduces the
// definition "x sides filled for interior rows, then y sides for all
// columns": a cell out of range in x and/or y is resolved axis by axis.
// ---------------------------------------------------------------------------
struct GhostMap {
  int src;      // source index along the axis (valid if !fixed)
  int flip;     // mirror across this axis
  int fixed;    // inflow: fixed state
  int side;     // 0 low, 1 high (for fixed states)
};

__device__ __forceinline__ GhostMap ghost_map(int c, int n, int bc_lo, int bc_hi) {
  GhostMap g{c, 0, 0, 0};
  if (c >= 0 && c < n) return g;
  const int side = c >= n;
  const int bc = side ? bc_hi : bc_lo;
  const int r = side ? c - n : -1 - c;  // ghost depth 0 or 1
  g.side = side;
  if (bc == HWENO_BC_PERIODIC) g.src = side ? r : n - 1 - r;
  else if (bc == HWENO_BC_OUTFLOW) g.src = side ? n - 1 : 0;
  else if (bc == HWENO_BC_REFLECT) { g.src = side ? n - 1 - r : r; g.flip = 1; }
  else { g.fixed = 1; g.src = side ? n - 1 : 0; }
  return g;
}

// Sign of field (d = 0 average, 1 x-moment, 2 y-moment; component k) under a
// mirror across a face normal to `axis` (the normal momentum and the
// moment along the normal change sign).
__device__ __forceinline__ bool mirror_negates(int eq, int d, int k, int axis) {
  const bool normal_mom = eq == HWENO_EQ_EULER && k == 1 + axis;
  const bool normal_der = d == 1 + axis;
  return normal_mom != normal_der;
}

}  // namespace hw
