// Real part of the Faddeeva function, Re w(x + i y) for y >= 0, in FP32.
//
// The Voigt profile of Sec. 6.1.1 is V = Re w(z) / (sigma sqrt(2 pi)) with
// z = (nu + i gamma) / (sigma sqrt 2) (Eqs. 4-11).  The paper's code uses a
// tabulated Pierluissi approximation; this library evaluates w directly with
// three regimes chosen so that Re w keeps a relative (not only absolute)
// error bound, also close to the real axis where Re w << |w|:
//
//  * |z| >= 24  one-pole truncation of the Laplace continued fraction
//               w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))),
//               w ~ (i/sqrt(pi)) z / (z^2 - 1/2), whose real part is written
//               without cancellation as
//               Re w = (y/sqrt(pi)) (u + 1) / (u^2 + 2 y^2),  u = x^2 + y^2 - 1/2;
//               relative error <= 2.52/|z|^4 <= 7.6e-6.
//  * 5 <= |z| < 24  the same continued fraction to depth 4 (|z| >= 8) or 6,
//               evaluated in complex FP32; Re w = Im t / (sqrt(pi) |t|^2)
//               where t is the fraction's denominator.  All imaginary parts
//               stay positive, so Re w keeps its relative accuracy for small
//               y.  Near the real axis the exponentially small term
//               exp(y^2 - x^2) cos(2xy) that the asymptotic fraction misses is
//               added back (y < 1).  Relative error <= 1e-6.
//  * |z| < 5    Taylor expansion about the nearest node z0 of a 41 x 41 grid
//               (spacing 1/8) on 0 <= x, y <= 5, with coefficients
//               c_n = w^(n)(z0)/n! from the recurrence of the derivatives
//               w' = -2 z w + 2i/sqrt(pi), w^(n+1) = -2 z w^(n) - 2n w^(n-1).
//               The node values are built once in FP64 (see faddeeva.cu); on
//               the real axis their real part is exactly exp(-x0^2).  Eight
//               terms, |z - z0| <= 0.09: relative error <= 3e-7.
// Re w is even in x; all branches use |x|.
#pragma once

#include "bart_internal.cuh"

namespace bartw {

constexpr float INV_SQRTPI = 0.56418958354775628695f;

__device__ __forceinline__ float rcp_approx(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// One-pole form, used where x^2 + y^2 >= 576.  Returns Re w * sqrt(pi) / y,
// i.e. (u + 1) / (u^2 + 2 y^2), so callers can fold constants.
__device__ __forceinline__ float onepole_ratio(float x, float qm, float q2) {
  float p = x * x;
  float u = p + qm;            // qm = y^2 - 1/2
  return (u + 1.0f) * rcp_approx(fmaf(u, u, q2));   // q2 = 2 y^2
}

__device__ __forceinline__ float onepole_re(float x, float y) {
  float q = y * y;
  return INV_SQRTPI * y * onepole_ratio(x, q - 0.5f, 2.0f * q);
}

// Continued fraction to `depth`, real part of w.
__device__ __forceinline__ float cf_re(float x, float y, int depth) {
  float tr = x, ti = y;
  for (int k = depth; k >= 1; --k) {
    float a = 0.5f * (float)k;
    float inv = rcp_approx(fmaf(tr, tr, ti * ti));
    float qr = a * tr * inv, qi = -a * ti * inv;
    tr = x - qr;
    ti = y - qi;
  }
  return INV_SQRTPI * ti * rcp_approx(fmaf(tr, tr, ti * ti));
}

// The continued fraction to depth 2, w = (i/sqrt(pi)) (z^2 - 1) / (z (z^2 - 3/2)),
// in closed real form.  With u = x^2 - y^2 and v = 2xy,
//   Re w = y (x^2 + v^2 + (u - 1)(u - 3/2)) / (sqrt(pi) (x^2 + y^2) ((u - 3/2)^2 + v^2)),
// where every term of the numerator carries the factor y (no cancellation near
// the real axis; (u - 1)(u - 3/2) > -1/16 is negligible against x^2 for
// |z| >= 14).  Relative error of Re w against the Faddeeva function (FP64):
// <= 7.3e-7 for 14 <= |z| < 24 (the truncation is ~5.25 / x^6 near the real
// axis), plus the FP32 rounding of about ten operations.  The Gaussian term
// exp(-x^2) is below the FP32 range there.
__device__ __forceinline__ float cf2_re(float x, float y) {
  const float x2 = x * x, y2 = y * y;
  const float u = x2 - y2;
  const float v2 = 4.0f * x2 * y2;
  const float um = u - 1.5f;
  const float num = y * (x2 + v2 + (u - 1.0f) * um);
  const float den = (x2 + y2) * fmaf(um, um, v2);
  return INV_SQRTPI * num * rcp_approx(den);
}

// Continued fraction plus the exponentially small Gaussian term
// exp(y^2 - x^2) cos(2xy) that the asymptotic fraction misses near the real
// axis (y < 1), branch free.  Relative error of Re w for |z| >= 8: <= 1e-6 at
// depth 3; for |z| >= 5: <= 5e-7 at depth 6.
__device__ __forceinline__ float cf_gauss_re(float x, float y, int depth) {
  const float v = cf_re(x, y, depth);
  const float g = fmaf(y, y, -x * x);
  const float gt = __expf(g) * __cosf(2.0f * x * y);
  return v + ((y < 1.0f && g > -87.0f) ? gt : 0.0f);
}

// Taylor expansion about the nearest table node (x >= 0, x^2 + y^2 < 25).
// UNROLL bounds the coefficient loads in flight (register pressure).
template <int UNROLL = wtab::NT - 1>
__device__ __forceinline__ float taylor_re(float x, float y, const float2* __restrict__ tab) {
  int ix = max(min((int)(x * (1.0f / wtab::H) + 0.5f), wtab::NX - 1), 0);
  int iy = max(min((int)(y * (1.0f / wtab::H) + 0.5f), wtab::NY - 1), 0);
  float a = x - (float)ix * wtab::H;
  float b = y - (float)iy * wtab::H;
  const float2* c = tab + ((size_t)iy * wtab::NX + ix) * wtab::NT;
  float2 t = __ldg(c + wtab::NT - 1);
  float ar = t.x, ai = t.y;
#pragma unroll UNROLL
  for (int n = wtab::NT - 2; n >= 0; --n) {
    float2 cn = __ldg(c + n);
    float r = fmaf(ar, a, fmaf(-ai, b, cn.x));
    float i = fmaf(ar, b, fmaf(ai, a, cn.y));
    ar = r;
    ai = i;
  }
  return ar;
}

// Re w(x + i y) for 0 <= y <= 0.02 and any x >= 0, from the expansion in y
// about the real axis (w is analytic, so d/dy = i d/dz):
//   Re w = e^{-x^2} (1 + y^2 (1 - 2 x^2)) + y G(x)
//          + (y^3 / 6) (4 / sqrt(pi) + G(x) (6 - 4 x^2)) + O(y^4),
// G(x) = -Im w'(x) = (2 / sqrt(pi)) (2 x F(x) - 1), F Dawson's integral.
// For x < 5, e^{-x^2} = Re w(x) and w'(x) come from the Taylor table's
// real-axis row (Horner in the real offset from the nearest node, no
// cancellation: the row holds the derivative coefficients themselves); for
// x >= 5, G from its asymptotic series
//   G = (2 / sqrt(pi)) sum_{k=1}^{10} (2k-1)!! / (2 x^2)^k
// (truncation <= 2.7e-7 relative at x = 5), e^{-x^2} with a compensated
// exponent.  The bracket of the y^3 term, 4 / sqrt(pi) + G (6 - 4 x^2), is
// O(x^-4) while its two parts are O(1): in FP32 it cancels with an absolute
// error ~ x^2 eps, which far in a line's wings would exceed the term itself.
// So the y^3 term is taken only below x = 40 (cancellation error there below
// 3e-8 of Re w); beyond, the whole term is below y^2 / x^2 <= 2.5e-7 of Re w
// and is left out.  One branch-free form for the core and the wings of a line with
// small y.  Relative error of Re w (FP32 against the FP64 Faddeeva function)
// <= 2.3e-6 for x >= 0, 1e-10 <= y <= 0.02.
constexpr float SMALL_Y = 0.02f;
__device__ __forceinline__ float small_y_re(float x, float y, const float2* __restrict__ tab) {
  constexpr float L2E = 1.4426950408889634f;
  constexpr float L2E_LO = (float)(1.4426950408889634 - (double)L2E);
  constexpr float LN2 = 0.6931471805599453f;
  constexpr float TWO_SQRTPI = 1.1283791670955126f;   // 2 / sqrt(pi)
  float e, g;
  if (x < 5.0f) {
    const int ix = min((int)(x * (1.0f / wtab::H) + 0.5f), wtab::NX - 1);
    const float a = x - (float)ix * wtab::H;
    const float2* c = tab + (size_t)ix * wtab::NT;   // nodes on the real axis (iy = 0)
    float2 cn = __ldg(c + wtab::NT - 1);
    float r = cn.x, d = (float)(wtab::NT - 1) * cn.y;
#pragma unroll
    for (int n = wtab::NT - 2; n >= 1; --n) {
      cn = __ldg(c + n);
      r = fmaf(r, a, cn.x);
      d = fmaf(d, a, (float)n * cn.y);
    }
    e = fmaf(r, a, __ldg(c).x);                     // Re w(x) = e^{-x^2}
    g = -d;                                          // -Im w'(x)
  } else {
    const float hi = x * x, lo = fmaf(x, x, -hi);   // x^2 = hi + lo exactly
    const float ah = -hi * L2E;
    const float al = -fmaf(hi, L2E, ah) - fmaf(lo, L2E, hi * L2E_LO);
    float e2;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e2) : "f"(ah));
    e = e2 * fmaf(al, LN2, 1.0f);
    const float t = rcp_approx(hi);
    // (2k-1)!! / 2^k, k = 10 .. 1
    float sum = 639383.8623046875f;
    sum = fmaf(sum, t, 67303.564453125f);
    sum = fmaf(sum, t, 7918.06640625f);
    sum = fmaf(sum, t, 1055.7421875f);
    sum = fmaf(sum, t, 162.421875f);
    sum = fmaf(sum, t, 29.53125f);
    sum = fmaf(sum, t, 6.5625f);
    sum = fmaf(sum, t, 1.875f);
    sum = fmaf(sum, t, 0.75f);
    sum = fmaf(sum, t, 0.5f);
    g = TWO_SQRTPI * t * sum;
  }
  const float x2 = x * x, y2 = y * y;
  const float cub = x < 40.0f ? fmaf(g, fmaf(-4.0f, x2, 6.0f), 2.0f * TWO_SQRTPI) : 0.0f;
  const float gy = fmaf(y2 * (1.0f / 6.0f), cub, g);
  return fmaf(e, fmaf(y2, fmaf(-2.0f, x2, 1.0f), 1.0f), y * gy);
}

// Accurate branch for x^2 + y^2 < 576 (also valid beyond).
__device__ __forceinline__ float core_re(float x, float y, const float2* __restrict__ tab) {
  x = fabsf(x);
  float s = fmaf(x, x, y * y);
  if (s < 25.0f) return taylor_re(x, y, tab);
  float v = cf_re(x, y, s >= 64.0f ? 4 : 6);
  if (y < 1.0f) {
    // the Gaussian term matters only near the real axis; there 2xy is small
    float g = y * y - x * x;
    if (g > -87.0f) v += __expf(g) * __cosf(2.0f * x * y);
  }
  return v;
}

__device__ __forceinline__ float faddeeva_re(float x, float y, const float2* __restrict__ tab) {
  float s = fmaf(x, x, y * y);
  if (s >= 576.0f) return onepole_re(x, y);
  return core_re(x, y, tab);
}

}  // namespace bartw
