// Device helpers of the forward model: T(P) profile, exponential integral,
// Planck function, fast exponentials.
#pragma once

#include "bart_internal.cuh"

namespace bartf {

__device__ __forceinline__ float ex2_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

__device__ __forceinline__ float rcp_approx(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// Exponential integral E2(x), x >= 0, FP32.
//  x < 1: E2 = exp(-x) - x E1(x) with the power series
//         E1(x) = -gamma - ln x - sum_{k>=1} (-x)^k / (k k!);
//  x >= 1: the continued fraction of E_n (n = 2) evaluated by the modified
//         Lentz method, E_n(x) = exp(-x) / (x + n - 1 n / (x + n + 2 - 2 (n+1) / ...)).
__device__ inline float expint2f(float x) {
  if (x <= 0.0f) return 1.0f;
  if (x < 1.0f) {
    const float euler = 0.5772156649015329f;
    float term = 1.0f, sum = 0.0f;
    for (int k = 1; k <= 20; ++k) {
      term *= -x / (float)k;                  // (-x)^k / k!
      sum += term / (float)k;
    }
    float e1 = -euler - logf(x) - sum;
    return expf(-x) - x * e1;
  }
  if (x > 80.0f) return 0.0f;
  const float tiny = 1e-30f;
  float b = x + 2.0f, c = 1.0f / tiny, d = 1.0f / b, h = d;
  for (int i = 1; i <= 64; ++i) {
    float an = -(float)i * (float)(1 + i);
    b += 2.0f;
    d = 1.0f / fmaf(an, d, b);
    c = b + an / c;
    float del = c * d;
    h *= del;
    if (fabsf(del - 1.0f) < 1e-7f) break;
  }
  return h * expf(-x);
}

// xi(gamma, tau) of the three-channel profile (see tp_temperature).
__device__ inline float xi_channel(float g, float tau) {
  float gt = g * tau;
  return 2.0f / 3.0f + 2.0f / (3.0f * g) * (1.0f + (0.5f * gt - 1.0f) * expf(-gt)) +
         2.0f * g / 3.0f * (1.0f - 0.5f * tau * tau) * expint2f(gt);
}

// Temperature at pressure p_cgs (dyn cm^-2) of the five-parameter profile
// (Sec. 7: five T(p) parameters of Line et al. 2013), read as
//   T^4 = 3/4 Tint^4 (2/3 + tau) + 3/4 Tirr^4 [(1-alpha) xi(g1, tau) + alpha xi(g2, tau)],
//   tau = kappa p / g,  Tirr = beta sqrt(R_star / 2a) T_star.
// th = (log10 kappa, log10 gamma1, log10 gamma2, alpha, beta).
__device__ inline float tp_temperature(const float* th, float p_cgs, float inv_g, float tint4,
                                       float tirr0) {
  float kappa = exp10f(th[0]), g1 = exp10f(th[1]), g2 = exp10f(th[2]);
  float alpha = th[3], tirr = th[4] * tirr0;
  float tirr4 = (tirr * tirr) * (tirr * tirr);
  float tau = kappa * p_cgs * inv_g;
  float T4 = 0.75f * tint4 * (2.0f / 3.0f + tau) +
             0.75f * tirr4 * ((1.0f - alpha) * xi_channel(g1, tau) + alpha * xi_channel(g2, tau));
  return sqrtf(sqrtf(T4));
}

}  // namespace bartf
