// Device evaluation of the stationary-phase template (App. A, Eq. A1) in FP64.
//   Psi(f) = 2 pi f tc - phic - pi/4 + 3/(128 eta) g(v),  v = (pi M f)^(1/3),
//   g(v)   = sum_k alpha_k v^(k-5) + a5log ln(v / v_lso) + a6log v ln(4 v),
//   Psi'   = 2 pi t(f) (Eq. A2),  Psi'' = 2 pi t'(f).
#pragma once

#include "rf_internal.h"

namespace rf {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kTwoPi = 6.28318530717958647692528676655900577;
constexpr double kSqrt6 = 2.44948974278317809819728407470589139;  // 1 / v_lso

__device__ __forceinline__ double tf2_series(const Tf2& p, double v) {
  const double iv = 1.0 / v;
  const double iv5 = iv * iv * iv * iv * iv;
  // sum_k a_k v^(k-5) = v^-5 (a0 + a1 v + ... + a7 v^7), Horner in v
  double poly = p.a[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) poly = poly * v + p.a[k];
  double g = poly * iv5;
  if (p.a5log != 0.0) g += p.a5log * log(v * kSqrt6);
  if (p.a6log != 0.0) g += p.a6log * v * log(4.0 * v);
  return g;
}

// Psi(f) in radians, f > 0.
__device__ __forceinline__ double tf2_phase(const Tf2& p, double f) {
  const double v = cbrt(kPi * p.M * f);
  return kTwoPi * f * p.tc - p.phic - 0.25 * kPi + p.pref * tf2_series(p, v);
}

// g'(v) and g''(v)
__host__ __device__ __forceinline__ void tf2_series_d(const Tf2& p, double v, double& g1, double& g2) {
  g1 = 0.0;
  g2 = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double e = (double)(k - 5);
    g1 += p.a[k] * e * pow(v, e - 1.0);
    g2 += p.a[k] * e * (e - 1.0) * pow(v, e - 2.0);
  }
  if (p.a5log != 0.0) {
    g1 += p.a5log / v;
    g2 -= p.a5log / (v * v);
  }
  if (p.a6log != 0.0) {
    g1 += p.a6log * (log(4.0 * v) + 1.0);
    g2 += p.a6log / v;
  }
}

// Psi'(f) = 2 pi tc + 3/(128 eta) g'(v) dv/df = 2 pi t(f) (Eq. A2)
__host__ __device__ __forceinline__ double tf2_dphase(const Tf2& p, double f) {
  const double v = cbrt(kPi * p.M * f);
  double g1, g2;
  tf2_series_d(p, v, g1, g2);
  return kTwoPi * p.tc + p.pref * g1 * (kPi * p.M / (3.0 * v * v));
}

// Psi''(f) = (pi M / (128 eta)) (g'' v^-2 - 2 g' v^-3) dv/df,  dv/df = pi M / (3 v^2)
__device__ __forceinline__ double tf2_d2phase(const Tf2& p, double f) {
  const double v = cbrt(kPi * p.M * f);
  double g1, g2;
  tf2_series_d(p, v, g1, g2);
  const double dv = kPi * p.M / (3.0 * v * v);
  return (kPi * p.M / (128.0 * p.eta)) * (g2 / (v * v) - 2.0 * g1 / (v * v * v)) * dv;
}

// B(f) = f^(-7/6)
__device__ __forceinline__ double tf2_amp(double f) { return exp(-7.0 / 6.0 * log(f)); }

// W(f) of Eq. (9)
__device__ __forceinline__ double window_w(double f, double f_low, double f_high, double dfl, double dfh) {
  if (f >= f_low && f <= f_high) return 1.0;
  if (f > f_low - dfl && f < f_low && dfl > 0.0) return 0.5 * (1.0 + cospi((f - f_low) / dfl));
  if (f > f_high && f < f_high + dfh && dfh > 0.0) return 0.5 * (1.0 - cospi((f - (f_high + dfh)) / dfh));
  return 0.0;
}

}  // namespace rf
