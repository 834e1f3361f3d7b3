// Tangent-space pose update (Sec. 3.1, implementation details, Eq. tangent):
// the optimiser steps a zero tangent xi = (nu, omega) in se(3), which is then
// applied to the pose as (R', t') = exp(xi) (R, t) and reset.  Host code, FP64.
#include <cmath>
#include <cstring>

#include "launch.h"

namespace adop {
namespace {

// The three scalar coefficients of the closed-form SE(3) exponential at
// angle th = |omega|:
//   a = sin(th) / th, b = (1 - cos(th)) / th^2, c = (th - sin(th)) / th^3.
// Below th = 1 each is summed from its power series (alternating terms
// th^(2k) / (2k + 1)!, (2k + 2)!, (2k + 3)!), which avoids the cancellation
// of the quotients at small angles; twelve terms leave an error below
// 1 / 25!.  From th = 1 on the quotients lose nothing and are used directly.
void se3_coefficients(double th, double& a, double& b, double& c) {
  if (th < 1.0) {
    const double t2 = th * th;
    a = b = c = 0.0;
    double fa = 1.0, fb = 2.0, fc = 6.0;  // (2k+1)!, (2k+2)!, (2k+3)! at k = 0
    double p = 1.0;                       // th^(2k)
    for (int k = 0; k < 12; ++k) {
      const double sgn = (k & 1) ? -1.0 : 1.0;
      a += sgn * p / fa;
      b += sgn * p / fb;
      c += sgn * p / fc;
      p *= t2;
      fa *= (2.0 * k + 2.0) * (2.0 * k + 3.0);
      fb *= (2.0 * k + 3.0) * (2.0 * k + 4.0);
      fc *= (2.0 * k + 4.0) * (2.0 * k + 5.0);
    }
    return;
  }
  const double s = std::sin(th);
  const double h = std::sin(0.5 * th);
  a = s / th;
  b = 2.0 * h * h / (th * th);  // 1 - cos(th) = 2 sin^2(th / 2)
  c = (th - s) / (th * th * th);
}

// exp(xi) as a rotation E (row-major 3x3) and a translation e:
//   E = I + a K + b K^2, e = (I + b K + c K^2) nu, K = [omega]_x.
void se3_exp(const double* xi, double (&E)[9], double (&e)[3]) {
  const double nu[3] = {xi[0], xi[1], xi[2]};
  const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
  const double th = std::sqrt(w0 * w0 + w1 * w1 + w2 * w2);
  double a, b, c;
  se3_coefficients(th, a, b, c);
  const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
  double K2[9];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m) s += K[3 * r + m] * K[3 * m + q];
      K2[3 * r + q] = s;
    }
  for (int j = 0; j < 9; ++j) {
    const double id = (j % 4 == 0) ? 1.0 : 0.0;
    E[j] = id + a * K[j] + b * K2[j];
  }
  for (int r = 0; r < 3; ++r) {
    double s = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double id = (r == q) ? 1.0 : 0.0;
      s += (id + b * K[3 * r + q] + c * K2[3 * r + q]) * nu[q];
    }
    e[r] = s;
  }
}

}  // namespace
}  // namespace adop

extern "C" adop_status adop_pose_apply_tangent(const double* xi, adop_pose* poses, int32_t n) {
  if (n < 0) {
    adop::set_last_error("adop_pose_apply_tangent: n must be >= 0");
    return ADOP_ERR_INVALID_ARG;
  }
  if (n > 0 && (!xi || !poses)) {
    adop::set_last_error("adop_pose_apply_tangent: xi and poses must not be NULL");
    return ADOP_ERR_INVALID_ARG;
  }
  for (int32_t k = 0; k < n; ++k) {
    for (int j = 0; j < 6; ++j)
      if (!std::isfinite(xi[6 * k + j])) {
        adop::set_last_error("adop_pose_apply_tangent: non-finite tangent");
        return ADOP_ERR_INVALID_ARG;
      }
  }
  for (int32_t k = 0; k < n; ++k) {
    double E[9], e[3];
    adop::se3_exp(xi + 6 * k, E, e);
    adop_pose& P = poses[k];
    // (R', t') = exp(xi) (R, t): R' = E R, t' = E t + e, rounded to FP32 once
    float R[9], t[3];
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += E[3 * r + m] * (double)P.R[3 * m + q];
        R[3 * r + q] = (float)s;
      }
      double s = e[r];
      for (int m = 0; m < 3; ++m) s += E[3 * r + m] * (double)P.t[m];
      t[r] = (float)s;
    }
    std::memcpy(P.R, R, sizeof(R));
    std::memcpy(P.t, t, sizeof(t));
  }
  adop::set_last_error("");
  return ADOP_OK;
}
