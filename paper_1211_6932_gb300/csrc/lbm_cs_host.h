// Host-side Carnahan-Starling pressure (Eq. 30), its density derivative and the
// integral of p / rho^2 (used by the Maxwell rule), shared by the host C++ files.
#pragma once
#include <cmath>

namespace lbm_host {

struct Cs {
  double a, b, R, T;
  double p(double r) const {
    const double x = b * r / 4.0;
    return r * R * T * (1.0 + x + x * x - x * x * x) / ((1.0 - x) * (1.0 - x) * (1.0 - x)) -
           a * r * r;
  }
  double dp(double r) const {
    // d/drho of rho R T Z(x) - a rho^2 = R T (Z + x Z') - 2 a rho
    const double x = b * r / 4.0, u = 1.0 - x;
    const double N = 1.0 + x + x * x - x * x * x, N1 = 1.0 + 2.0 * x - 3.0 * x * x;
    const double Z = N / (u * u * u), Z1 = N1 / (u * u * u) + 3.0 * N / (u * u * u * u);
    return R * T * (Z + x * Z1) - 2.0 * a * r;
  }
  double phi(double r) const {
    const double x = b * r / 4.0, u = 1.0 - x;
    return R * T * (std::log(r) + (4.0 * x - 3.0 * x * x) / (u * u)) - a * r;
  }
};

}  // namespace lbm_host
