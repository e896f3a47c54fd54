// Host-side thermodynamics of the Carnahan-Starling fluid used by the library:
// the Maxwell equal-area construction (Eq. 22) for Eq. 30.
//
// With x = b rho / 4 the integral of p / rho^2 has the closed form
//   Phi(rho) = R T [ln rho + (4x - 3x^2) / (1 - x)^2] - a rho
// (the Carnahan-Starling excess free energy), so the equal-area condition
//   int_{rho_v}^{rho_l} (p0 - p) / rho^2 d rho = 0
// becomes p0 (1/rho_v - 1/rho_l) = Phi(rho_l) - Phi(rho_v) with p(rho_v) = p(rho_l) = p0.
// p0 is found by bisection between the spinodal pressures; each root by bisection.
#include <cmath>

#include "../../include/lbm.h"
#include "lbm_cs_host.h"

namespace {

using lbm_host::Cs;

template <typename F>
double bisect(F f, double lo, double hi, int iters = 200) {
  double flo = f(lo);
  for (int i = 0; i < iters; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double fm = f(mid);
    if ((fm > 0) == (flo > 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int lbm_maxwell(lbm_eos eos, double* rho_l, double* rho_v) {
  if (!rho_l || !rho_v || !(eos.a > 0) || !(eos.b > 0) || !(eos.R > 0) || !(eos.T > 0))
    return LBM_EINVAL;
  const Cs c{eos.a, eos.b, eos.R, eos.T};
  const double rmax = 4.0 / eos.b;
  // Spinodals: sign changes of dp/drho on a fine grid, refined by bisection.
  const int n = 4000;
  double sp[2];
  int ns = 0;
  double prev_r = rmax * 0.5 / n, prev = c.dp(prev_r);
  for (int i = 1; i < n && ns < 2; ++i) {
    const double r = rmax * (i + 0.5) / n;
    const double v = c.dp(r);
    if ((v > 0) != (prev > 0)) {
      sp[ns++] = bisect([&](double z) { return c.dp(z); }, prev_r, r);
    }
    prev = v;
    prev_r = r;
  }
  if (ns < 2) return LBM_EINVAL;  // not below the critical temperature
  const double s1 = sp[0], s2 = sp[1];
  const double p_hi = c.p(s1);
  double p_lo = c.p(s2);
  if (p_lo < 0.0) p_lo = 0.0;
  auto roots = [&](double p0, double& rv, double& rl) {
    rv = bisect([&](double r) { return c.p(r) - p0; }, 0.0, s1);
    rl = bisect([&](double r) { return c.p(r) - p0; }, s2, rmax * (1.0 - 1e-15));
  };
  auto g = [&](double p0) {
    double rv, rl;
    roots(p0, rv, rl);
    return p0 * (1.0 / rv - 1.0 / rl) - (c.phi(rl) - c.phi(rv));
  };
  const double span = p_hi - p_lo;
  const double lo = p_lo > 0 ? p_lo + 1e-9 * span : p_hi * 1e-9;
  const double hi = p_hi - 1e-9 * span;
  if ((g(lo) > 0) == (g(hi) > 0)) return LBM_EINVAL;
  const double p0 = bisect(g, lo, hi);
  double rv, rl;
  roots(p0, rv, rl);
  *rho_l = rl;
  *rho_v = rv;
  return LBM_OK;
}
