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

extern "C" int lbm_eos_psi2(lbm_eos eos, double G, double rho, double* out) {
  if (!out || !(eos.a > 0) || !(eos.b > 0) || !(eos.R > 0) || !(eos.T > 0) || !(G != 0) ||
      !(rho > 0) || !(rho < 4.0 / eos.b))
    return LBM_EINVAL;
  const Cs c{eos.a, eos.b, eos.R, eos.T};
  *out = 2.0 * (c.p(rho) - rho / 3.0) / G;
  return LBM_OK;
}

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

// ---------------------------------------------------------------------------------------
// The mechanical-stability condition of Eq. 21 for the potential of Eq. 24,
//   int_{rho_v}^{rho_l} (p0 - p(rho)) psi'(rho) / psi(rho)^(1 + eps) d rho = 0,
// with p0 = p(rho_v) = p(rho_l) and eps = -2 (alpha + 24 G sigma) / beta, alpha = 0,
// beta = 3 (nearest neighbours, Eq. 20 with the improved forcing of Eq. 25).  Since
// psi^2 = 2 (p - rho/3) / G, psi' = (p' - 1/3) / (G psi).  The integral is taken in
// t = ln rho (the weight spans orders of magnitude between the phases) with composite
// 8-point Gauss-Legendre on 256 equal panels; p0 by bisection as for Eq. 22.
namespace {

const double kGL8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                         -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                         0.7966664774136267,  0.9602898564975363};
const double kGL8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                         0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                         0.2223810344533745, 0.1012285362903763};

bool spinodals(const Cs& c, double rmax, double& s1, double& s2) {
  const int n = 4000;
  double sp[2];
  int ns = 0;
  double prev_r = rmax * 0.5 / n, prev = c.dp(prev_r);
  for (int i = 1; i < n && ns < 2; ++i) {
    const double r = rmax * (i + 0.5) / n;
    const double v = c.dp(r);
    if ((v > 0) != (prev > 0)) sp[ns++] = bisect([&](double z) { return c.dp(z); }, prev_r, r);
    prev = v;
    prev_r = r;
  }
  if (ns < 2) return false;
  s1 = sp[0];
  s2 = sp[1];
  return true;
}

int mech_stability(const lbm_eos& eos, double G, double sigma, double* rho_l, double* rho_v) {
  if (!rho_l || !rho_v || !(eos.a > 0) || !(eos.b > 0) || !(eos.R > 0) || !(eos.T > 0) ||
      !(G < 0) || !(sigma >= 0))
    return LBM_EINVAL;
  const Cs c{eos.a, eos.b, eos.R, eos.T};
  const double rmax = 4.0 / eos.b;
  double s1, s2;
  if (!spinodals(c, rmax, s1, s2)) return LBM_EINVAL;
  const double eps = -16.0 * G * sigma;
  auto weight = [&](double r) {  // psi' / psi^(1+eps)
    const double psi2 = 2.0 * (c.p(r) - r / 3.0) / G;
    if (!(psi2 > 0.0)) return 0.0;
    const double psi = std::sqrt(psi2);
    return (c.dp(r) - 1.0 / 3.0) / (G * psi) / std::pow(psi, 1.0 + eps);
  };
  auto roots = [&](double p0, double& rv, double& rl) {
    rv = bisect([&](double r) { return c.p(r) - p0; }, 0.0, s1);
    rl = bisect([&](double r) { return c.p(r) - p0; }, s2, rmax * (1.0 - 1e-15));
  };
  auto g = [&](double p0) {
    double rv, rl;
    roots(p0, rv, rl);
    const double t0 = std::log(rv), t1 = std::log(rl);
    const int panels = 256;
    const double h = (t1 - t0) / panels;
    double sum = 0.0;
    for (int k = 0; k < panels; ++k) {
      const double mid = t0 + (k + 0.5) * h;
      for (int j = 0; j < 8; ++j) {
        const double r = std::exp(mid + 0.5 * h * kGL8x[j]);
        sum += kGL8w[j] * 0.5 * h * r * (p0 - c.p(r)) * weight(r);
      }
    }
    return sum;
  };
  const double p_hi = c.p(s1);
  double p_lo = c.p(s2);
  if (p_lo < 0.0) p_lo = 0.0;
  const double span = p_hi - p_lo;
  const double lo = p_lo > 0 ? p_lo + 1e-9 * span : p_hi * 1e-9;
  const double hi = p_hi - 1e-9 * span;
  if ((g(lo) > 0) == (g(hi) > 0)) return LBM_EINVAL;
  const double p0 = bisect(g, lo, hi, 120);
  double rv, rl;
  roots(p0, rv, rl);
  *rho_l = rl;
  *rho_v = rv;
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_mechanical_stability(lbm_eos eos, double G, double sigma, double* rho_l,
                                        double* rho_v) {
  return mech_stability(eos, G, sigma, rho_l, rho_v);
}

extern "C" int lbm_sigma_consistent(lbm_eos eos, double G, double* sigma) {
  if (!sigma) return LBM_EINVAL;
  double ml, mv;
  if (lbm_maxwell(eos, &ml, &mv) != LBM_OK) return LBM_EINVAL;
  // The vapour density of Eq. 21 rises with sigma.  Scan sigma = 0.01 .. 0.5 for the
  // first pair of solvable neighbours across which ln(rho_v / rho_v^M) changes sign (Eq. 21
  // has no solution for small sigma at low temperatures), then bisect between them.
  auto h = [&](double s, bool& ok) {
    double rl, rv;
    ok = mech_stability(eos, G, s, &rl, &rv) == LBM_OK;
    return ok ? std::log(rv / mv) : 0.0;
  };
  double lo = -1.0, hi = -1.0, prev_s = -1.0, prev_h = 0.0;
  for (int k = 1; k <= 50; ++k) {
    const double sk = 0.01 * k;
    bool ok;
    const double hk = h(sk, ok);
    if (!ok) {
      prev_s = -1.0;
      continue;
    }
    if (prev_s >= 0.0 && prev_h < 0.0 && hk >= 0.0) {
      lo = prev_s;
      hi = sk;
      break;
    }
    prev_s = sk;
    prev_h = hk;
  }
  if (lo < 0.0) return LBM_EINVAL;
  for (int i = 0; i < 40; ++i) {
    const double mid = 0.5 * (lo + hi);
    bool ok;
    const double hm = h(mid, ok);
    if (!ok) return LBM_EINVAL;
    if (hm > 0.0) hi = mid;
    else lo = mid;
  }
  *sigma = 0.5 * (lo + hi);
  return LBM_OK;
}
