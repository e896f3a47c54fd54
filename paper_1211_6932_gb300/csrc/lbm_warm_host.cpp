// Host-side warm-start helpers (declared in include/lbm_warm.h): measurement of flat-film
// and droplet equilibria, the network target encoding, and the phase densities around
// curved interfaces.  Definitions are stated in the header.
#include <cmath>
#include <vector>

#include "../../include/lbm_warm.h"
#include "lbm_cs_host.h"

namespace {

using lbm_host::Cs;

// Value of the periodic row profile at real position y (linear interpolation).
double at(const std::vector<double>& prof, double y) {
  const int n = (int)prof.size();
  const double f = std::floor(y);
  const double w = y - f;
  int i0 = (int)f % n;
  if (i0 < 0) i0 += n;
  const int i1 = (i0 + 1) % n;
  return (1.0 - w) * prof[i0] + w * prof[i1];
}

bool valid_eos(const lbm_eos& e) { return e.a > 0 && e.b > 0 && e.R > 0 && e.T > 0; }

}  // namespace

extern "C" {

int lbm_measure_film(const double* rho, int nx, int ny, lbm_warm_params* out) {
  if (!rho || !out || nx < 1 || ny < 8) return LBM_EINVAL;
  std::vector<double> prof(ny, 0.0);
  for (int y = 0; y < ny; ++y) {
    double s = 0.0;
    for (int x = 0; x < nx; ++x) s += rho[(size_t)y * nx + x];
    prof[y] = s / nx;
  }
  const double c = 0.5 * (ny - 1);
  const double rl = at(prof, c);
  const double rv = at(prof, -0.5 + ny);  // the vapour centre, y = -1/2 (periodic)
  const double d = rl - rv;
  if (!(d > 0.0) || !std::isfinite(d)) return LBM_EINVAL;
  double L = 0.0, G = 0.0;  // over one period, in rows: both interfaces
  for (int y = 0; y < ny; ++y) {
    const double g = (prof[y] - rv) / d;
    L += g;
    G += g * (1.0 - g);
  }
  const double yg = c + 0.5 * L;  // equimolar surface of the upper interface
  // centroid of g (1 - g) over the upper interface: rows floor(c) + 1 .. floor(c) + ny/2
  double sw = 0.0, swy = 0.0;
  const int y0 = (int)std::floor(c);
  for (int k = 1; k <= ny / 2; ++k) {
    const double g = (prof[(y0 + k) % ny] - rv) / d;
    sw += g * (1.0 - g);
    swy += g * (1.0 - g) * (double)(y0 + k);
  }
  if (!(G > 0.0) || !(sw > 0.0)) return LBM_EINVAL;
  const double yh = swy / sw;
  out->rho_l = rl;
  out->rho_v = rv;
  out->width = 2.0 * G;  // 4 * (G / 2) per interface
  out->shift = yh - yg;
  out->curvature = 0.0;
  return LBM_OK;
}

int lbm_measure_droplet(const double* rho, int nx, int ny, lbm_eos eos, double* rho_in,
                        double* rho_out, double* radius, double* laplace) {
  if (!rho || nx < 2 || ny < 2 || !valid_eos(eos)) return LBM_EINVAL;
  // mean of the nodes nearest to a point with half-integer or integer coordinates
  auto mean_at = [&](double px, double py) {
    const int x0 = (int)std::floor(px), x1 = (int)std::ceil(px);
    const int y0 = (int)std::floor(py), y1 = (int)std::ceil(py);
    auto v = [&](int x, int y) {
      x = ((x % nx) + nx) % nx;
      y = ((y % ny) + ny) % ny;
      return rho[(size_t)y * nx + x];
    };
    return 0.25 * (v(x0, y0) + v(x1, y0) + v(x0, y1) + v(x1, y1));
  };
  const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1);
  const double ri = mean_at(cx, cy);
  const double ro = mean_at(cx + 0.5 * nx, cy + 0.5 * ny);
  if (!(ri > ro) || !std::isfinite(ri) || !std::isfinite(ro) || !(ro > 0.0)) return LBM_EINVAL;
  double M = 0.0;
  for (size_t k = 0; k < (size_t)nx * ny; ++k) M += rho[k];
  const double excess = M - (double)nx * ny * ro;
  if (!(excess > 0.0)) return LBM_EINVAL;
  const double R = std::sqrt(excess / (M_PI * (ri - ro)));
  const Cs cs{eos.a, eos.b, eos.R, eos.T};
  if (rho_in) *rho_in = ri;
  if (rho_out) *rho_out = ro;
  if (radius) *radius = R;
  if (laplace) *laplace = (cs.p(ri) - cs.p(ro)) * R;
  return LBM_OK;
}

int lbm_warm_encode(lbm_eos eos, const lbm_warm_params* p, double y[5]) {
  if (!p || !y || !valid_eos(eos)) return LBM_EINVAL;
  double ml = 0.0, mv = 0.0;
  if (lbm_maxwell(eos, &ml, &mv) != LBM_OK) return LBM_EINVAL;
  if (!(p->rho_l > 0.0) || !(p->rho_v > 0.0) || !(p->curvature > 0.0)) return LBM_EINVAL;
  y[0] = p->rho_l / ml - 1.0;
  y[1] = std::log(p->rho_v / mv);
  y[2] = p->width;
  y[3] = p->shift;
  y[4] = std::log(p->curvature);
  return LBM_OK;
}

int lbm_warm_decode(lbm_eos eos, const double y[5], lbm_warm_params* p) {
  if (!p || !y || !valid_eos(eos)) return LBM_EINVAL;
  double ml = 0.0, mv = 0.0;
  if (lbm_maxwell(eos, &ml, &mv) != LBM_OK) return LBM_EINVAL;
  p->rho_l = ml * (1.0 + y[0]);
  p->rho_v = mv * std::exp(y[1]);
  p->width = y[2];
  p->shift = y[3];
  p->curvature = std::exp(y[4]);
  return p->rho_l > 0.0 ? LBM_OK : LBM_EINVAL;
}

int lbm_vapour_law(double r1, double ro1, double r2, double ro2, double* rho_v,
                   double* curvature) {
  if (!rho_v || !curvature || !(r1 > 0.0) || !(r2 > 0.0) || r1 == r2) return LBM_EINVAL;
  const double slope = (ro1 - ro2) / (1.0 / r1 - 1.0 / r2);  // rho_v * curvature
  const double icpt = ro2 - slope / r2;
  *rho_v = icpt;
  *curvature = slope / icpt;
  return LBM_OK;
}

int lbm_curved_densities(lbm_eos eos, const lbm_warm_params* p, double kappa, double* rho_in,
                         double* rho_out) {
  if (!p || !rho_in || !rho_out || !valid_eos(eos) || !(kappa >= 0.0)) return LBM_EINVAL;
  const Cs cs{eos.a, eos.b, eos.R, eos.T};
  const double slope = cs.dp(p->rho_l);
  if (!(slope > 0.0)) return LBM_EINVAL;  // rho_l is not on the stable liquid branch
  const double ro = p->rho_v * (1.0 + p->curvature * kappa);
  if (!(ro > 0.0)) return LBM_EINVAL;
  *rho_out = ro;
  *rho_in = p->rho_l + (cs.p(ro) - cs.p(p->rho_v)) / slope;
  return LBM_OK;
}

}  // extern "C"
