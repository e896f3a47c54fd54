/*
 * Warm start: measuring equilibria, encoding them for the network of lbm_mlp.h, and
 * initialising droplet fields from them.
 *
 * The paper initialises droplets with the tanh profile of Eq. 31 between the Maxwell
 * coexistence densities (Eq. 22) with W = 5 (Sec. IV A).  The lattice then relaxes to the
 * coexistence state the model actually selects (Eq. 21 for a flat interface), shifted
 * across curved interfaces by the Laplace pressure.  A warm start puts the field closer to
 * that state from the outset: coexistence densities, interface width and offset, and the
 * curvature shift of the vapour density, as predicted by the network from (a, T/T_c,
 * sigma, viscosity ratio).  The paper has no warm start; the quantities below are defined
 * here.
 *
 * Equilibrium quantities (physical units, lattice units for lengths):
 *   rho_l         bulk liquid density of a flat film;
 *   rho_v         vapour density in equilibrium with a droplet of infinite radius: the
 *                 vapour around droplets of equimolar radius R follows
 *                 rho_out(R) = rho_v (1 + curvature / R), and rho_v and curvature are the
 *                 intercept and slope of that law through two droplets of different radii;
 *   width         W of Eq. 31 as an integral width: with g = (rho - rho_v) / (rho_l - rho_v)
 *                 across one interface, W = 4 * integral of g (1 - g) (for the tanh profile
 *                 g (1 - g) = sech^2(2 d / W) / 4, whose integral is W / 4);
 *   shift         centroid of g (1 - g) across the interface (the centre of the tanh
 *                 profile that has the same centroid) minus the position of the equimolar
 *                 (Gibbs) dividing surface, positive towards the vapour (0 for Eq. 31);
 *   curvature     the Laplace correction of the vapour density in that law (a length,
 *                 > 0).  In this model the shift is far larger than the Kelvin shift of
 *                 the Carnahan-Starling fluid, because Eq. 21 weights the pressure by
 *                 psi'/psi^(1+eps) rather than 1/rho.
 *
 * All functions here except lbm_init_droplets and lbm_phase_stats are host-only and
 * synchronous, and need no GPU.  Return values as in lbm.h.
 */
#ifndef LBM_WARM_H
#define LBM_WARM_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double rho_l;
  double rho_v;
  double width;
  double shift;
  double curvature;
} lbm_warm_params;

typedef struct {
  double cx, cy;  /* centre, in node coordinates (node (x, y) sits at (x, y)) */
  double radius;  /* equimolar radius */
} lbm_droplet;

/*
 * Measure a flat film: rho (ny, nx) host doubles of a film that is uniform in x, with
 * the liquid centred on y = (ny - 1)/2 and the vapour centred on y = -1/2 (periodic).
 * The profile is the mean over x.  rho_l is its value at the film centre, rho_v at the
 * vapour centre (linear interpolation between rows); the Gibbs surface follows from the
 * liquid excess over the whole period, the width from the sum of g (1 - g) over the whole
 * period (two interfaces); the centroid of the shift from the rows above the film centre
 * up to the vapour centre (the upper interface).
 * Sets every field of *out but curvature (set to 0).  LBM_EINVAL if ny < 8 or if
 * rho_l <= rho_v.
 */
int lbm_measure_film(const double* rho, int nx, int ny, lbm_warm_params* out);

/*
 * Measure a droplet centred on ((nx - 1)/2, (ny - 1)/2) in a periodic nx x ny box:
 * rho_in at the centre and rho_out at the farthest point (mean of the nearest nodes),
 * the equimolar radius R from the total mass, pi R^2 (rho_in - rho_out) = sum(rho) -
 * nx ny rho_out, and the Laplace law's surface tension, laplace = (p(rho_in) -
 * p(rho_out)) R with p of Eq. 30 for `eos`.
 * Any output pointer may be NULL.  LBM_EINVAL if rho_in <= rho_out.
 */
int lbm_measure_droplet(const double* rho, int nx, int ny, lbm_eos eos, double* rho_in,
                        double* rho_out, double* radius, double* laplace);

/*
 * Network targets from equilibrium quantities and back, relative to the Maxwell densities
 * (rho_l^M, rho_v^M) of `eos` (Eq. 22):
 *   y = (rho_l / rho_l^M - 1, ln(rho_v / rho_v^M), width, shift, ln curvature).
 * LBM_EINVAL if eos is not below its critical temperature, or a density or the curvature
 * is not positive.
 */
int lbm_warm_encode(lbm_eos eos, const lbm_warm_params* p, double y[5]);
int lbm_warm_decode(lbm_eos eos, const double y[5], lbm_warm_params* p);

/*
 * The vapour law through two droplets: given the far vapour densities ro1, ro2 around
 * droplets of equimolar radii r1 != r2, the intercept rho_v and the curvature of
 * rho_out(R) = rho_v (1 + curvature / R).  LBM_EINVAL if r1 == r2 or a radius is not
 * positive.
 */
int lbm_vapour_law(double r1, double ro1, double r2, double ro2, double* rho_v,
                   double* curvature);

/*
 * Phase densities around droplets of mean curvature kappa (the mean of 1/R over the
 * droplets): rho_out = rho_v (1 + curvature kappa), and the liquid at the vapour's raised
 * pressure, to first order, rho_in = rho_l + (p(rho_out) - p(rho_v)) / p'(rho_l).
 * LBM_EINVAL if kappa < 0, rho_out <= 0 or rho_l is not on the stable liquid branch.
 */
int lbm_curved_densities(lbm_eos eos, const lbm_warm_params* p, double kappa, double* rho_in,
                         double* rho_out);

#define LBM_WARM_CURVATURE 1 /* flag: phase densities of lbm_curved_densities */
#define LBM_WARM_BALANCED 2  /* flag: start from u0 = -F / (2 rho) (F of Eq. 7 for the
                                field) instead of rest, so that the force-corrected velocity
                                of Eq. 6 is zero at t = 0 */

/*
 * Initialise the lattice with droplets (populations at the equilibrium of Eq. 3 at
 * u = 0, or at u0 with LBM_WARM_BALANCED, as lbm_init_fields): at every node the largest
 * over droplets of
 *   (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh(2 (r - R - shift) / width),
 * r the periodic distance to the droplet centre, R its radius; rho_out where no droplet
 * is within 8 widths.  (rho_in, rho_out) = (p->rho_l, p->rho_v), or with
 * LBM_WARM_CURVATURE those of lbm_curved_densities for the droplets' mean curvature.
 * With p = (Maxwell densities, W, shift 0) and no flags this is Eq. 31 for each droplet.
 * 1 <= n <= 65536.  The field is built on the device.
 * Resets the step counter and the dinf reference.  Synchronous.
 */
int lbm_init_droplets(lbm_handle* h, const lbm_droplet* drops, int n, const lbm_warm_params* p,
                      int flags);

/*
 * Phase-averaged densities of the current state: out[0] = mean rho over nodes with
 * rho < rho_vap_max, out[1] = their count, out[2] = mean rho over nodes with
 * rho > rho_liq_min, out[3] = their count (means 0 for empty sets).  Densities as in
 * lbm_moments (Eq. 6); sums in double, in a fixed order.  Synchronous.
 */
int lbm_phase_stats(lbm_handle* h, double rho_vap_max, double rho_liq_min, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
