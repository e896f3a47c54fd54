/*
 * A plain C caller of the library (include/lbm.h): a 128 x 96 droplet at a = 0.25,
 * T = 0.7 T_c with the improved forcing (sigma = 0.114, the value of Sec. IV B for
 * a = 0.25), started from the Maxwell densities (Eq. 22) with the tanh profile of Eq. 31,
 * stepped 500 times on the GPU.  Prints one line: mass drift, max |v|, centre and corner densities; exits non-zero
 * on any library error.  Built and run by tests/test_c_caller.py.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

#define NX 128
#define NY 96

static int check(int rc, lbm_handle* h, const char* what) {
  if (rc != LBM_OK) {
    fprintf(stderr, "%s failed (%d): %s\n", what, rc, lbm_last_error(h));
    return 1;
  }
  return 0;
}

int main(void) {
  const double a = 0.25, b = 4.0, R = 1.0;
  const double Tc = 0.3773 * a / (b * R);
  lbm_eos eos = {a, b, R, 0.7 * Tc};
  double rl = 0.0, rv = 0.0;
  if (lbm_maxwell(eos, &rl, &rv) != LBM_OK) return 2;
  const double s[9] = {1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0};
  lbm_options opt;
  lbm_options_default(&opt);
  opt.precision = LBM_FP32_DEV;
  lbm_handle* h = NULL;
  if (check(lbm_create(&h, NX, NY, eos, -1.0, 0.114, s, 0.0, 0.0, &opt), NULL, "lbm_create"))
    return 3;
  double* rho = malloc(sizeof(double) * NX * NY);
  for (int y = 0; y < NY; ++y)
    for (int x = 0; x < NX; ++x) {
      const double d = hypot(x - (NX - 1) / 2.0, y - (NY - 1) / 2.0);
      rho[y * NX + x] = 0.5 * (rl + rv) - 0.5 * (rl - rv) * tanh(2.0 * (d - 25.0) / 4.0);
    }
  int bad = check(lbm_init_fields(h, rho, NULL, NULL), h, "lbm_init_fields");
  lbm_diag d0, d1;
  bad = bad || check(lbm_diagnostics(h, &d0), h, "lbm_diagnostics");
  bad = bad || check(lbm_step(h, 500), h, "lbm_step");
  bad = bad || check(lbm_sync(h), h, "lbm_sync");
  bad = bad || check(lbm_diagnostics(h, &d1), h, "lbm_diagnostics");
  bad = bad || check(lbm_moments(h, rho, NULL, NULL), h, "lbm_moments");
  if (!bad)
    printf("mass_drift %.3e max_u %.3e rho_centre %.6f rho_corner %.6f steps %lld\n",
           fabs(d1.mass / d0.mass - 1.0), d1.max_u, rho[(NY / 2) * NX + NX / 2], rho[0],
           d1.step);
  free(rho);
  lbm_destroy(h);
  return bad ? 4 : 0;
}
