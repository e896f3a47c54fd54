// Discrete pressure tensor of Eq. 18 (lbm_pressure_tensor): a diagnostic, evaluated in
// double precision from the node densities of the current state.
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

// One thread per node (grid-stride):
//   P = rho c_s^2 I + (G/2) psi(x) sum_q w_q psi(x + e_q) e_q e_q,   w = 1/3 (axes), 1/12,
// plus, when sigma != 0, the isotropic 2 sigma |F/psi|^2 of the improved forcing (the
// extra stress of Eq. 26, 2 G^2 sigma |grad psi|^2, with the gradient of the force
// stencil, F/psi = -G sum_q w_q psi(x + e_q) e_q).  psi of a ghost row beyond a wall is
// psi of the adjacent fluid row, as in the step.
template <typename S>
__global__ void __launch_bounds__(256) pressure_kernel(const S* __restrict__ rho, InstParams P,
                                                       double sigma, double* __restrict__ pxx,
                                                       double* __restrict__ pyy,
                                                       double* __restrict__ pxy) {
  const int nx = P.nx, ny = P.ny;
  const long long N = (long long)nx * ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    auto psi_at = [&](int xx, int yy) {
      xx = wrapi(xx, nx);
      yy = P.walls ? (yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy)) : wrapi(yy, ny);
      return psi_eval_f64((double)rho[(long long)yy * nx + xx], P.b4, P.RT, P.a, P.two_over_G);
    };
    double sxx = 0.0, syy = 0.0, sxy = 0.0, gx = 0.0, gy = 0.0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      const int ex = ex_of(q), ey = ey_of(q);
      const double w = (q <= 4) ? (1.0 / 3.0) : (1.0 / 12.0);
      const double wp = w * psi_at(x + ex, y + ey);
      sxx += wp * ex * ex;
      syy += wp * ey * ey;
      sxy += wp * ex * ey;
      gx += wp * ex;
      gy += wp * ey;
    }
    const double r = (double)rho[i];
    const double hp = 0.5 * P.G * psi_at(x, y);
    double iso = r / 3.0;
    if (sigma != 0.0) iso += 2.0 * sigma * P.G * P.G * (gx * gx + gy * gy);
    pxx[i] = iso + hp * sxx;
    pyy[i] = iso + hp * syy;
    pxy[i] = hp * sxy;
  }
}

}  // namespace

template <typename S>
cudaError_t launch_pressure(const S* rho, const InstParams& P, double sigma, double* pxx,
                            double* pyy, double* pxy, cudaStream_t st) {
  const long long N = (long long)P.nx * P.ny;
  long long g = (N + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  pressure_kernel<S><<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(rho, P, sigma, pxx, pyy, pxy);
  return cudaGetLastError();
}

template cudaError_t launch_pressure<float>(const float*, const InstParams&, double, double*,
                                            double*, double*, cudaStream_t);
template cudaError_t launch_pressure<double>(const double*, const InstParams&, double, double*,
                                             double*, double*, cudaStream_t);

}  // namespace lbm
