// Device side of the warm start (include/lbm_warm.h): the droplet-field fill and the
// phase-averaged density sums.
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kFillThreads = 256;
constexpr int kDropTile = 256;  // droplets staged in shared memory per pass

// One thread per node: the largest tanh profile over the droplets within reach (8
// widths beyond the half-density circle), else rho_v.
__global__ void __launch_bounds__(kFillThreads) fill_droplets_kernel(
    double* __restrict__ rho, int nx, int ny, const DropRec* __restrict__ drops, int n,
    double rho_v, double width) {
  __shared__ DropRec sd[kDropTile];
  const long long N = (long long)nx * ny;
  const long long node = (long long)blockIdx.x * kFillThreads + threadIdx.x;
  const bool live = node < N;
  const int x = live ? (int)(node % nx) : 0, y = live ? (int)(node / nx) : 0;
  const double reach = 8.0 * width;
  double best = rho_v;
  for (int base = 0; base < n; base += kDropTile) {
    const int m = min(kDropTile, n - base);
    __syncthreads();
    if ((int)threadIdx.x < m) sd[threadIdx.x] = drops[base + threadIdx.x];
    __syncthreads();
    if (!live) continue;
    for (int k = 0; k < m; ++k) {
      const DropRec d = sd[k];
      double dx = fabs((double)x - d.cx);
      dx = fmin(dx, (double)nx - dx);
      double dy = fabs((double)y - d.cy);
      dy = fmin(dy, (double)ny - dy);
      const double s = sqrt(dx * dx + dy * dy) - d.r_half;
      if (s > reach) continue;
      const double v = 0.5 * (d.rho_in + rho_v) - 0.5 * (d.rho_in - rho_v) * tanh(2.0 * s / width);
      best = fmax(best, v);
    }
  }
  if (live) rho[node] = best;
}

// u0 = -F / (2 rho) with F of Eq. 7 from psi of Eq. 24 of the density field: the initial
// velocity for which the force-corrected velocity of Eq. 6, (sum e f + F/2) / rho, is zero
// when f is the equilibrium at (rho, u0).  psi beyond a wall is that of the adjacent row.
__global__ void __launch_bounds__(256) balanced_velocity_kernel(
    const double* __restrict__ rho, InstParams P, double* __restrict__ ux,
    double* __restrict__ uy) {
  const int nx = P.nx, ny = P.ny;
  const long long N = (long long)nx * ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    auto psi_at = [&](int xx, int yy) {
      xx = wrapi(xx, nx);
      yy = P.walls ? (yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy)) : wrapi(yy, ny);
      return psi_eval_f64(rho[(long long)yy * nx + xx], P.b4, P.RT, P.a, P.two_over_G);
    };
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      const double w = (q <= 4) ? (1.0 / 3.0) : (1.0 / 12.0);
      const double wp = w * psi_at(x + ex_of(q), y + ey_of(q));
      gx += wp * ex_of(q);
      gy += wp * ey_of(q);
    }
    const double f = -P.G * psi_at(x, y);  // F = -G psi(x) sum w psi(x + e) e
    const double r = rho[i];
    ux[i] = -0.5 * f * gx / r;
    uy[i] = -0.5 * f * gy / r;
  }
}

template <typename S>
__global__ void __launch_bounds__(256) phase_sums_kernel(const S* __restrict__ rho, long long n,
                                                         double vmax, double lmin,
                                                         double* __restrict__ part) {
  __shared__ double red[4][256];
  double sv = 0.0, cv = 0.0, sl = 0.0, cl = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n;
       i += (long long)gridDim.x * 256) {
    const double r = (double)rho[i];
    if (r < vmax) {
      sv += r;
      cv += 1.0;
    }
    if (r > lmin) {
      sl += r;
      cl += 1.0;
    }
  }
  const int t = threadIdx.x;
  red[0][t] = sv;
  red[1][t] = cv;
  red[2][t] = sl;
  red[3][t] = cl;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h)
      for (int k = 0; k < 4; ++k) red[k][t] += red[k][t + h];
    __syncthreads();
  }
  if (t < 4) part[4 * blockIdx.x + t] = red[t][0];
}

}  // namespace

cudaError_t launch_fill_droplets(double* rho, int nx, int ny, const DropRec* drops, int n,
                                 double rho_v, double width, cudaStream_t st) {
  const long long N = (long long)nx * ny;
  const long long blocks = (N + kFillThreads - 1) / kFillThreads;
  fill_droplets_kernel<<<(unsigned)blocks, kFillThreads, 0, st>>>(rho, nx, ny, drops, n, rho_v,
                                                                  width);
  return cudaGetLastError();
}

cudaError_t launch_balanced_velocity(const double* rho, const InstParams& P, double* ux,
                                    double* uy, cudaStream_t st) {
  const long long N = (long long)P.nx * P.ny;
  long long g = (N + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  balanced_velocity_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(rho, P, ux, uy);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_phase_sums(const S* rho, long long n, double vmax, double lmin, double* part,
                              cudaStream_t st) {
  phase_sums_kernel<S><<<kPhaseBlocks, 256, 0, st>>>(rho, n, vmax, lmin, part);
  return cudaGetLastError();
}

template cudaError_t launch_phase_sums<float>(const float*, long long, double, double, double*,
                                              cudaStream_t);
template cudaError_t launch_phase_sums<double>(const double*, long long, double, double, double*,
                                               cudaStream_t);

}  // namespace lbm
