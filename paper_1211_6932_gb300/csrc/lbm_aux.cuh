// Conversions between the canonical population layout and the step kernel's storage,
// equilibrium initialisation, psi evaluation and the diagnostics reduction.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

// Storage slot that holds the population f_q of node (x, y) at the current time.
// Pull streaming stores f*_q(x - e_q) at x - e_q; next to a wall the bounced population
// f*_{opp q}(x) of the node itself plays that role (halfway bounce-back).
__device__ __forceinline__ long long slot_of(const InstParams& P, int q, int x, int y,
                                             int& qs) {
  int ys = y - ey_of(q);
  int xs = x - ex_of(q);
  qs = q;
  if (ys < 0 || ys >= P.ny) {
    if (P.walls) {
      qs = opp_of(q);
      ys = y;
      xs = x;
    } else {
      ys = ys < 0 ? ys + P.ny : ys - P.ny;
    }
  }
  xs = xs < 0 ? xs + P.nx : (xs >= P.nx ? xs - P.nx : xs);
  return P.off + (long long)qs * P.plane + (long long)ys * P.pitch + GHOST + xs;
}

// Refresh the ghost columns -2, -1, nx, nx+1 of every row from the columns they mirror
// (periodic x); the step kernel keeps them current afterwards.
template <typename S>
__global__ void fill_ghosts_kernel(S* __restrict__ buf, InstParams P) {
  const long long total = (long long)Q * P.ny * 4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i & 3);
    const long long qy = i >> 2;
    const int y = (int)(qy % P.ny), q = (int)(qy / P.ny);
    const int g = k == 0 ? -2 : (k == 1 ? -1 : (k == 2 ? P.nx : P.nx + 1));
    S* row = buf + P.off + (long long)q * P.plane + (long long)y * P.pitch + GHOST;
    row[g] = row[wrapi(g, P.nx)];
  }
}

// Canonical host-order populations (Q, ny, nx) -> storage.
template <typename S>
__global__ void set_pops_kernel(const double* __restrict__ fc, S* __restrict__ buf,
                                InstParams P) {
  const long long N = (long long)P.nx * P.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % P.nx), y = (int)(n / P.nx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int qs;
      const long long s = slot_of(P, q, x, y, qs);
      buf[s] = (S)(fc[q * N + n] - tw_of(q) * P.rho_ref);
    }
  }
}

// Storage -> canonical populations (Q, ny, nx) in double.
template <typename S>
__global__ void get_pops_kernel(const S* __restrict__ buf, double* __restrict__ fc,
                                InstParams P) {
  const long long N = (long long)P.nx * P.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % P.nx), y = (int)(n / P.nx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int qs;
      const long long s = slot_of(P, q, x, y, qs);
      fc[q * N + n] = (double)buf[s] + tw_of(q) * P.rho_ref;
    }
  }
}

// Second-order equilibrium f_q = t_q rho [1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2] (its moments
// are Eq. 3), stored as deviations.  rho, ux, uy: dense (ny, nx) doubles; ux/uy may be null.
template <typename S>
__global__ void init_eq_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                               const double* __restrict__ uy, S* __restrict__ buf,
                               InstParams P, int* __restrict__ bad) {
  // Arithmetic in the storage type; only the deviation rho - rho_ref is formed in double.
  typedef S R;
  const PhysParams<R>& pp = phys_params<R>(P);
  const long long N = (long long)P.nx * P.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % P.nx), y = (int)(n / P.nx);
    const double rd = rho[n];
    const R r = (R)rd, dr = (R)(rd - P.rho_ref);
    const R u = ux ? (R)ux[n] : (R)0, v = uy ? (R)uy[n] : (R)0;
    const R xb = pp.b4 * r;
    const R brk = pp.RT * (((R)1 + xb * ((R)1 + xb * ((R)1 - xb))) /
                           (((R)1 - xb) * ((R)1 - xb) * ((R)1 - xb))) -
                  pp.a * r - (R)(1.0 / 3.0);
    const R psi2 = pp.two_over_G * r * brk;
    if (!(r > (R)0) || !(xb < (R)1) || !(psi2 >= (R)0) || !isfinite(u) || !isfinite(v))
      atomicAdd(bad, 1);
    const R u2 = u * u + v * v;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const R eu = (R)ex_of(q) * u + (R)ey_of(q) * v;
      // t_q rho [1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2] - t_q rho_ref
      const R h = (R)tw_of(q) * (dr + r * ((R)3 * eu + (R)4.5 * eu * eu - (R)1.5 * u2));
      int qs;
      const long long s = slot_of(P, q, x, y, qs);
      buf[s] = (S)h;
    }
  }
}

// psi as the step kernel evaluates it (same precision and mode), for testing.
template <typename S>
__global__ void psi_kernel(const double* __restrict__ rho, double* __restrict__ out,
                           long long n, const InstParams* __restrict__ Pp) {
  const Phys<S> ph = load_phys<S>(*Pp);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)psi_t<S, S>((S)rho[i], ph);
}

}  // namespace lbm
