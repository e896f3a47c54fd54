// Device side of the D2Q9 MRT pseudopotential step (Li, Luo & Li, arXiv:1211.6932).
//
// One fused kernel per time step.  A CTA owns a strip of W columns and a chunk of rows of
// one lattice instance and sweeps the chunk row by row:
//   pull the nine populations of the next row (Eq. 5, pull form), sum them to rho (Eq. 6),
//   evaluate psi (Eqs. 24 and 30) into a four-row ring in shared memory, and, one row
//   behind, form F from the 3x3 psi stencil (Eq. 7), v (Eq. 6), the MRT collision with the
//   improved forcing term (Eqs. 3, 4, 25) and store the post-collision populations at the
//   node itself (aligned, vectorised stores).
// psi of the two halo columns and halo rows is recomputed from the populations, so every
// population value is read from DRAM once per step and written once: 72 B per lattice
// update in FP32.
//
// Storage: structure of arrays, plane q at fin[off + q*plane + y*pitch + x].  The stored
// value is the post-collision population of the previous step minus t_q * rho_ref
// (deviation storage; rho_ref = 0 gives plain storage).  The population at node x and the
// current time is the pulled value f_q(x) = buf_q(x - e_q) + t_q rho_ref.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 9;
constexpr int NT = 128;  // threads per CTA in the sweep kernel

// D2Q9 velocities: rest, E, N, W, S, NE, NW, SW, SE.
__host__ __device__ constexpr int ex_of(int q) {
  return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int q) {
  return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int q) {
  return q == 0 ? 0 : (q <= 4 ? ((q + 1) & 3) + 1 : ((q - 3) & 3) + 5);
}
// Equilibrium weights t_q: 4/9, 1/9 (axes), 1/36 (diagonals).
__host__ __device__ constexpr double tw_of(int q) {
  return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

enum { VISC_CONST = 0, VISC_STEP = 1, VISC_LINEAR = 2 };
enum { MODE_STEP = 0, MODE_MOMENTS = 1 };
enum { MOM_FIELDS = 1, MOM_DIAG = 2, MOM_UPDATE_PREV = 4 };
enum { STATUS_NONFINITE = 1 };

// Parameters of one lattice instance (host fills, kernels read).
struct InstParams {
  int nx, ny;
  int pitch;           // row stride in elements, a multiple of 4
  int walls;           // 0: periodic in y; 1: halfway bounce-back walls at y=-1/2, ny-1/2
  long long off;       // element offset of plane 0 inside the population slab
  long long plane;     // elements per population plane (ny * pitch)
  long long dense_off; // element offset inside dense (ny*nx) per-node arrays
  int visc_mode;       // VISC_*
  int psi_fp64;        // FP32 storage only: evaluate psi in double precision
  double b4;           // b / 4 (Eq. 30)
  double RT, a;        // R T and a (Eq. 30)
  double two_over_G;   // 2 / G (Eq. 24, c = 1)
  double G;            // interaction strength (Eq. 7)
  double s[Q];         // relaxation rates (Eq. 2)
  double sig12_e;      // 12 sigma s_e: (1 - s_e/2) * 12 sigma / (tau_e - 1/2) (Eq. 25)
  double sig12_z;      // 12 sigma s_zeta, same reduction for the third row of Eq. 25
  double tau_l, tau_v; // 3 nu + 1/2 for the liquid and vapour viscosities
  double rho_c;        // switch density of VISC_STEP
  double rho_l, rho_v; // end points of VISC_LINEAR
  double rho_ref;      // deviation reference density
};

// One CTA's share of the work: columns [x0, x0 + W) and rows [y0, y1) of instance inst.
// dir = +1 sweeps upwards, -1 downwards.  Alternating the direction between neighbouring
// chunks makes the two CTAs that share a halo row reach it at about the same time, so the
// second read of that row hits L2.
struct WorkItem {
  int inst, x0, y0, y1;
  int dir, pad0, pad1, pad2;
};

template <typename S>
struct MomArgs {
  S* rho;              // dense ny*nx per instance (dense_off), or null
  S* ux;
  S* uy;
  S* rho_prev;         // previous density for the |d rho|_inf diagnostic, or null
  double* part_sum;    // 3 per work item: sum rho, sum rho v_x, sum rho v_y
  float* part_max;     // 2 per work item: max |v|, max |rho - rho_prev|
  int* part_bad;       // 1 per work item: count of non-finite nodes
  int flags;           // MOM_*
};

template <typename R>
struct Phys {
  R b4, RT, a, two_over_G, G;
  R s1, s2, s4, s6, s7, s8;
  R sig12_e, sig12_z;
  R tau_l, tau_v, rho_c, rho_l, inv_drho_lv, rho_v;
  R rho_ref;
  int visc_mode, psi_fp64;
  double b4d, RTd, ad, two_over_Gd;
};

template <typename R>
__device__ __forceinline__ Phys<R> load_phys(const InstParams& P) {
  Phys<R> p;
  p.b4 = (R)P.b4; p.RT = (R)P.RT; p.a = (R)P.a; p.two_over_G = (R)P.two_over_G; p.G = (R)P.G;
  p.s1 = (R)P.s[1]; p.s2 = (R)P.s[2]; p.s4 = (R)P.s[4]; p.s6 = (R)P.s[6];
  p.s7 = (R)P.s[7]; p.s8 = (R)P.s[8];
  p.sig12_e = (R)P.sig12_e; p.sig12_z = (R)P.sig12_z;
  p.tau_l = (R)P.tau_l; p.tau_v = (R)P.tau_v; p.rho_c = (R)P.rho_c;
  p.rho_l = (R)P.rho_l; p.rho_v = (R)P.rho_v;
  p.inv_drho_lv = (P.rho_l != P.rho_v) ? (R)(1.0 / (P.rho_l - P.rho_v)) : (R)0;
  p.rho_ref = (R)P.rho_ref;
  p.visc_mode = P.visc_mode; p.psi_fp64 = P.psi_fp64;
  p.b4d = P.b4; p.RTd = P.RT; p.ad = P.a; p.two_over_Gd = P.two_over_G;
  return p;
}

__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float recip(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }

// psi of Eq. 24 with the Carnahan-Starling pressure of Eq. 30, written in factored form
//   psi^2 = (2/G) * rho * (R T Z(x) - a rho - 1/3),  x = b rho / 4,
//   Z(x) = (1 + x + x^2 - x^3) / (1 - x)^3,
// which equals 2 (p_EOS - rho/3) / G.  Pulling rho out of the bracket leaves three terms
// of comparable size and no cancellation at vapour density.  Negative arguments clamp to 0.
template <typename R>
__device__ __forceinline__ R psi_eval(R rho, const Phys<R>& p) {
  R x = p.b4 * rho;
  R num = (R)1 + x * ((R)1 + x * ((R)1 - x));
  R omx = (R)1 - x;
  R z = fast_div(num, omx * omx * omx);
  R brk = p.RT * z - p.a * rho - (R)(1.0 / 3.0);
  R arg = p.two_over_G * rho * brk;
  return sqrt_(arg > (R)0 ? arg : (R)0);
}
__device__ __forceinline__ double psi_eval_f64(double rho, double b4, double RT, double a,
                                               double two_over_G) {
  double x = b4 * rho;
  double num = 1.0 + x * (1.0 + x * (1.0 - x));
  double omx = 1.0 - x;
  double z = num / (omx * omx * omx);
  double arg = two_over_G * rho * (RT * z - a * rho - (1.0 / 3.0));
  return sqrt(arg > 0.0 ? arg : 0.0);
}
template <typename R>
__device__ __forceinline__ R psi_of(R rho, const Phys<R>& p) {
  if (sizeof(R) == 4 && p.psi_fp64)
    return (R)psi_eval_f64((double)rho, p.b4d, p.RTd, p.ad, p.two_over_Gd);
  return psi_eval<R>(rho, p);
}

// Stress-moment rate for the viscosity modes (Eq. 10: nu = (tau - 1/2)/3).
template <typename R>
__device__ __forceinline__ R stress_rate(R rho, R s_const, const Phys<R>& p) {
  if (p.visc_mode == VISC_CONST) return s_const;
  R tau;
  if (p.visc_mode == VISC_STEP) {
    tau = rho >= p.rho_c ? p.tau_l : p.tau_v;
  } else {
    R fr = (rho - p.rho_v) * p.inv_drho_lv;
    fr = fr < (R)0 ? (R)0 : (fr > (R)1 ? (R)1 : fr);
    tau = p.tau_v + fr * (p.tau_l - p.tau_v);
  }
  return recip(tau);
}

// ---------------------------------------------------------------------------------------
// Vector memory helpers.  VEC consecutive elements of type S, aligned to VEC*sizeof(S).
template <typename S, int VEC> struct VecT;
template <> struct VecT<float, 1> { typedef float T; };
template <> struct VecT<float, 2> { typedef float2 T; };
template <> struct VecT<float, 4> { typedef float4 T; };
template <> struct VecT<double, 1> { typedef double T; };
template <> struct VecT<double, 2> { typedef double2 T; };

template <typename S, int VEC>
__device__ __forceinline__ void vload(const S* __restrict__ p, S (&v)[VEC]) {
  typedef typename VecT<S, VEC>::T V;
  V t = __ldg(reinterpret_cast<const V*>(p));
  const S* e = reinterpret_cast<const S*>(&t);
#pragma unroll
  for (int k = 0; k < VEC; ++k) v[k] = e[k];
}
template <typename S, int VEC>
__device__ __forceinline__ void vstore(S* p, const S (&v)[VEC]) {
  typedef typename VecT<S, VEC>::T V;
  V t;
  S* e = reinterpret_cast<S*>(&t);
#pragma unroll
  for (int k = 0; k < VEC; ++k) e[k] = v[k];
  *reinterpret_cast<V*>(p) = t;
}

__device__ __forceinline__ int wrapi(int i, int n) {
  // Any integer to [0, n): cheap for the common one-period offsets.
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Context of one CTA sweeping one work item.
template <typename S, int VEC>
struct Sweep {
  const S* __restrict__ base;  // plane 0 of this instance, input buffer
  int nx, ny, pitch, walls;
  long long plane;
  int c0;       // first logical column of this thread
  bool fast;    // all VEC logical columns of this thread lie in [0, nx)
  int lane;

  // Pull the nine populations for the VEC nodes (logical columns c0..c0+VEC-1) of
  // physical row y (0 <= y < ny).  out[q][k] = buf_q(x - e_q) with periodic x, periodic or
  // bounce-back y.
  __device__ __forceinline__ void pull_row(int y, S (&out)[Q][VEC]) const {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int exq = ex_of(q), eyq = ey_of(q);
      int ys = y - eyq;
      int qs = q;
      bool bounce = false;
      if (eyq != 0) {
        if (ys < 0 || ys >= ny) {
          if (walls) {
            bounce = true;
            qs = opp_of(q);
            ys = y;
          } else {
            ys = ys < 0 ? ys + ny : ys - ny;
          }
        }
      }
      const S* row = base + (long long)qs * plane + (long long)ys * pitch;
      S v[VEC];
      if (fast) {
        vload<S, VEC>(row + c0, v);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = __ldg(row + wrapi(c0 + k, nx));
      }
      if (bounce || exq == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) out[q][k] = v[k];
      } else if (exq == 1) {
        // node column c needs column c - 1
        S left = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
        if (lane == 0) left = __ldg(row + wrapi(c0 - 1, nx));
        out[q][0] = left;
#pragma unroll
        for (int k = 1; k < VEC; ++k) out[q][k] = v[k - 1];
      } else {
        // node column c needs column c + 1
        S right = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (lane == 31) right = __ldg(row + wrapi(c0 + VEC, nx));
#pragma unroll
        for (int k = 0; k < VEC - 1; ++k) out[q][k] = v[k + 1];
        out[q][VEC - 1] = right;
      }
    }
  }
};

template <typename S, typename R, int VEC>
__device__ __forceinline__ void density_row(const S (&f)[Q][VEC], R rho_ref, R (&drho)[VEC],
                                            R (&rho)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; ++k) {
    R d = ((R)f[0][k] + ((R)f[1][k] + (R)f[3][k])) + (((R)f[2][k] + (R)f[4][k]) +
          (((R)f[5][k] + (R)f[7][k]) + ((R)f[6][k] + (R)f[8][k])));
    drho[k] = d;
    rho[k] = rho_ref + d;
  }
}

// Collision of one node in moment space (Eqs. 3, 4, 25), deviation form.
//   h: pulled deviation populations (in), post-collision deviations (out)
//   drho = sum h, rho = rho_ref + drho
//   fpx, fpy: F / psi(x) (Eq. 7 without the leading psi), psi_c = psi(x)
// The moments of h differ from those of f only in m0..m2 (by rho_ref (1, -2, 1)), so the
// equilibria of Eq. 3 enter as m_eq - rho_ref (1, -2, 1, 0, ...).  The update is applied as
// h* = h + M^{-1} dm with M^{-1} = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
// Conserved moments: dm0 = 0, and for j the relaxation cancels against half the force,
// leaving dm3 = F_x, dm5 = F_y exactly.  The sigma term of Eq. 25 times (1 - s/2) reduces to
// 12 sigma s |F/psi|^2 (because tau - 1/2 = (1 - s/2)/s).
template <typename R>
__device__ __forceinline__ void collide_node(R (&h)[Q], R drho, R rho, R psi_c, R fpx, R fpy,
                                             const Phys<R>& p, R& ux_out, R& uy_out) {
  const R Fx = psi_c * fpx, Fy = psi_c * fpy;
  const R jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
  const R jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
  const R ir = recip(rho);
  const R ux = (jx + (R)0.5 * Fx) * ir;
  const R uy = (jy + (R)0.5 * Fy) * ir;
  ux_out = ux;
  uy_out = uy;
  const R sa = (h[1] + h[3]) + (h[2] + h[4]);
  const R sd = (h[5] + h[7]) + (h[6] + h[8]);
  const R m1 = (R)2 * sd - sa - (R)4 * h[0];
  const R m2 = sd - (R)2 * sa + (R)4 * h[0];
  const R m4 = (R)-2 * (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
  const R m6 = (R)-2 * (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
  const R m7 = (h[1] + h[3]) - (h[2] + h[4]);
  const R m8 = (h[5] + h[7]) - (h[6] + h[8]);
  const R rux = rho * ux, ruy = rho * uy;
  const R ru2 = rux * ux + ruy * uy;
  const R e1 = (R)3 * ru2 - (R)2 * drho;
  const R e2 = drho - (R)3 * ru2;
  const R e7 = rux * ux - ruy * uy;
  const R e8 = rux * uy;
  const R vF = ux * Fx + uy * Fy;
  const R F2 = fpx * fpx + fpy * fpy;
  const R snu7 = stress_rate<R>(rho, p.s7, p);
  const R snu8 = p.visc_mode == VISC_CONST ? p.s8 : snu7;
  // dm_k = -s_k (m_k - meq_k) + (1 - s_k/2) S_k, S from Eq. 25.
  const R d1 = -p.s1 * (m1 - e1) + ((R)1 - (R)0.5 * p.s1) * ((R)6 * vF) + p.sig12_e * F2;
  const R d2 = -p.s2 * (m2 - e2) - ((R)1 - (R)0.5 * p.s2) * ((R)6 * vF) - p.sig12_z * F2;
  const R d4 = -p.s4 * (m4 + rux) - ((R)1 - (R)0.5 * p.s4) * Fx;
  const R d6 = -p.s6 * (m6 + ruy) - ((R)1 - (R)0.5 * p.s6) * Fy;
  const R d7 = -snu7 * (m7 - e7) + ((R)1 - (R)0.5 * snu7) * ((R)2 * (ux * Fx - uy * Fy));
  const R d8 = -snu8 * (m8 - e8) + ((R)1 - (R)0.5 * snu8) * (ux * Fy + uy * Fx);
  const R a1 = d1 * (R)(1.0 / 36.0), a2 = d2 * (R)(1.0 / 36.0);
  const R a3 = Fx * (R)(1.0 / 6.0), a5 = Fy * (R)(1.0 / 6.0);
  const R a4 = d4 * (R)(1.0 / 12.0), a6 = d6 * (R)(1.0 / 12.0);
  const R a7 = d7 * (R)0.25, a8 = d8 * (R)0.25;
  const R A = -a1 - (R)2 * a2;
  const R B = (R)2 * a1 + a2;
  const R Px = a3 - (R)2 * a4, Py = a5 - (R)2 * a6;
  const R X = a3 + a4, Y = a5 + a6;
  h[0] += (R)4 * (a2 - a1);
  h[1] += A + Px + a7;
  h[3] += A - Px + a7;
  h[2] += A + Py - a7;
  h[4] += A - Py - a7;
  h[5] += B + X + Y + a8;
  h[6] += B - X + Y - a8;
  h[7] += B - X - Y + a8;
  h[8] += B + X - Y - a8;
}

template <typename R>
__device__ __forceinline__ bool finite_(R v) { return isfinite(v); }

// ---------------------------------------------------------------------------------------
// The fused sweep kernel.  One CTA per work item; NT threads, VEC columns per thread.
// Threads 1..NT-2 own columns [x0, x0 + (NT-2) VEC); threads 0 and NT-1 hold the halo
// columns x0 - 1 and x0 + W (their psi is needed by the owned edge nodes).
template <typename S, int VEC, int MODE>
__global__ void __launch_bounds__(NT) sweep_kernel(const S* __restrict__ fin,
                                                   S* __restrict__ fout,
                                                   const InstParams* __restrict__ insts,
                                                   const WorkItem* __restrict__ items,
                                                   int n_items, MomArgs<S> mo,
                                                   int* __restrict__ status) {
  typedef S R;  // arithmetic type follows the storage type
  constexpr int W = (NT - 2) * VEC;
  __shared__ R psi_s[4][NT * VEC];
  __shared__ double red_d[NT / 32][3];
  __shared__ float red_f[NT / 32][2];
  __shared__ int red_i[NT / 32];

  if ((int)blockIdx.x >= n_items) return;
  const WorkItem it = items[blockIdx.x];
  const InstParams& P = insts[it.inst];
  const Phys<R> ph = load_phys<R>(P);
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  Sweep<S, VEC> sw;
  sw.nx = P.nx;
  sw.ny = P.ny;
  sw.pitch = P.pitch;
  sw.walls = P.walls;
  sw.plane = P.plane;
  sw.base = fin + P.off;
  sw.lane = lane;
  sw.c0 = it.x0 - VEC + tid * VEC;
  sw.fast = sw.c0 >= 0 && sw.c0 + VEC <= sw.nx;
  const int nx = sw.nx, ny = sw.ny;

  // Owned columns of this thread: logical columns in [x0, min(x0 + W, nx)).
  const int xend = min(it.x0 + W, nx);
  const bool owner = tid >= 1 && tid <= NT - 2 && sw.c0 < xend;
  const bool full_owner = owner && sw.c0 + VEC <= xend;
  const int sidx = tid * VEC;  // this thread's first slot in a psi row

  // Rows: psi is needed on rows y0-1 .. y1 (ghost rows mirror the wall row).
  const int y0 = it.y0, y1 = it.y1;
  const int dir = it.dir < 0 ? -1 : 1;
  const int r_first = dir > 0 ? y0 - 1 : y1;      // first psi row
  const int nrows = y1 - y0 + 2;

  auto phys_row = [&](int r) -> int {
    if (sw.walls) return r < 0 ? 0 : (r >= ny ? ny - 1 : r);
    return r < 0 ? r + ny : (r >= ny ? r - ny : r);
  };

  S cur[Q][VEC], nxt[Q][VEC];
  R cur_drho[VEC], cur_rho[VEC];
  double acc_m = 0.0, acc_x = 0.0, acc_y = 0.0;
  float mx_u = 0.f, mx_d = 0.f;
  int bad = 0;
  bool flag_bad = false;

  // Prologue: row r_first (psi only), then row r_first+dir (psi and kept as centre).
  sw.pull_row(phys_row(r_first), nxt);
  {
    R d[VEC], rr[VEC];
    density_row<S, R, VEC>(nxt, ph.rho_ref, d, rr);
#pragma unroll
    for (int k = 0; k < VEC; ++k) psi_s[r_first & 3][sidx + k] = psi_of<R>(rr[k], ph);
  }
  int r = r_first + dir;
  sw.pull_row(phys_row(r), cur);
  density_row<S, R, VEC>(cur, ph.rho_ref, cur_drho, cur_rho);
#pragma unroll
  for (int k = 0; k < VEC; ++k) psi_s[r & 3][sidx + k] = psi_of<R>(cur_rho[k], ph);
  r += dir;
  sw.pull_row(phys_row(r), nxt);

  for (int i = 2; i < nrows; ++i, r += dir) {
    // psi of row r from the populations loaded in the previous iteration.
    R nd[VEC], nr[VEC];
    density_row<S, R, VEC>(nxt, ph.rho_ref, nd, nr);
#pragma unroll
    for (int k = 0; k < VEC; ++k) psi_s[r & 3][sidx + k] = psi_of<R>(nr[k], ph);
    // Prefetch the populations of the next psi row while this row is collided.
    S pre[Q][VEC];
    const bool more = i + 1 < nrows;
    if (more) sw.pull_row(phys_row(r + dir), pre);
    __syncthreads();

    // Centre row rc = r - dir.
    const int rc = r - dir;
    const int yc = rc;  // always inside [0, ny) for centre rows
    const R* ps_m = psi_s[(rc - 1) & 3];
    const R* ps_0 = psi_s[rc & 3];
    const R* ps_p = psi_s[(rc + 1) & 3];
    if (owner) {
      R outv[Q][VEC];
      R uxv[VEC], uyv[VEC];
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        const int s0 = sidx + k;
        const R pE = ps_0[s0 + 1], pW = ps_0[s0 - 1];
        const R pN = ps_p[s0], pS = ps_m[s0];
        const R pNE = ps_p[s0 + 1], pNW = ps_p[s0 - 1];
        const R pSW = ps_m[s0 - 1], pSE = ps_m[s0 + 1];
        const R w1 = (R)(1.0 / 3.0), w2 = (R)(1.0 / 12.0);
        const R fpx = -ph.G * (w1 * (pE - pW) + w2 * ((pNE - pNW) + (pSE - pSW)));
        const R fpy = -ph.G * (w1 * (pN - pS) + w2 * ((pNE + pNW) - (pSE + pSW)));
        const R pc = ps_0[s0];
        R h[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) h[q] = (R)cur[q][k];
        if (MODE == MODE_STEP) {
          R ux, uy;
          collide_node<R>(h, cur_drho[k], cur_rho[k], pc, fpx, fpy, ph, ux, uy);
#pragma unroll
          for (int q = 0; q < Q; ++q) outv[q][k] = h[q];
          if (!(cur_rho[k] > (R)0) || !finite_(cur_rho[k])) flag_bad = true;
        } else {
          const R Fx = pc * fpx, Fy = pc * fpy;
          const R jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
          const R jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
          const R px = jx + (R)0.5 * Fx, py = jy + (R)0.5 * Fy;
          const R ir = (R)1 / cur_rho[k];
          uxv[k] = px * ir;
          uyv[k] = py * ir;
          if (mo.flags & MOM_DIAG) {
            const int col = sw.c0 + k;
            if (col < xend) {
              const R rh = cur_rho[k];
              const bool fin_ok = finite_(rh) && finite_(uxv[k]) && finite_(uyv[k]);
              if (!fin_ok) {
                ++bad;
              } else {
                acc_m += (double)rh;
                acc_x += (double)px;
                acc_y += (double)py;
                const float u = (float)sqrt((double)(uxv[k] * uxv[k] + uyv[k] * uyv[k]));
                mx_u = fmaxf(mx_u, u);
                if (mo.rho_prev) {
                  const long long di = P.dense_off + (long long)yc * nx + col;
                  const float dd = (float)fabs((double)rh - (double)mo.rho_prev[di]);
                  mx_d = fmaxf(mx_d, dd);
                }
              }
            }
          }
        }
      }
      if (MODE == MODE_STEP) {
        S* dst = fout + P.off + (long long)yc * sw.pitch + sw.c0;
        if (full_owner) {
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            S v[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[k] = (S)outv[q][k];
            vstore<S, VEC>(dst + (long long)q * sw.plane, v);
          }
        } else {
#pragma unroll
          for (int k = 0; k < VEC; ++k)
            if (sw.c0 + k < xend) {
#pragma unroll
              for (int q = 0; q < Q; ++q) dst[(long long)q * sw.plane + k] = (S)outv[q][k];
            }
        }
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          const int col = sw.c0 + k;
          if (col < xend) {
            const long long di = P.dense_off + (long long)yc * nx + col;
            if (mo.flags & MOM_FIELDS) {
              if (mo.rho) mo.rho[di] = (S)cur_rho[k];
              if (mo.ux) mo.ux[di] = (S)uxv[k];
              if (mo.uy) mo.uy[di] = (S)uyv[k];
            }
            if ((mo.flags & MOM_UPDATE_PREV) && mo.rho_prev) mo.rho_prev[di] = (S)cur_rho[k];
          }
        }
      }
    }
    // Rotate: the row whose psi was just computed becomes the centre row.
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int k = 0; k < VEC; ++k) cur[q][k] = nxt[q][k];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      cur_drho[k] = nd[k];
      cur_rho[k] = nr[k];
    }
    if (more) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k = 0; k < VEC; ++k) nxt[q][k] = pre[q][k];
    }
  }

  if (MODE == MODE_STEP) {
    if (flag_bad) atomicOr(status, STATUS_NONFINITE);
  } else if (mo.flags & MOM_DIAG) {
    // Block reduction: warp shuffles, then one value per warp through shared memory.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_m += __shfl_down_sync(0xffffffffu, acc_m, o);
      acc_x += __shfl_down_sync(0xffffffffu, acc_x, o);
      acc_y += __shfl_down_sync(0xffffffffu, acc_y, o);
      mx_u = fmaxf(mx_u, __shfl_down_sync(0xffffffffu, mx_u, o));
      mx_d = fmaxf(mx_d, __shfl_down_sync(0xffffffffu, mx_d, o));
      bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    const int wid = tid >> 5;
    if (lane == 0) {
      red_d[wid][0] = acc_m;
      red_d[wid][1] = acc_x;
      red_d[wid][2] = acc_y;
      red_f[wid][0] = mx_u;
      red_f[wid][1] = mx_d;
      red_i[wid] = bad;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0, s1 = 0, s2 = 0;
      float f0 = 0.f, f1 = 0.f;
      int b = 0;
      for (int w = 0; w < NT / 32; ++w) {
        s0 += red_d[w][0];
        s1 += red_d[w][1];
        s2 += red_d[w][2];
        f0 = fmaxf(f0, red_f[w][0]);
        f1 = fmaxf(f1, red_f[w][1]);
        b += red_i[w];
      }
      mo.part_sum[3 * blockIdx.x + 0] = s0;
      mo.part_sum[3 * blockIdx.x + 1] = s1;
      mo.part_sum[3 * blockIdx.x + 2] = s2;
      mo.part_max[2 * blockIdx.x + 0] = f0;
      mo.part_max[2 * blockIdx.x + 1] = f1;
      mo.part_bad[blockIdx.x] = b;
    }
  }
}

}  // namespace lbm
