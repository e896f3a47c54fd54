// Device side of the D2Q9 MRT pseudopotential step (Li, Luo & Li, arXiv:1211.6932).
//
// One fused kernel per time step.  A CTA owns a strip of NT columns (one column per
// thread) and a chunk of rows of one lattice instance, and sweeps the chunk row by row:
//   - one elected thread streams the population rows of the strip (plus a 4-column halo
//     on each side) into an 8-row ring in shared memory with bulk asynchronous copies
//     (cp.async.bulk, completion on an mbarrier per slot), up to six rows ahead;
//   - every thread pulls the nine populations of its node from the ring (Eq. 5, pull
//     form), sums them to rho (Eq. 6) and evaluates psi (Eqs. 24, 30) into a four-row
//     psi ring, keeping the pulled values in registers;
//   - one row behind, it forms F from the 3x3 psi stencil (Eq. 7), v (Eq. 6) and the MRT
//     collision with the improved forcing (Eqs. 3, 4, 25), and stores the post-collision
//     populations at the node itself.
// psi of halo rows and columns is recomputed from the populations, so every population
// value is read from DRAM once per step and written once: 72 B per lattice update (FP32).
//
// Storage: structure of arrays.  Plane q of instance P holds row y at
//   base + P.off + q*P.plane + y*P.pitch + GHOST + x,    x in [-GHOST, pitch - GHOST),
// i.e. every row carries GHOST columns on each side.  Columns -2, -1, nx, nx+1 are kept
// equal to columns nx-2, nx-1, 0, 1 (periodic x), so the halo of any strip is one
// contiguous, 16-byte aligned copy whatever nx is.  The stored value is the
// post-collision population of the previous step minus t_q rho_ref (deviation storage;
// rho_ref = 0 gives plain storage): the population at node x and the current time is
// buf_q(x - e_q) + t_q rho_ref.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 9;
constexpr int GHOST = 8;     // storage columns kept on each side of a row (32 B in FP32)
constexpr int SEG_HALO = 4;  // shared-memory row segment starts 4 columns left of a strip
constexpr int NSLOT = 8;     // population rows in the shared-memory ring (power of 2)
constexpr int PSI_ROWS = 4;  // psi rows in the psi ring (power of 2)
constexpr long long WAIT_LIMIT = 1LL << 26;  // bounded mbarrier polls before giving up

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
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

// Parameters of one lattice instance (host fills, kernels read).
struct InstParams {
  int nx, ny;
  int pitch;           // row stride in elements: a multiple of 8, >= nx + 2 GHOST
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

// One CTA's share of the work: columns [x0, x0 + NT) and rows [y0, y1) of instance inst.
// dir = +1 sweeps upwards, -1 downwards.  Alternating the direction between neighbouring
// chunks makes the two CTAs that share halo rows read them at about the same time, so
// the second read hits L2.
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

// Reciprocal and square root.  FP32 uses the hardware approximations (a couple of ulps);
// FP64 keeps IEEE division and sqrt.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float recip(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ float sqrt_pos(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }
__device__ __forceinline__ double sqrt_pos(double a) { return a > 0.0 ? sqrt(a) : 0.0; }

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
  return sqrt_pos(p.two_over_G * rho * brk);
}
__device__ __forceinline__ double psi_eval_f64(double rho, double b4, double RT, double a,
                                               double two_over_G) {
  double x = b4 * rho;
  double num = 1.0 + x * (1.0 + x * (1.0 - x));
  double omx = 1.0 - x;
  double z = num / (omx * omx * omx);
  double arg = two_over_G * rho * (RT * z - a * rho - (1.0 / 3.0));
  return arg > 0.0 ? sqrt(arg) : 0.0;
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

__device__ __forceinline__ int wrapi(int i, int n) {
  // Any integer to [0, n): cheap for the common one-period offsets.
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------------------
// Bulk asynchronous copies and mbarriers (inline PTX, sm_90 and later).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the completion of phase `parity` of bar; false after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---------------------------------------------------------------------------------------
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
                                             const Phys<R>& p) {
  const R Fx = psi_c * fpx, Fy = psi_c * fpy;
  const R jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
  const R jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
  const R ir = recip(rho);
  const R ux = (jx + (R)0.5 * Fx) * ir;
  const R uy = (jy + (R)0.5 * Fy) * ir;
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

// Shared-memory layout of the sweep kernel (dynamic), in bytes.
template <typename S, int NT>
struct SweepSmem {
  static constexpr int SEG = NT + 2 * SEG_HALO;                    // columns per ring row
  static constexpr size_t BARS = 128;                              // NSLOT mbarriers
  static constexpr size_t POP = (size_t)NSLOT * Q * SEG * sizeof(S);
  static constexpr size_t PSI = (size_t)PSI_ROWS * (NT + 2) * sizeof(S);
  static constexpr size_t BYTES = BARS + POP + PSI;
};

// ---------------------------------------------------------------------------------------
// The fused sweep kernel.  One CTA per work item, NT threads, thread t owns column x0 + t.
// Threads 0 and 1 also evaluate psi of the halo columns x0 - 1 and x0 + NT.
template <typename S, int NT, int MODE>
__global__ void __launch_bounds__(NT) sweep_kernel(const S* __restrict__ fin,
                                                   S* __restrict__ fout,
                                                   const InstParams* __restrict__ insts,
                                                   const WorkItem* __restrict__ items,
                                                   int n_items, MomArgs<S> mo,
                                                   int* __restrict__ status) {
  typedef S R;  // arithmetic type follows the storage type
  typedef SweepSmem<S, NT> L;
  constexpr int SEG = L::SEG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  S* ring = reinterpret_cast<S*>(smem_raw + L::BARS);
  R* psis = reinterpret_cast<R*>(smem_raw + L::BARS + L::POP);
  __shared__ int s_abort;
  __shared__ double red_d[NT / 32][3];
  __shared__ float red_f[NT / 32][2];
  __shared__ int red_i[NT / 32];

  if ((int)blockIdx.x >= n_items) return;
  const WorkItem it = items[blockIdx.x];
  const InstParams& P = insts[it.inst];
  const Phys<R> ph = load_phys<R>(P);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int nx = P.nx, ny = P.ny, pitch = P.pitch, walls = P.walls;
  const long long plane = P.plane;
  const int x0 = it.x0;
  const int x = x0 + tid;
  const int xend = min(x0 + NT, nx);
  const bool owner = x < xend;
  const int dir = it.dir < 0 ? -1 : 1;
  const int y0 = it.y0, y1 = it.y1;
  const int nload = y1 - y0 + 4;              // population rows y0-2 .. y1+1
  const int rstart = dir > 0 ? y0 - 2 : y1 + 1;
  const int seg0 = GHOST + x0 - SEG_HALO;     // storage column of the ring's column 0
  const int len = min(SEG, pitch - seg0);     // elements per copied plane-row
  const uint32_t plane_bytes = (uint32_t)len * (uint32_t)sizeof(S);
  const S* gsrc = fin + P.off + seg0;

  // Physical row held by ring row j (walls: clamped, so every slot is filled uniformly;
  // the clamped copies are never pulled from because bounce-back replaces those reads).
  auto phys_load_row = [&](int j) -> int {
    const int r = rstart + j * dir;
    if (walls) return r < 0 ? 0 : (r >= ny ? ny - 1 : r);
    return wrapi(r, ny);
  };
  auto issue_row = [&](int j) {
    const int slot = j & (NSLOT - 1);
    const S* src = gsrc + (long long)phys_load_row(j) * pitch;
    mbar_arrive_expect_tx(&bars[slot], plane_bytes * Q);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      bulk_g2s(ring + ((size_t)slot * Q + q) * SEG, src + (long long)q * plane, plane_bytes,
               &bars[slot]);
  };

  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  int issued = 0;  // meaningful in thread 0 only
  if (tid == 0) {
    const int n0 = min(nload, NSLOT);
    for (int j = 0; j < n0; ++j) issue_row(j);
    issued = n0;
  }

  S cur[Q], nxt[Q];
  R cur_drho = 0, cur_rho = 1;
  bool flag_bad = false;
  double acc_m = 0.0, acc_x = 0.0, acc_y = 0.0;
  float mx_u = 0.f, mx_d = 0.f;
  int bad = 0;
  int waited = 0;  // ring rows waited for so far (all threads)

  for (int s = 1; s <= nload - 2; ++s) {
    // Refill the slot freed by row s-2 (all threads left it at the previous barrier).
    if (tid == 0 && s >= 2 && issued < nload) {
      fence_proxy_async_smem();
      issue_row(issued);
      ++issued;
    }
    // Rows s-1, s, s+1 must be resident.
    while (waited <= s + 1) {
      if (!mbar_wait_bounded(&bars[waited & (NSLOT - 1)], (uint32_t)((waited / NSLOT) & 1)))
        s_abort = 1;
      ++waited;
    }
    const int rpsi = rstart + s * dir;  // psi row of this iteration
    const bool ghost = walls && (rpsi < 0 || rpsi >= ny);
    R* ps_now = psis + (s & (PSI_ROWS - 1)) * (NT + 2);
    R nrho = 1, ndrho = 0;
    if (!ghost) {
      const int rp = walls ? rpsi : wrapi(rpsi, ny);
      const bool bb_low = walls && rp == 0;          // e_y = +1 would come from row -1
      const bool bb_high = walls && rp == ny - 1;    // e_y = -1 would come from row ny
      // Pull for columns c (CTA-relative): own column, and the halo columns for t < 2.
      auto pull = [&](int c, S (&v)[Q]) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int eyq = ey_of(q), exq = ex_of(q);
          const bool bb = (eyq > 0 && bb_low) || (eyq < 0 && bb_high);
          const int j = bb ? s : s - eyq * dir;
          const int qs = bb ? opp_of(q) : q;
          const int col = SEG_HALO + c - (bb ? 0 : exq);
          v[q] = ring[((size_t)(j & (NSLOT - 1)) * Q + qs) * SEG + col];
        }
      };
      auto density = [&](const S (&v)[Q], R& d) {
        d = ((R)v[0] + ((R)v[1] + (R)v[3])) +
            (((R)v[2] + (R)v[4]) + (((R)v[5] + (R)v[7]) + ((R)v[6] + (R)v[8])));
        return ph.rho_ref + d;
      };
      pull(tid, nxt);
      nrho = density(nxt, ndrho);
      ps_now[1 + tid] = psi_of<R>(nrho, ph);
      if (tid < 2) {
        S hv[Q];
        const int c = tid == 0 ? -1 : NT;
        pull(c, hv);
        R hd;
        ps_now[1 + c] = psi_of<R>(density(hv, hd), ph);
      }
      if (walls && s == 2) {
        // The first psi row of a sweep that starts at a wall is the ghost row: it mirrors
        // the row just computed.
        const int rfirst = rstart + dir;
        if (rfirst < 0 || rfirst >= ny) {
          R* ps_g = psis + (1 & (PSI_ROWS - 1)) * (NT + 2);
          ps_g[1 + tid] = ps_now[1 + tid];
          if (tid < 2) ps_g[tid == 0 ? 0 : NT + 1] = ps_now[tid == 0 ? 0 : NT + 1];
        }
      }
    } else if (s > 1) {
      // Ghost row at the end of a sweep: mirror the previous (wall) row.
      const R* ps_prev = psis + ((s - 1) & (PSI_ROWS - 1)) * (NT + 2);
      ps_now[1 + tid] = ps_prev[1 + tid];
      if (tid < 2) ps_now[tid == 0 ? 0 : NT + 1] = ps_prev[tid == 0 ? 0 : NT + 1];
    }
    __syncthreads();
    if (s_abort) break;

    if (s >= 3) {
      // Centre row rc = rstart + (s-1) dir; psi rows rc - dir and rc + dir around it.
      const int yc = rstart + (s - 1) * dir;
      const R* ps_c = psis + ((s - 1) & (PSI_ROWS - 1)) * (NT + 2);
      const R* ps_a = psis + ((s - 2) & (PSI_ROWS - 1)) * (NT + 2);  // row yc - dir
      const R* ps_b = ps_now;                                         // row yc + dir
      const R* ps_n = dir > 0 ? ps_b : ps_a;  // north (y + 1)
      const R* ps_s = dir > 0 ? ps_a : ps_b;  // south (y - 1)
      if (owner) {
        const int c = 1 + tid;
        const R pE = ps_c[c + 1], pW = ps_c[c - 1];
        const R pN = ps_n[c], pS = ps_s[c];
        const R pNE = ps_n[c + 1], pNW = ps_n[c - 1];
        const R pSW = ps_s[c - 1], pSE = ps_s[c + 1];
        const R w1 = (R)(1.0 / 3.0), w2 = (R)(1.0 / 12.0);
        const R fpx = -ph.G * (w1 * (pE - pW) + w2 * ((pNE - pNW) + (pSE - pSW)));
        const R fpy = -ph.G * (w1 * (pN - pS) + w2 * ((pNE + pNW) - (pSE + pSW)));
        const R pc = ps_c[c];
        R h[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) h[q] = (R)cur[q];
        if (MODE == MODE_STEP) {
          collide_node<R>(h, cur_drho, cur_rho, pc, fpx, fpy, ph);
          if (!(cur_rho > (R)0) || !isfinite(cur_rho)) flag_bad = true;
          S* dst = fout + P.off + (long long)yc * pitch + GHOST;
#pragma unroll
          for (int q = 0; q < Q; ++q) dst[(long long)q * plane + x] = (S)h[q];
          if (x < 2 || x >= nx - 2) {
            // Keep the ghost columns -2, -1, nx, nx+1 equal to the columns they mirror.
            auto put = [&](int g) {
              if (wrapi(g, nx) == x) {
#pragma unroll
                for (int q = 0; q < Q; ++q) dst[(long long)q * plane + g] = (S)h[q];
              }
            };
            put(-2);
            put(-1);
            put(nx);
            put(nx + 1);
          }
        } else {
          const R Fx = pc * fpx, Fy = pc * fpy;
          const R jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
          const R jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
          const R px = jx + (R)0.5 * Fx, py = jy + (R)0.5 * Fy;
          const R ir = (R)1 / cur_rho;
          const R ux = px * ir, uy = py * ir;
          const long long di = P.dense_off + (long long)yc * nx + x;
          if (mo.flags & MOM_FIELDS) {
            if (mo.rho) mo.rho[di] = (S)cur_rho;
            if (mo.ux) mo.ux[di] = (S)ux;
            if (mo.uy) mo.uy[di] = (S)uy;
          }
          if (mo.flags & MOM_DIAG) {
            const bool ok = isfinite(cur_rho) && isfinite(ux) && isfinite(uy);
            if (!ok) {
              ++bad;
            } else {
              acc_m += (double)cur_rho;
              acc_x += (double)px;
              acc_y += (double)py;
              mx_u = fmaxf(mx_u, (float)sqrt((double)ux * ux + (double)uy * uy));
              if (mo.rho_prev)
                mx_d = fmaxf(mx_d, (float)fabs((double)cur_rho - (double)mo.rho_prev[di]));
            }
          }
          if ((mo.flags & MOM_UPDATE_PREV) && mo.rho_prev) mo.rho_prev[di] = (S)cur_rho;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    cur_drho = ndrho;
    cur_rho = nrho;
  }

  if (s_abort) {
    // A copy did not complete in time: wait (bounded) for the copies still in flight so
    // no write lands in shared memory after this CTA has exited, then report.
    if (tid == 0) {
      // The newest row issued into each slot: once its phase completed, every earlier
      // copy into that slot has too.
      for (int k = 0; k < NSLOT && k < issued; ++k) {
        const int j = issued - 1 - ((issued - 1 - k) & (NSLOT - 1));
        mbar_wait_bounded(&bars[k], (uint32_t)((j / NSLOT) & 1));
      }
      atomicOr(status, STATUS_TIMEOUT);
    }
    return;
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
