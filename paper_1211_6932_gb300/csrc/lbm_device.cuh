// Device side of the D2Q9 MRT pseudopotential step (Li, Luo & Li, arXiv:1211.6932).
//
// One fused kernel per time step.  A CTA owns a strip of NT*VEC columns (VEC adjacent
// columns per thread) and a chunk of rows of one lattice instance, and sweeps the chunk
// row by row:
//   - one elected thread streams the population rows of the strip (plus a 4-column halo
//     on each side) into a ring of NSLOT rows in shared memory with bulk asynchronous
//     copies (cp.async.bulk, completion on an mbarrier per slot), NSLOT-3 rows ahead;
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
constexpr int PSI_ROWS = 4;  // psi rows in the psi ring (power of 2)
constexpr int PSI_OFF = 2;   // psi ring column of CTA column 0 (keeps pairs 8-byte aligned)
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
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2, STATUS_BOUNDS = 4 };

// Index checks of the bounds-check build (-DLBM_BOUNDS_CHECK, a stand-in for a memory
// sanitizer): LBM_IN(ok) is ok, and a false ok sets STATUS_BOUNDS in the kernel's status
// word; the caller skips the access it guards.  In the normal build LBM_IN(ok) is true and
// the checks compile away.
#ifdef LBM_BOUNDS_CHECK
__device__ __forceinline__ bool lbm_in_bounds(bool ok, int* status) {
  if (!ok) atomicOr(status, STATUS_BOUNDS);
  return ok;
}
#define LBM_IN(ok) ::lbm::lbm_in_bounds((ok), status)
#else
#define LBM_IN(ok) true
#endif

// Physical parameters in the arithmetic type of a kernel, prepared on the host so the
// kernels convert nothing (double-to-float conversions run on the slow FP64 pipe).
template <typename R>
struct PhysParams {
  R b4, RT, a, two_over_G, G;           // Eqs. 24, 30 and 7
  R s1, s2, s4, s6, s7, s8;             // rates of Eq. 2 that are not conserved
  R c1, c2, c4, c6, c7, c8;             // 1 - s/2 for the same rates (Eq. 4)
  R sig12_e, sig12_z;                   // 12 sigma s_e, 12 sigma s_zeta (Eq. 25 reduced)
  R tau_l, tau_v, dtau, rho_c;          // viscosity modes; dtau = tau_l - tau_v
  R rho_v, inv_drho_lv;                 // linear mode: 1 / (rho_l - rho_v)
  R rho_ref;                            // deviation reference density
  // The same constants folded with the weights of Eq. 7 and the column norms of M^{-1},
  // as the step kernel uses them (see collide_t).
  R g1, g2;                             // -G/3, -G/12
  R k1s, k1v, k1f;                      // s1/36, c1/6, 12 sigma s1/36
  R k2s, k2v, k2f;                      // s2/36, c2/6, 12 sigma s2/36
  R k4s, k4f, k6s, k6f;                 // s4/12, c4/12, s6/12, c6/12
  R k7s, k7v, k8s, k8v;                 // s7/4, c7/2, s8/4, c8/4 (constant viscosity)
};

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
  PhysParams<float> pf;  // the above in float, for FP32 kernels
  PhysParams<double> pd; // and in double, for FP64 kernels
};

// One CTA's share of the work: columns [x0, x0 + NT*VEC) and rows [y0, y1) of instance
// inst.
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
struct Phys : PhysParams<R> {
  int visc_mode, psi_fp64;
  double b4d, RTd, ad, two_over_Gd;  // psi in double precision for FP32 storage
};

template <typename R>
__device__ __forceinline__ const PhysParams<R>& phys_params(const InstParams& P);
template <>
__device__ __forceinline__ const PhysParams<float>& phys_params<float>(const InstParams& P) {
  return P.pf;
}
template <>
__device__ __forceinline__ const PhysParams<double>& phys_params<double>(const InstParams& P) {
  return P.pd;
}

template <typename R>
__device__ __forceinline__ Phys<R> load_phys(const InstParams& P) {
  Phys<R> p;
  static_cast<PhysParams<R>&>(p) = phys_params<R>(P);
  p.visc_mode = P.visc_mode;
  p.psi_fp64 = P.psi_fp64;
  p.b4d = P.b4; p.RTd = P.RT; p.ad = P.a; p.two_over_Gd = P.two_over_G;
  return p;
}

// psi of Eq. 24 with the Carnahan-Starling pressure of Eq. 30 in double precision, for
// the option of evaluating psi in FP64 under FP32 storage (see psi_t for the form).
__device__ __forceinline__ double psi_eval_f64(double rho, double b4, double RT, double a,
                                               double two_over_G) {
  double x = b4 * rho;
  double num = 1.0 + x * (1.0 + x * (1.0 - x));
  double omx = 1.0 - x;
  double z = num / (omx * omx * omx);
  double arg = two_over_G * rho * (RT * z - a * rho - (1.0 / 3.0));
  return arg > 0.0 ? sqrt(arg) : 0.0;
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
// Wait for the completion of phase `parity` of bar; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;  // the common case: the phase has completed
  const int n = limit < (1LL << 30) ? (int)limit : (1 << 30);  // a 32-bit loop counter
  for (int i = 1; i < n; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The step kernels' wait: false after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  return mbar_wait_polls(bar, parity, WAIT_LIMIT);
}

// Compensated (Kahan) running sum: per-thread diagnostics sums stay accurate to the last
// bits of the storage type without per-node double-precision arithmetic.
template <typename R>
struct CompSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------------------------------------------
// Arithmetic used by the collision, written once for three number types: float and
// double (one node per value) and float2 (two nodes per value, Blackwell's packed FP32
// instructions: one FFMA2/FADD2/FMUL2 does the work of two scalar instructions).
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

template <typename T> struct Num;
// FP32 quotient and square root for psi (Eq. 24 with Eq. 30): the hardware approximations
// (MUFU reciprocal and reciprocal square root) refined by one Newton-Raphson step each,
// with the residual correction of Markstein.  The bare approximations are a few ulps off
// with a consistent sign; psi enters the force of Eq. 7 as differences of neighbours, and
// over 10^4 steps that bias moves interfaces measurably against FP64.  Refined, the
// results are within about one ulp.  The collision keeps the bare reciprocal (1/rho and
// 1/tau): refining those as well did not lower the long-run error (maximum relative
// density error of the 1024^2 ellipse after 20000 steps: 8.8e-5 with, 6.3e-5 without).
//   a/b:    r = ~1/b, r' = r + r (1 - b r), q = a r', q' = q + r' (a - b q)
//   sqrt a: y = ~1/sqrt(a), s = a y, s' = s + (y/2) (a - s^2)
__device__ __forceinline__ float div_nr(float a, float b) {
  const float r0 = __fdividef(1.0f, b);
  const float r = fmaf(r0, fmaf(-b, r0, 1.0f), r0);
  const float q = a * r;
  return fmaf(r, fmaf(-b, q, a), q);
}
__device__ __forceinline__ float sqrt_nr(float a) {  // a > 0
  const float y = rsqrtf(a);
  const float s = a * y;
  return fmaf(0.5f * y, fmaf(-s, s, a), s);
}

template <> struct Num<float> {
  typedef float S;
  static __device__ __forceinline__ float k(float v) { return v; }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
  static __device__ __forceinline__ float div(float a, float b) { return div_nr(a, b); }
  static __device__ __forceinline__ float sqrtp(float a) { return a > 0.f ? sqrt_nr(a) : 0.f; }
  static __device__ __forceinline__ float clamp01(float a) { return fminf(fmaxf(a, 0.f), 1.f); }
  static __device__ __forceinline__ float sel_ge(float a, float t, float x, float y) {
    return a >= t ? x : y;
  }
};
template <> struct Num<double> {
  typedef double S;
  static __device__ __forceinline__ double k(double v) { return v; }
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return ::fma(a, b, c);
  }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrtp(double a) { return a > 0.0 ? sqrt(a) : 0.0; }
  static __device__ __forceinline__ double clamp01(double a) { return fmin(fmax(a, 0.0), 1.0); }
  static __device__ __forceinline__ double sel_ge(double a, double t, double x, double y) {
    return a >= t ? x : y;
  }
};
template <> struct Num<float2> {
  typedef float S;
  static __device__ __forceinline__ float2 k(float v) { return make_float2(v, v); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
  static __device__ __forceinline__ float2 rcp(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
  }
  // div_nr and sqrt_nr on pairs (packed FFMA2 after the two scalar MUFU approximations)
  static __device__ __forceinline__ float2 div(float2 a, float2 b) {
    const float2 r0 = rcp(b);
    const float2 nb = make_float2(-b.x, -b.y);
    const float2 r = fma(r0, fma(nb, r0, k(1.f)), r0);
    const float2 q = a * r;
    return fma(r, fma(nb, q, a), q);
  }
  static __device__ __forceinline__ float2 sqrtp(float2 a) {
    const float2 y = make_float2(rsqrtf(a.x), rsqrtf(a.y));
    const float2 s = a * y;
    const float2 t = fma(k(0.5f) * y, fma(make_float2(-s.x, -s.y), s, a), s);
    return make_float2(a.x > 0.f ? t.x : 0.f, a.y > 0.f ? t.y : 0.f);
  }
  static __device__ __forceinline__ float2 clamp01(float2 a) {
    return make_float2(Num<float>::clamp01(a.x), Num<float>::clamp01(a.y));
  }
  static __device__ __forceinline__ float2 sel_ge(float2 a, float t, float x, float y) {
    return make_float2(a.x >= t ? x : y, a.y >= t ? x : y);
  }
};

// psi of Eq. 24 with the Carnahan-Starling pressure of Eq. 30, written in factored form
//   psi^2 = (2/G) * rho * (R T Z(x) - a rho - 1/3),  x = b rho / 4,
//   Z(x) = (1 + x + x^2 - x^3) / (1 - x)^3,
// which equals 2 (p_EOS - rho/3) / G.  Pulling rho out of the bracket leaves three terms
// of comparable size and no cancellation at vapour density.  Negative arguments clamp to 0.
template <typename T, typename R>
__device__ __forceinline__ T psi_t(T rho, const Phys<R>& p) {
  typedef Num<T> N;
  if constexpr (sizeof(R) == 4) {
    if (p.psi_fp64) {
      if constexpr (sizeof(T) == 8) {
        return make_float2((float)psi_eval_f64((double)rho.x, p.b4d, p.RTd, p.ad, p.two_over_Gd),
                           (float)psi_eval_f64((double)rho.y, p.b4d, p.RTd, p.ad, p.two_over_Gd));
      } else {
        return (T)psi_eval_f64((double)rho, p.b4d, p.RTd, p.ad, p.two_over_Gd);
      }
    }
  }
  const T x = N::k(p.b4) * rho;
  const T num = N::fma(x, N::fma(x, N::k(1) - x, N::k(1)), N::k(1));
  const T omx = N::k(1) - x;
  const T z = N::div(num, omx * omx * omx);
  const T brk = N::fma(N::k(p.RT), z, N::fma(N::k(-p.a), rho, N::k(-1.0 / 3.0)));
  return N::sqrtp(N::k(p.two_over_G) * rho * brk);
}

// Collision of one node (or a pair) in moment space, Eqs. 3, 4 and 25, deviation form.
//   h: pulled deviation populations (in), post-collision deviations (out)
//   drho = sum h, rho = rho_ref + drho
//   fpx, fpy: F / psi(x) (Eq. 7 without the leading psi), psi_c = psi(x)
// The moments of h differ from those of f only in m0..m2 (by rho_ref (1, -2, 1)), so the
// equilibria of Eq. 3 enter as m_eq - rho_ref (1, -2, 1, 0, ...).  The update is applied
// as h* = h + M^{-1} dm with M^{-1} = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4,
// 1/4); the column norms and the rates are folded into the per-instance constants
// PhysParams::k* (a_k = dm_k / |row k of M|^2).  Conserved moments: dm0 = 0, and for j
// the relaxation cancels against half the force, leaving dm3 = F_x, dm5 = F_y.  The sigma
// term of Eq. 25 times (1 - s/2) reduces to 12 sigma s |F/psi|^2 (tau - 1/2 = (1 - s/2)/s).
template <typename T, typename R>
__device__ __forceinline__ void collide_t(T (&h)[Q], T drho, T rho, T psi_c, T fpx, T fpy,
                                          const Phys<R>& p) {
  typedef Num<T> N;
  const T Fx = psi_c * fpx, Fy = psi_c * fpy;
  const T d13 = h[1] - h[3], d24 = h[2] - h[4];
  const T s13 = h[1] + h[3], s24 = h[2] + h[4];
  const T s57 = h[5] + h[7], s68 = h[6] + h[8];
  const T tx = (h[5] - h[6]) - (h[7] - h[8]);  // h5 - h6 - h7 + h8
  const T ty = (h[5] + h[6]) - (h[7] + h[8]);  // h5 + h6 - h7 - h8
  const T ir = N::rcp(rho);
  const T ux = N::fma(N::k(0.5), Fx, d13 + tx) * ir;
  const T uy = N::fma(N::k(0.5), Fy, d24 + ty) * ir;
  const T sa = s13 + s24, sd = s57 + s68;
  const T m1 = N::fma(N::k(-4), h[0], sd + (sd - sa));
  const T m2 = N::fma(N::k(4), h[0], sd - (sa + sa));
  const T m4 = N::fma(N::k(-2), d13, tx);
  const T m6 = N::fma(N::k(-2), d24, ty);
  const T m7 = s13 - s24;
  const T m8 = s57 - s68;
  const T rux = rho * ux, ruy = rho * uy;
  const T ru2 = N::fma(rux, ux, ruy * uy);
  const T e1 = N::fma(N::k(3), ru2, N::k(-2) * drho);
  const T e2 = N::fma(N::k(-3), ru2, drho);
  const T e7 = N::fma(rux, ux, N::k(0) - ruy * uy);
  const T e8 = rux * uy;
  const T vF = N::fma(ux, Fx, uy * Fy);
  const T F2 = N::fma(fpx, fpx, fpy * fpy);
  const T wxy = N::fma(ux, Fx, N::k(0) - uy * Fy), vxy = N::fma(ux, Fy, uy * Fx);
  T k7s, k7v, k8s, k8v;
  if (p.visc_mode == VISC_CONST) {
    k7s = N::k(p.k7s);
    k7v = N::k(p.k7v);
    k8s = N::k(p.k8s);
    k8v = N::k(p.k8v);
  } else {
    T tau;
    if (p.visc_mode == VISC_STEP) {
      tau = N::sel_ge(rho, p.rho_c, p.tau_l, p.tau_v);
    } else {
      const T fr = N::clamp01((rho - N::k(p.rho_v)) * N::k(p.inv_drho_lv));
      tau = N::fma(fr, N::k(p.dtau), N::k(p.tau_v));
    }
    k7s = N::k(0.25) * N::rcp(tau);  // s_nu / 4 with s_nu = 1 / tau (Eq. 10)
    k7v = N::k(0.5) - k7s;           // (1 - s_nu / 2) / 2
    k8s = k7s;
    k8v = N::k(0.5) * k7v;
  }
  const T a1 = N::fma(N::k(-p.k1s), m1 - e1, N::fma(N::k(p.k1v), vF, N::k(p.k1f) * F2));
  const T a2 = N::fma(N::k(-p.k2s), m2 - e2, N::fma(N::k(-p.k2v), vF, N::k(-p.k2f) * F2));
  const T a3 = N::k(1.0 / 6.0) * Fx, a5 = N::k(1.0 / 6.0) * Fy;
  const T a4 = N::fma(N::k(-p.k4s), m4 + rux, N::k(-p.k4f) * Fx);
  const T a6 = N::fma(N::k(-p.k6s), m6 + ruy, N::k(-p.k6f) * Fy);
  const T a7 = N::fma(N::k(0) - k7s, m7 - e7, k7v * wxy);
  const T a8 = N::fma(N::k(0) - k8s, m8 - e8, k8v * vxy);
  const T A = N::fma(N::k(-2), a2, N::k(0) - a1), B = N::fma(N::k(2), a1, a2);
  const T Px = N::fma(N::k(-2), a4, a3), Py = N::fma(N::k(-2), a6, a5);
  const T X = a3 + a4, Y = a5 + a6;
  const T XpY = X + Y, XmY = X - Y;
  const T Ap = A + a7, Am = A - a7, Bp = B + a8, Bm = B - a8;
  h[0] = N::fma(N::k(4), a2 - a1, h[0]);
  h[1] = h[1] + (Ap + Px);
  h[3] = h[3] + (Ap - Px);
  h[2] = h[2] + (Am + Py);
  h[4] = h[4] + (Am - Py);
  h[5] = h[5] + (Bp + XpY);
  h[7] = h[7] + (Bp - XpY);
  h[6] = h[6] + (Bm - XmY);
  h[8] = h[8] + (Bm + XmY);
}

// Force of Eq. 7 divided by psi(x) from the 3x3 psi stencil (c centre, n north = y + 1,
// s south = y - 1; E, W = x +- 1), with g1 = -G/3 and g2 = -G/12.
template <typename T, typename R>
__device__ __forceinline__ void force_t(T pE, T pW, T pN, T pS, T pNE, T pNW, T pSE, T pSW,
                                        const Phys<R>& p, T& fpx, T& fpy) {
  typedef Num<T> N;
  fpx = N::fma(N::k(p.g1), pE - pW, N::k(p.g2) * ((pNE - pNW) + (pSE - pSW)));
  fpy = N::fma(N::k(p.g1), pN - pS, N::k(p.g2) * ((pNE + pNW) - (pSE + pSW)));
}

// Bulk asynchronous store shared -> global and its completion tracking.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Configuration and shared-memory layout (dynamic, bytes) of one sweep instantiation.
// Thread t handles CTA column c = t - 2: threads 1 and NT-2 evaluate psi of the halo
// columns -1 and WO, threads 2 .. NT-3 own the WO = NT - 4 columns of the strip, thread 0
// issues the bulk copies.
template <typename S, int NT>
struct SweepCfg {
  static constexpr int WO = NT - 4;          // owned columns per CTA (a multiple of 4)
  static constexpr int SEG = NT + 4;         // ring row: columns x0-4 .. x0+WO+3
  static constexpr int NSLOT = 8;            // ring rows (NSLOT - 3 rows in flight)
  static constexpr size_t BARS = 128;        // mbarriers
  static constexpr size_t POP = (size_t)NSLOT * Q * SEG * sizeof(S);
  static constexpr size_t PSI = (size_t)PSI_ROWS * NT * sizeof(S);
  static constexpr size_t OUT = (size_t)2 * Q * NT * sizeof(S);  // two staged output rows
  static constexpr size_t BYTES = BARS + POP + PSI + OUT;
};

// FP32 instantiations are held to 128 registers per thread so that enough CTAs stay
// resident; FP64 (a correctness mode) is left unconstrained.
template <typename S, int NT>
struct MinBlocks {
  static constexpr int value = sizeof(S) == 4 ? (65536 / (NT * 128)) : 1;
};

// ---------------------------------------------------------------------------------------
// The fused sweep kernel.  One CTA per work item (a strip of WO columns and a chunk of
// rows).  MODE_STEP writes the post-collision populations (staged in shared memory, one
// bulk store per plane and row); MODE_MOMENTS writes rho, v and/or reduces diagnostics.
template <typename S, int NT, int MODE>
__global__ void __launch_bounds__(NT, MinBlocks<S, NT>::value) sweep_kernel(
    const S* __restrict__ fin, S* __restrict__ fout, const InstParams* __restrict__ insts,
    const WorkItem* __restrict__ items, int n_items, MomArgs<S> mo, int* __restrict__ status) {
  typedef S R;  // arithmetic type follows the storage type
  typedef SweepCfg<S, NT> C;
  constexpr int WO = C::WO, SEG = C::SEG, NS = C::NSLOT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  S* ring = reinterpret_cast<S*>(smem_raw + C::BARS);
  R* psis = reinterpret_cast<R*>(smem_raw + C::BARS + C::POP);
  S* outs = reinterpret_cast<S*>(smem_raw + C::BARS + C::POP + C::PSI);
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
  const bool issuer = tid == 0;
  const int nx = P.nx, ny = P.ny, pitch = P.pitch, walls = P.walls;
  const long long plane = P.plane;
  const int x0 = it.x0;
  const int c = tid - 2;                  // CTA column of this thread
  const int x = x0 + c;                   // its global column
  const int xend = min(x0 + WO, nx);
  const bool psi_thread = tid >= 1 && tid <= NT - 2;
  const bool owner = c >= 0 && c < WO && x < xend;
  const int n_bulk = ((xend - x0) / 4) * 4;  // columns written by the bulk store
  const int dir = it.dir < 0 ? -1 : 1;
  const int y0 = it.y0, y1 = it.y1;
  const int nload = y1 - y0 + 4;          // population rows y0-2 .. y1+1
  const int rstart = dir > 0 ? y0 - 2 : y1 + 1;
  const int seg0 = GHOST + x0 - SEG_HALO; // storage column of ring column 0
  const int len = min(SEG, pitch - seg0); // elements per copied plane-row
  const uint32_t plane_bytes = (uint32_t)len * (uint32_t)sizeof(S);
  const S* gsrc = fin + P.off + seg0;

  // Ring row j holds physical row rstart + j*dir (walls: clamped, so every slot is filled
  // the same way; those clamped copies are never read because bounce-back replaces them).
  auto issue_row = [&](int j) {
    const int slot = j % NS;
    const int r = rstart + j * dir;
    const int rp = walls ? (r < 0 ? 0 : (r >= ny ? ny - 1 : r)) : wrapi(r, ny);
    const S* src = gsrc + (long long)rp * pitch;
    const bool ok = LBM_IN(rp >= 0 && rp < ny && seg0 >= 0 && len > 0 && len <= SEG &&
                           seg0 + len <= pitch);  // bounds-check build
    mbar_arrive_expect_tx(&bars[slot], ok ? plane_bytes * Q : 0u);
    if (!ok) return;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      bulk_g2s(ring + ((size_t)slot * Q + q) * SEG, src + (long long)q * plane, plane_bytes,
               &bars[slot]);
  };
  // Bulk store of the staged output row of centre row yc (out slot k).
  auto store_row = [&](int k, int yc) {
    if (n_bulk <= 0) return;
    if (!LBM_IN(yc >= 0 && yc < ny && x0 >= 0 && GHOST + x0 + n_bulk <= pitch)) return;
    S* dst = fout + P.off + (long long)yc * pitch + GHOST + x0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      bulk_s2g(dst + (long long)q * plane, outs + ((size_t)k * Q + q) * NT,
               (uint32_t)(n_bulk * sizeof(S)));
    bulk_commit();
  };

  int issued = 0;  // rows issued (meaningful in the issuing thread)
  if (issuer) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (issuer) {
    const int n0 = min(nload, NS);
    for (int j = 0; j < n0; ++j) issue_row(j);
    issued = n0;
  }

  S cur[Q], nxt[Q];
  R cur_rho = 1, cur_dr = 0;
  bool flag_bad = false;
  CompSum<R> acc_m, acc_x, acc_y;  // per-thread compensated sums (diagnostics)
  float mx_u = 0.f, mx_d = 0.f;    // max |v|^2, max |rho - rho_prev|
  int bad = 0;
  int waited = 0;  // ring rows waited for so far (same in every thread)
  const int last = nload - 2;
  int s = 1;
  for (; s <= last; ++s) {
    if (issuer) {
      if (s >= 2 && issued < nload) {
        fence_proxy_async_smem();  // our reads of the freed slot precede the new copy
        issue_row(issued);
        ++issued;
      }
      if (MODE == MODE_STEP) bulk_wait_read_all();  // the staged row about to be reused
    }
    while (waited <= s + 1) {  // rows s-1, s, s+1 must be resident
      if (!mbar_wait_bounded(&bars[waited % NS], (uint32_t)((waited / NS) & 1))) s_abort = 1;
      ++waited;
    }
    const int rpsi = rstart + s * dir;
    const bool ghost = walls && (rpsi < 0 || rpsi >= ny);
    R* ps_now = psis + (s & (PSI_ROWS - 1)) * NT;
    R nrho = 1, ndr = 0;
    if (!ghost) {
      if (psi_thread) {
        const bool bb_low = walls && rpsi == 0;        // e_y = +1 would come from row -1
        const bool bb_high = walls && rpsi == ny - 1;  // e_y = -1 would come from row ny
        const int j0 = s % NS, js = (s - dir) % NS, jn = (s + dir) % NS;
        const S* rowC = ring + (size_t)j0 * Q * SEG + SEG_HALO + c;
        const S* rowS = ring + (size_t)js * Q * SEG + SEG_HALO + c;  // row y - 1
        const S* rowN = ring + (size_t)jn * Q * SEG + SEG_HALO + c;  // row y + 1
        if (!(bb_low || bb_high)) {
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int eyq = ey_of(q);
            nxt[q] = (eyq > 0 ? rowS : (eyq < 0 ? rowN : rowC))[q * SEG - ex_of(q)];
          }
        } else {
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int eyq = ey_of(q);
            const bool bb = (eyq > 0 && bb_low) || (eyq < 0 && bb_high);
            nxt[q] = bb ? rowC[opp_of(q) * SEG]
                        : (eyq > 0 ? rowS : (eyq < 0 ? rowN : rowC))[q * SEG - ex_of(q)];
          }
        }
        ndr = ((R)nxt[0] + ((R)nxt[1] + (R)nxt[3])) +
              (((R)nxt[2] + (R)nxt[4]) + (((R)nxt[5] + (R)nxt[7]) + ((R)nxt[6] + (R)nxt[8])));
        nrho = ph.rho_ref + ndr;
        ps_now[tid] = psi_t<R, R>(nrho, ph);
        if (walls && s == 2) {
          // A sweep that starts at a wall begins with the ghost row: it mirrors this row.
          const int rfirst = rstart + dir;
          if (rfirst < 0 || rfirst >= ny) psis[(1 & (PSI_ROWS - 1)) * NT + tid] = ps_now[tid];
        }
      }
    } else if (s > 1 && psi_thread) {
      // Ghost row at the end of a sweep: mirror the previous (wall) row.
      ps_now[tid] = psis[((s - 1) & (PSI_ROWS - 1)) * NT + tid];
    }
    __syncthreads();
    if (s_abort) break;
    if (MODE == MODE_STEP && issuer && s >= 4)
      store_row((s - 1) & 1, rstart + (s - 2) * dir);  // staged in the previous iteration

    if (s >= 3 && owner) {
      // Collision of the centre row yc = rstart + (s-1) dir.
      const int yc = rstart + (s - 1) * dir;
      const R* pa = psis + ((s - 2) & (PSI_ROWS - 1)) * NT + tid;  // row yc - dir
      const R* pc = psis + ((s - 1) & (PSI_ROWS - 1)) * NT + tid;  // row yc
      const R* pb = ps_now + tid;                                   // row yc + dir
      const R* pn = dir > 0 ? pb : pa;   // north (y + 1)
      const R* pso = dir > 0 ? pa : pb;  // south (y - 1)
      const R pE = pc[1], pW = pc[-1], pN = pn[0], pS = pso[0];
      const R pNE = pn[1], pNW = pn[-1], pSW = pso[-1], pSE = pso[1];
      R fpx, fpy;
      force_t<R, R>(pE, pW, pN, pS, pNE, pNW, pSE, pSW, ph, fpx, fpy);
      R h[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) h[q] = (R)cur[q];
      if (MODE == MODE_STEP) {
        collide_t<R, R>(h, cur_dr, cur_rho, pc[0], fpx, fpy, ph);
        flag_bad |= !(cur_rho > (R)0 && cur_rho < (R)INFINITY);
        S* ost = outs + (size_t)(s & 1) * Q * NT + c;
#pragma unroll
        for (int q = 0; q < Q; ++q) ost[q * NT] = (S)h[q];
        fence_proxy_async_smem();  // the staged values are read by a bulk store
        if (c >= n_bulk || x < 2 || x >= nx - 2) {
          // Columns past the last full group of four, and the ghost copies -2, -1, nx,
          // nx+1 of the columns they mirror, are written directly.
          S* dst = fout + P.off + (long long)yc * pitch + GHOST;
          auto col_ok = [&](int col) {  // bounds-check build
            return LBM_IN(yc >= 0 && yc < ny && col >= -GHOST && col < pitch - GHOST);
          };
          if (c >= n_bulk && col_ok(x)) {
#pragma unroll
            for (int q = 0; q < Q; ++q) dst[(long long)q * plane + x] = (S)h[q];
          }
          auto put = [&](int g) {
            if (wrapi(g, nx) == x && col_ok(g)) {
#pragma unroll
              for (int q = 0; q < Q; ++q) dst[(long long)q * plane + g] = (S)h[q];
            }
          };
          if (x < 2 || x >= nx - 2) {
            put(-2);
            put(-1);
            put(nx);
            put(nx + 1);
          }
        }
      } else {
        const R Fx = pc[0] * fpx, Fy = pc[0] * fpy;
        const R jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
        const R jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
        const R px = jx + (R)0.5 * Fx, py = jy + (R)0.5 * Fy;
        const R ir = (R)1 / cur_rho;
        const R ux = px * ir, uy = py * ir;
        const long long di = P.dense_off + (long long)yc * nx + x;
        const bool di_ok = LBM_IN(yc >= 0 && yc < ny && x >= 0 && x < nx);
        if ((mo.flags & MOM_FIELDS) && di_ok) {
          if (mo.rho) mo.rho[di] = (S)cur_rho;
          if (mo.ux) mo.ux[di] = (S)ux;
          if (mo.uy) mo.uy[di] = (S)uy;
        }
        if ((mo.flags & MOM_DIAG) && di_ok) {
          if (!(isfinite(cur_rho) && isfinite(ux) && isfinite(uy))) {
            ++bad;
          } else {
            acc_m.add(cur_rho);
            acc_x.add(px);
            acc_y.add(py);
            mx_u = fmaxf(mx_u, (float)(ux * ux + uy * uy));
            if (mo.rho_prev) mx_d = fmaxf(mx_d, (float)fabs(cur_rho - mo.rho_prev[di]));
          }
        }
        if ((mo.flags & MOM_UPDATE_PREV) && mo.rho_prev && di_ok) mo.rho_prev[di] = (S)cur_rho;
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    cur_rho = nrho;
    cur_dr = ndr;
  }

  if (s <= last) {
    // A copy did not complete in time: wait (bounded) for the loads still in flight and
    // for the stores, so nothing touches shared memory after this CTA has exited.
    if (issuer) {
      for (int k = 0; k < NS && k < issued; ++k) {
        const int j = issued - 1 - ((issued - 1 - k) % NS);
        mbar_wait_bounded(&bars[k], (uint32_t)((j / NS) & 1));
      }
      if (MODE == MODE_STEP) bulk_wait_all();
      atomicOr(status, STATUS_TIMEOUT);
    }
    return;
  }
  if (MODE == MODE_STEP) {
    __syncthreads();  // the last staged row is complete
    if (issuer) {
      if (last >= 3) store_row(last & 1, rstart + (last - 1) * dir);
      bulk_wait_all();
    }
    if (flag_bad) atomicOr(status, STATUS_NONFINITE);
  } else if (mo.flags & MOM_DIAG) {
    // Block reduction in double: warp shuffles, then one value per warp through shared
    // memory.  max |v| is taken from the max of |v|^2.
    double sm = acc_m.value(), sx = acc_x.value(), sy = acc_y.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sm += __shfl_down_sync(0xffffffffu, sm, o);
      sx += __shfl_down_sync(0xffffffffu, sx, o);
      sy += __shfl_down_sync(0xffffffffu, sy, o);
      mx_u = fmaxf(mx_u, __shfl_down_sync(0xffffffffu, mx_u, o));
      mx_d = fmaxf(mx_d, __shfl_down_sync(0xffffffffu, mx_d, o));
      bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    const int wid = tid >> 5;
    if (lane == 0) {
      red_d[wid][0] = sm;
      red_d[wid][1] = sx;
      red_d[wid][2] = sy;
      red_f[wid][0] = sqrtf(mx_u);
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

// ---------------------------------------------------------------------------------------
// FP32 pair kernel: thread t handles the two adjacent CTA columns c0 = 2t - 2 and c0 + 1
// and does their arithmetic with packed float2 instructions.  Threads 1 .. NT-2 own the
// WO = 2 NT - 4 columns of the strip; threads 0 and NT-1 evaluate psi of the halo
// columns -1 and WO (their other column is unused); thread 0 issues the bulk copies.
// Owners write their post-collision pair straight from registers (one 8-byte store per
// population).
//
// Shared-memory ring by plane group.  A node of row y pulls the planes with e_y = -dir
// (three of them) from the row ahead in the sweep, the e_y = 0 planes from its own row and
// the e_y = +dir planes from the row behind, so each plane of a loaded row is read exactly
// once, one, two or three sweep steps after the row is needed first.  The three groups
// therefore live in rings of 3, 4 and 5 rows ("ahead", "centre", "behind"): 36 plane
// rows, as many as a ring of 4 whole rows, but with two rows in flight instead of one.
// Row j (in sweep order) is issued after the row barrier of step j - 3 and waited for at
// step j - 1; the ahead planes of row j are read at steps j - 1 (pull of row j - 1) and j
// (bounce-back at a wall row j), the centre planes at step j, the behind planes at steps
// j (bounce-back) and j + 1, so each slot is free again when the next row issued into it
// is issued (ring depth 3, 4, 5 and issue lead 3).  The ahead planes of row 0 are never
// read and not copied (their slot is row 3's).
__host__ __device__ constexpr int kidx_of(int q) {  // index of plane q inside its group
  return q == 0 || q == 2 || q == 4 ? 0 : (q == 1 || q == 5 || q == 7 ? 1 : 2);
}

template <int NT>
struct Sweep2Cfg {
  static constexpr int WO = 2 * NT - 4;      // owned columns per CTA (a multiple of 4)
  static constexpr int SEG = WO + 8;         // ring row: columns x0-4 .. x0+WO+3
  static constexpr int DA = 3, DC = 4, DB = 5;  // ring depths: ahead, centre, behind
  static constexpr int NBAR = 5;             // row barriers (rows issued and not retired)
  static constexpr int LEAD = 3;             // row j is issued at step j - LEAD
  static constexpr int PLANE_ROWS = 3 * (DA + DC + DB);
  static constexpr int PSW = 2 * NT + 4;     // psi ring row: CTA columns -2 .. 2 NT + 1
  static constexpr int PSW_STRIP = 2 * NT;   // rows of the strip instantiation: -2 .. WO+1
  static constexpr size_t BARS = 128;
  static constexpr size_t POP = (size_t)PLANE_ROWS * SEG * sizeof(float);
  static constexpr size_t PSI = (size_t)PSI_ROWS * PSW * sizeof(float);
  static constexpr size_t BYTES = BARS + POP + PSI;
};

// Resident CTAs per SM the pair kernel is compiled for (the register cap follows): shared
// memory allows 19 / 10 / 7 / 5 CTAs of 32 / 64 / 96 / 128 threads, and these targets are
// the largest that compile without spills (94-96 registers).
constexpr int sweep2_min_blocks(int nt) {
  return nt == 32 ? 20 : nt == 64 ? 10 : nt == 96 ? 6 : nt == 128 ? 5 : 65536 / (nt * 128);
}

// Work a pair-kernel item does besides its own: none for one item per CTA (sweep2_kernel);
// the persistent kernel's queue and dependency bookkeeping otherwise (PersistHook).  Lane 0
// of the CTA's last warp runs start() once the item's first row copies are issued (while
// every warp waits for those rows) and row(s) after the copy issue of sweep step s.
struct NoHook {
  __device__ __forceinline__ void start() {}
  __device__ __forceinline__ void row(int) {}
};

// One work item of the pair kernel (a strip of rows [y0, y1) of one instance), the body of
// sweep2_kernel and sweep2_persist_kernel.  FULL selects the full-width strip (1) or the
// strip (0) at compile time (its own instantiation, so that the strip-mode code keeps
// constant load offsets), or (2) per item: full-width if the instance's rows fit one strip
// (nx <= 2 NT), for a work list of both kinds in one kernel.
// Returns true if a bounded wait ran out: the CTA has then waited for its copies in flight
// and set STATUS_TIMEOUT.  `part` indexes the diagnostics partials (MODE_MOMENTS).
template <int NT, int MODE, int FULL, typename Hook>
__device__ __forceinline__ bool sweep2_item(const float* __restrict__ fin,
                                            float* __restrict__ fout, const InstParams& P,
                                            const WorkItem& it, const MomArgs<float>& mo,
                                            int* __restrict__ status, int part, Hook& hook) {
  typedef Sweep2Cfg<NT> C;
  typedef Num<float2> N;
  constexpr int WO = C::WO, SEG = C::SEG, NB = C::NBAR;
  constexpr int PSW = FULL == 0 ? C::PSW_STRIP : C::PSW;
  constexpr int DA = C::DA, DC = C::DC, DB = C::DB, RING = C::PLANE_ROWS * SEG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float* ring = reinterpret_cast<float*>(smem_raw + C::BARS);
  float* ringA = ring;                    // ahead planes, DA rows of 3 planes
  float* ringC = ring + 3 * DA * SEG;     // centre planes, DC rows
  float* ringB = ring + 3 * (DA + DC) * SEG;  // behind planes, DB rows
  float* psis = reinterpret_cast<float*>(smem_raw + C::BARS + C::POP);
  __shared__ int s_abort;
  __shared__ double red_d[NT / 32][3];
  __shared__ float red_f[NT / 32][2];
  __shared__ int red_i[NT / 32];

  const Phys<float> ph = load_phys<float>(P);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const bool issuer = tid == 0;
  const int nx = P.nx, ny = P.ny, pitch = P.pitch, walls = P.walls;
  const long long plane = P.plane;
  const int x0 = it.x0;
  // Full-width strip (nx <= 2 NT, one strip per row, x0 = 0): thread t owns columns 2t,
  // 2t + 1, the row is loaded from its first column, the periodic neighbours of the two
  // edge columns are read across the row in shared memory, and the ghost columns are
  // neither read nor written.  Otherwise threads 1 .. NT-2 own WO columns from x0 and
  // threads 0 and NT-1 evaluate psi of the halo columns.
  const bool full = FULL == 2 ? nx <= 2 * NT : FULL == 1;
  const int c0 = full ? 2 * tid : 2 * tid - 2;  // first CTA column of this thread
  const int xa = x0 + c0;                 // its global column (xa, xa + 1)
  const int xend = full ? nx : min(x0 + WO, nx);
  const bool owner = full ? xa < nx : (tid >= 1 && tid <= NT - 2 && xa < xend);
  // Columns the pull and the force read besides c0 (the pair's left neighbour, its second
  // column and right neighbour), wrapped across the row in a full-width strip: only the
  // first thread (left) and the last one or two (right) wrap.  For nx = 1 the second and
  // right columns are not wrapped onto the row; they only feed the unused second column.
  const int cL = c0 - 1 + (full && c0 == 0 ? nx : 0);
  const int cR1 = c0 + 1 - (full && c0 + 1 >= nx ? nx : 0);
  const int cR2 = c0 + 2 - (full && c0 + 2 >= nx ? nx : 0);
  // Ghost columns (periodic copies at -2, -1, nx, nx+1), kept current by strip-mode
  // sweeps.  For even nx >= 4 the owners of the pairs (0, 1) and (nx-2, nx-1) mirror them
  // as pairs to (nx, nx+1) and (-2, -1); every other case (odd nx, nx < 4) takes the
  // general per-column path.
  const bool ghost_pairs = (nx & 1) == 0 && nx >= 4;
  constexpr int NO_GHOST = -(1 << 30);
  const int gpair = full || !ghost_pairs ? NO_GHOST
                                         : xa == 0 ? nx : xa == nx - 2 ? -2 : NO_GHOST;
  const bool ghost_slow = !full && !ghost_pairs && (xa < 2 || xa + 1 >= nx - 2);
  const int dir = it.dir < 0 ? -1 : 1;
  const int y0 = it.y0, y1 = it.y1;
  const int nload = y1 - y0 + 4;
  const int rstart = dir > 0 ? y0 - 2 : y1 + 1;
  // copy of a plane row: storage columns [seg0, seg0 + len) into ring columns from dst0
  const int seg0 = full ? GHOST : GHOST + x0 - SEG_HALO;
  const int dst0 = full ? SEG_HALO : 0;
  const int len = full ? (nx + 3) & ~3 : min(SEG, pitch - seg0);
  const uint32_t plane_bytes = (uint32_t)len * (uint32_t)sizeof(float);
  const float* gsrc = fin + P.off + seg0;
  const float2 rho_ref2 = N::k(ph.rho_ref);
  // bounds-check build: this thread's psi pair, and an owner's psi neighbours
  const bool psi_ok = LBM_IN(2 + c0 >= 0 && 2 + c0 + 2 <= PSW);
  const bool psi_nb_ok =
      !owner || LBM_IN(2 + cL >= 0 && 2 + cL < PSW && 2 + cR1 < PSW && 2 + cR2 < PSW);

  // Row j of the sweep: the planes of each group into that group's ring (see Sweep2Cfg),
  // completion on row barrier j % NB.
  auto issue_row = [&](int j) {
    const int r = rstart + j * dir;
    const int rp = walls ? (r < 0 ? 0 : (r >= ny ? ny - 1 : r)) : wrapi(r, ny);
    const float* src = gsrc + (long long)rp * pitch;
    const bool ok = LBM_IN(rp >= 0 && rp < ny && seg0 >= 0 && len > 0 && dst0 + len <= SEG &&
                           seg0 + len <= pitch);
    const bool ahead = j >= 1;  // the ahead planes of row 0 are never read
    uint64_t* bar = &bars[j % NB];
    mbar_arrive_expect_tx(bar, ok ? plane_bytes * (ahead ? 9u : 6u) : 0u);
    if (!ok) return;
    float* dA = ringA + (j % DA) * 3 * SEG;
    float* dC = ringC + (j % DC) * 3 * SEG;
    float* dB = ringB + (j % DB) * 3 * SEG;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int g = ey_of(q);
      float* dst = g == 0 ? dC : ((g < 0) == (dir > 0) ? dA : dB);
      if (dst == dA && !ahead) continue;
      if (!LBM_IN(dst + kidx_of(q) * SEG >= ring && dst + (kidx_of(q) + 1) * SEG <= ring + RING))
        continue;
      bulk_g2s(dst + kidx_of(q) * SEG + dst0, src + (long long)q * plane, plane_bytes, bar);
    }
  };

  int issued = 0;  // rows issued (issuer only)
  if (issuer) {
    s_abort = 0;
    for (int k = 0; k < NB; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (issuer) {
    const int n0 = min(nload, C::LEAD + 1);
    fence_proxy_async_smem();  // reads of the slots by an earlier item precede the copies
    for (int j = 0; j < n0; ++j) issue_row(j);
    issued = n0;
  }
  if (tid == NT - 32) hook.start();

  float2 cur[Q], nxt[Q];
  float2 cur_rho = N::k(1.f), cur_dr = N::k(0.f);
  bool flag_bad = false;
  CompSum<float> acc_m, acc_x, acc_y;  // per-thread compensated sums (diagnostics)
  float mx_u = 0.f, mx_d = 0.f;        // max |v|^2, max |rho - rho_prev|
  int bad = 0;
  // Ring bookkeeping without division: the row barrier and phase of the next row to wait
  // for (rows are waited for in order, one per iteration after the first), and the ring
  // slots of the rows an iteration reads.
  int waited = 0, wslot = 0;
  uint32_t wphase = 0;
  int sa = 2 % DA, sc = 1 % DC, sb = 0;  // slots: ahead of row s+1, centre of row s, behind of row s-1
  const int last = nload - 2;
  int s = 1;
  for (; s <= last; ++s) {
    while (waited <= s + 1) {
      if (!mbar_wait_bounded(&bars[wslot], wphase)) s_abort = 1;
      ++waited;
      if (++wslot == NB) {
        wslot = 0;
        wphase ^= 1u;
      }
    }
    const int rpsi = rstart + s * dir;
    const bool ghost = walls && (rpsi < 0 || rpsi >= ny);
    float* ps_now = psis + (s & (PSI_ROWS - 1)) * PSW;
    float2 nrho = N::k(1.f), ndr = N::k(0.f);
    if (!ghost) {
      const bool bb_low = walls && rpsi == 0;
      const bool bb_high = walls && rpsi == ny - 1;
      // group bases of this pull: e_y = -1 planes (from y + 1), e_y = 0 (row y), e_y = +1
      // (from y - 1); ahead is y + dir
      const float* pA = ringA + sa * 3 * SEG + SEG_HALO;  // row s+1 (ring column of CTA column 0)
      const float* pC = ringC + sc * 3 * SEG + SEG_HALO;  // row s
      const float* pB = ringB + sb * 3 * SEG + SEG_HALO;  // row s-1
      const float* gm = dir > 0 ? pA : pB;
      const float* gp = dir > 0 ? pB : pA;
      auto in_ring = [&](const float* p) {  // bounds-check build
        return LBM_IN(p >= ring && p < ring + RING);
      };
      // plane row p: the pair of columns (c0, c0+1) shifted by -e_x (8-byte aligned load
      // when e_x = 0)
      auto pull = [&](const float* p, int exq) -> float2 {
        const float* a = p + (exq > 0 ? cL : (exq < 0 ? cR1 : c0));
        const float* b = p + (exq > 0 ? c0 : (exq < 0 ? cR2 : c0 + 1));
        if (!(in_ring(a) && in_ring(b))) return N::k(0.f);
        return exq == 0 ? *reinterpret_cast<const float2*>(a) : make_float2(*a, *b);
      };
      if (!(bb_low || bb_high)) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int eyq = ey_of(q);
          nxt[q] = pull((eyq < 0 ? gm : (eyq > 0 ? gp : pC)) + kidx_of(q) * SEG, ex_of(q));
        }
      } else {
        // Halfway bounce-back: a plane that would come from beyond the wall is the
        // opposite plane of this row; those are in the ahead or behind ring of row s.
        const float* sA = ringA + (s % DA) * 3 * SEG + SEG_HALO;
        const float* sB = ringB + (s % DB) * 3 * SEG + SEG_HALO;
        const float* cm = dir > 0 ? sA : sB;  // e_y = -1 planes of row s
        const float* cp = dir > 0 ? sB : sA;  // e_y = +1 planes of row s
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int eyq = ey_of(q);
          const bool bb = (eyq > 0 && bb_low) || (eyq < 0 && bb_high);
          if (bb) {
            const int o = opp_of(q);
            nxt[q] = pull((ey_of(o) < 0 ? cm : cp) + kidx_of(o) * SEG, 0);
          } else {
            nxt[q] = pull((eyq < 0 ? gm : (eyq > 0 ? gp : pC)) + kidx_of(q) * SEG, ex_of(q));
          }
        }
      }
      ndr = (nxt[0] + (nxt[1] + nxt[3])) + ((nxt[2] + nxt[4]) + ((nxt[5] + nxt[7]) + (nxt[6] + nxt[8])));
      nrho = rho_ref2 + ndr;
      if (psi_ok) {
        *reinterpret_cast<float2*>(ps_now + 2 + c0) = psi_t<float2, float>(nrho, ph);
        if (walls && s == 2) {
          const int rfirst = rstart + dir;
          if (rfirst < 0 || rfirst >= ny)
            *reinterpret_cast<float2*>(psis + (1 & (PSI_ROWS - 1)) * PSW + 2 + c0) =
                *reinterpret_cast<const float2*>(ps_now + 2 + c0);
        }
      }
    } else if (s > 1 && psi_ok) {
      *reinterpret_cast<float2*>(ps_now + 2 + c0) =
          *reinterpret_cast<const float2*>(psis + ((s - 1) & (PSI_ROWS - 1)) * PSW + 2 + c0);
    }
    __syncthreads();
    if (s_abort) break;
    if (issuer && s + C::LEAD < nload) {
      // the slots of row s + LEAD were last read before this row barrier
      fence_proxy_async_smem();  // our reads of the freed slots precede the new copies
      issue_row(s + C::LEAD);
      issued = s + C::LEAD + 1;
    }
    if (tid == NT - 32) hook.row(s);  // bookkeeping of the persistent kernel

    if (s >= 3 && owner && psi_nb_ok) {
      const int yc = rstart + (s - 1) * dir;
      const float* pa = psis + ((s - 2) & (PSI_ROWS - 1)) * PSW + 2;  // row yc - dir
      const float* pc = psis + ((s - 1) & (PSI_ROWS - 1)) * PSW + 2;  // row yc
      const float* pb = ps_now + 2;                                    // row yc + dir
      const float* pn = dir > 0 ? pb : pa;
      const float* pso = dir > 0 ? pa : pb;
      // psi at the columns left of, in and right of the pair (c0, c0+1) in the three rows.
      // The east neighbour of column c0 is column c0+1 except for the odd last column of
      // a full-width strip, whose neighbour is column 0.
      const bool wrap_e = cR1 != c0 + 1;
      const float2 cC = *reinterpret_cast<const float2*>(pc + c0);
      const float2 cN = *reinterpret_cast<const float2*>(pn + c0);
      const float2 cS = *reinterpret_cast<const float2*>(pso + c0);
      const float cWm = pc[cL], cEp = pc[cR2], nWm = pn[cL], nEp = pn[cR2], sWm = pso[cL],
                  sEp = pso[cR2];
      const float cE1 = wrap_e ? pc[cR1] : cC.y, nE1 = wrap_e ? pn[cR1] : cN.y,
                  sE1 = wrap_e ? pso[cR1] : cS.y;
      const float2 pE = make_float2(cE1, cEp), pW = make_float2(cWm, cC.x);
      const float2 pNE = make_float2(nE1, nEp), pNW = make_float2(nWm, cN.x);
      const float2 pSE = make_float2(sE1, sEp), pSW = make_float2(sWm, cS.x);
      float2 fpx, fpy;
      force_t<float2, float>(pE, pW, cN, cS, pNE, pNW, pSE, pSW, ph, fpx, fpy);
      float2 h[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) h[q] = cur[q];
      if (MODE == MODE_STEP) {
        collide_t<float2, float>(h, cur_dr, cur_rho, cC, fpx, fpy, ph);
        const bool ok0 = cur_rho.x > 0.f && cur_rho.x < INFINITY;
        const bool ok1 = cur_rho.y > 0.f && cur_rho.y < INFINITY;
        flag_bad |= !ok0 || (xa + 1 < xend && !ok1);
        float* dst = fout + P.off + (long long)yc * pitch + GHOST;
        // bounds-check build: a storage column c of row yc lies in [-GHOST, pitch - GHOST)
        auto col_ok = [&](int c, int n) {
          return LBM_IN(yc >= 0 && yc < ny && c >= -GHOST && c + n <= pitch - GHOST);
        };
        if (xa + 1 < xend && col_ok(xa, 2)) {
          // both columns from registers: xa is even, so the pair is 8-byte aligned
#pragma unroll
          for (int q = 0; q < Q; ++q)
            *reinterpret_cast<float2*>(dst + (long long)q * plane + xa) = h[q];
          if (gpair != NO_GHOST && col_ok(gpair, 2)) {
            // the mirrored pair starts at an even column too (nx even)
#pragma unroll
            for (int q = 0; q < Q; ++q)
              *reinterpret_cast<float2*>(dst + (long long)q * plane + gpair) = h[q];
          }
        }
        const bool tail = xa + 1 >= xend;
        if (tail || ghost_slow) {
          // The odd last column (not covered above), and the ghost copies -2, -1, nx,
          // nx+1 of the columns they mirror when they are not written as pairs, column by
          // column.
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int x = xa + k;
            if (x >= xend) continue;
            float v[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) v[q] = k == 0 ? h[q].x : h[q].y;
            if (tail && col_ok(x, 1)) {
#pragma unroll
              for (int q = 0; q < Q; ++q) dst[(long long)q * plane + x] = v[q];
            }
            if (!full && !ghost_pairs && (x < 2 || x >= nx - 2)) {
              auto put = [&](int g) {
                if (wrapi(g, nx) == x && col_ok(g, 1)) {
#pragma unroll
                  for (int q = 0; q < Q; ++q) dst[(long long)q * plane + g] = v[q];
                }
              };
              put(-2);
              put(-1);
              put(nx);
              put(nx + 1);
            }
          }
        }
      } else {
        const float2 Fx = cC * fpx, Fy = cC * fpy;
        const float2 jx = (h[1] - h[3]) + ((h[5] - h[6]) - (h[7] - h[8]));
        const float2 jy = (h[2] - h[4]) + ((h[5] + h[6]) - (h[7] + h[8]));
        const float2 px = N::fma(N::k(0.5f), Fx, jx), py = N::fma(N::k(0.5f), Fy, jy);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int x = xa + k;
          if (x >= xend || !LBM_IN(yc >= 0 && yc < ny && x >= 0 && x < nx)) continue;
          const float r = k == 0 ? cur_rho.x : cur_rho.y;
          const float mx = k == 0 ? px.x : px.y, my = k == 0 ? py.x : py.y;
          const float ux = mx / r, uy = my / r;
          const long long di = P.dense_off + (long long)yc * nx + x;
          if (mo.flags & MOM_FIELDS) {
            if (mo.rho) mo.rho[di] = r;
            if (mo.ux) mo.ux[di] = ux;
            if (mo.uy) mo.uy[di] = uy;
          }
          if (mo.flags & MOM_DIAG) {
            if (!(isfinite(r) && isfinite(ux) && isfinite(uy))) {
              ++bad;
            } else {
              acc_m.add(r);
              acc_x.add(mx);
              acc_y.add(my);
              mx_u = fmaxf(mx_u, ux * ux + uy * uy);
              if (mo.rho_prev) mx_d = fmaxf(mx_d, fabsf(r - mo.rho_prev[di]));
            }
          }
          if ((mo.flags & MOM_UPDATE_PREV) && mo.rho_prev) mo.rho_prev[di] = r;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    cur_rho = nrho;
    cur_dr = ndr;
    sa = sa + 1 == DA ? 0 : sa + 1;
    sc = sc + 1 == DC ? 0 : sc + 1;
    sb = sb + 1 == DB ? 0 : sb + 1;
  }

  if (s <= last) {
    if (issuer) {
      // The newest row issued into each slot: once its phase completed, every earlier
      // copy into that slot has too.
      for (int k = 0; k < NB && k < issued; ++k) {
        const int j = issued - 1 - ((issued - 1 - k) % NB);
        mbar_wait_bounded(&bars[k], (uint32_t)((j / NB) & 1));
      }
      atomicOr(status, STATUS_TIMEOUT);
    }
    return true;
  }
  if (MODE == MODE_STEP) {
    if (flag_bad) atomicOr(status, STATUS_NONFINITE);
  } else if (mo.flags & MOM_DIAG) {
    double sm = acc_m.value(), sx = acc_x.value(), sy = acc_y.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sm += __shfl_down_sync(0xffffffffu, sm, o);
      sx += __shfl_down_sync(0xffffffffu, sx, o);
      sy += __shfl_down_sync(0xffffffffu, sy, o);
      mx_u = fmaxf(mx_u, __shfl_down_sync(0xffffffffu, mx_u, o));
      mx_d = fmaxf(mx_d, __shfl_down_sync(0xffffffffu, mx_d, o));
      bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    const int wid = tid >> 5;
    if (lane == 0) {
      red_d[wid][0] = sm;
      red_d[wid][1] = sx;
      red_d[wid][2] = sy;
      red_f[wid][0] = sqrtf(mx_u);
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
      mo.part_sum[3 * part + 0] = s0;
      mo.part_sum[3 * part + 1] = s1;
      mo.part_sum[3 * part + 2] = s2;
      mo.part_max[2 * part + 0] = f0;
      mo.part_max[2 * part + 1] = f1;
      mo.part_bad[part] = b;
    }
  }
  return false;
}

// Pair kernel, one CTA per work item.  A CTA whose instance does not match the FULL
// instantiation returns at once (the moments pass launches both over one item list).
template <int NT, int MODE, bool FULL>
__global__ void __launch_bounds__(NT, sweep2_min_blocks(NT)) sweep2_kernel(
    const float* __restrict__ fin, float* __restrict__ fout, const InstParams* __restrict__ insts,
    const WorkItem* __restrict__ items, int n_items, MomArgs<float> mo,
    int* __restrict__ status) {
  if ((int)blockIdx.x >= n_items) return;
  const WorkItem it = items[blockIdx.x];
  const InstParams& P = insts[it.inst];
  // the step launches hold items of one kind only (the host groups them, strips_for)
  if (MODE == MODE_MOMENTS && (P.nx <= 2 * NT) != FULL) return;
  NoHook hook;
  sweep2_item<NT, MODE, FULL>(fin, fout, P, it, mo, status, (int)blockIdx.x, hook);
}

// Dependencies of a work item of the persistent kernel: its chunk (a chunk row of one
// instance: every strip of rows [y0, y1)), the strips of a chunk row of its instance, and
// up to four chunks, its own among them, whose previous step it waits for: the chunks
// whose rows it reads (its rows and the two beyond each end, wrapped, or clamped at walls)
// and the chunks that read its rows (whose previous-step reads its stores would overwrite).
// Unused dependency entries repeat a used one.
struct ItemLink {
  int chunk, strips, dep[4], pad0, pad1;
};

constexpr int DEP_WAIT_LIMIT = 1 << 24;  // polls (with a short sleep) before giving up

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void red_add_relaxed_gpu(int* p, int v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Whether every dependency chunk of ln has `need` completed strips (acquire loads, issued
// together).
__device__ __forceinline__ bool deps_met(const int* done, const ItemLink& ln, int need) {
  const int a = ld_acquire_gpu(done + ln.dep[0]), b = ld_acquire_gpu(done + ln.dep[1]);
  const int c = ld_acquire_gpu(done + ln.dep[2]), d = ld_acquire_gpu(done + ln.dep[3]);
  return min(min(a, b), min(c, d)) >= need;
}

// Wait until deps_met; false after `limit` rounds.
__device__ __forceinline__ bool wait_deps(const int* done, const ItemLink& ln, int need,
                                          int limit) {
  for (int polls = 0; !deps_met(done, ln, need); ++polls) {
    if (polls + 1 >= limit) return false;
    __nanosleep(64);
  }
  return true;
}

// Queue and dependency bookkeeping of the persistent kernel, done by lane 0 of the CTA's
// last warp inside an item so that its latencies overlap the item's rows: once the
// item's first row copies are issued, while every warp waits for those rows, it releases
// the previous item (its chunk counter is incremented; the CTA barrier at that item's end
// ordered every thread's stores before this thread's release fence) and takes the next
// item from the queue and reads its dependency link; after the copy issue of sweep step
// 4 it reads the next item's dependency counters.  If those already show the next
// item's dependencies met, the next item starts without waiting.  (Doing this on the
// issuing thread delayed warp 0, and with it every row barrier, by the fence and the queue
// atomic: 82.1 against 84.0 GLUPS on the 4096^2 field; taking two items ahead and
// reading everything at the start measured 86.4 against 87.6 at 32-row chunks, reading
// the link at step 2 instead of at the start 87.6 against 87.8; a second set of row
// barriers, so that the next item could be published before the end-of-item barrier and
// two of the three barriers per item dropped, 87.2 against 87.6.)  The
// state lives in shared memory, not in every thread's registers.
struct PersistState {
  ItemLink ln;   // the next item's dependency link once have_link
  int release;   // chunk of the finished item not yet released, or -1
  int next;      // the item taken for after the current one
  int have_link, dep_ok;
};

struct PersistHook {
  PersistState* st;
  int* queue;
  const ItemLink* links2;
  int* done;
  int n_items, total;
  __device__ __forceinline__ void release_done() {
    if (st->release >= 0) {
      fence_acq_rel_gpu();
      red_add_relaxed_gpu(done + st->release, 1);
      st->release = -1;
    }
  }
  __device__ __forceinline__ void start() {
    const int next = atomicAdd(queue, 1);
    release_done();  // its fence drains while the atomic is in flight
    st->next = next;
    st->have_link = st->dep_ok = 0;
    if (next < total && next >= n_items) {
      const int t = next / n_items;
      st->ln = links2[(t & 1) * n_items + (next - t * n_items)];
      st->have_link = 1;
    }
  }
  __device__ __forceinline__ void row(int s) {
    if (s != 4 || !st->have_link) return;
    st->dep_ok = deps_met(done, st->ln, st->ln.strips * (st->next / n_items));
  }
};

// Persistent pair kernel for `steps` time steps of one work list (STEP mode): the CTAs
// take work items in order from *queue, item q being step t = q / n_items, entry
// k = q - t n_items of that step's list (items2 and links2 hold the even steps' list, then
// the odd steps', which visits each instance's chunks starting from the middle, so that
// the first items of a step do not wait on the last ones of the step before).  Step t
// reads slab t & 1 and writes the other.  An item's copies start only once each
// dependency chunk has completed all strips of steps 0 .. t-1 (done[] counts completed
// strips per chunk; acquire loads, then a proxy fence before the bulk reads); a finished
// item is released (a CTA barrier, then a release fence and an increment by thread 0) at
// the latest before its CTA waits for anything.  A CTA takes its next item from the queue
// while it works on the current one (PersistHook).  An item waits only on items earlier
// in the queue: the earliest unfinished item is some CTA's current one (a CTA's next item
// comes after its current one), its dependencies are finished and released, so every
// wait ends unless a CTA gives up; a CTA that gives up sets STATUS_TIMEOUT and returns,
// and the CTAs waiting on it give up in turn.  dep_limit bounds each dependency wait
// (DEP_WAIT_LIMIT; a failure-detection self-test passes a short one).  KIND selects the
// item body: PERSIST_STRIP or PERSIST_FULL for a group of one kind of strip, PERSIST_MIXED
// for a list holding both kinds (a batch of narrow and wide instances, one queue), where
// each item takes the full-width body if its instance's rows fit one strip (nx <= 2 NT).
constexpr int PERSIST_STRIP = 0, PERSIST_FULL = 1, PERSIST_MIXED = 2;

template <int NT, int KIND>
__global__ void __launch_bounds__(NT, sweep2_min_blocks(NT)) sweep2_persist_kernel(
    float* slab0, float* slab1, const InstParams* __restrict__ insts,
    const WorkItem* __restrict__ items2, const ItemLink* __restrict__ links2, int n_items,
    int steps, int* queue, int* done, int* __restrict__ status, int dep_limit) {
  __shared__ int s_q, s_stop;
  __shared__ PersistState ps;
  const MomArgs<float> mo{};
  const int total = steps * n_items;
  PersistHook h{&ps, queue, links2, done, n_items, total};
  if (threadIdx.x == 0) {
    ps.release = -1;
    ps.have_link = ps.dep_ok = 0;
    ps.next = atomicAdd(queue, 1);
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const int q = ps.next;
      int stop = 0;
      if (q < total) {
        const int t = q / n_items;
        if (t > 0 && !ps.dep_ok) {
          h.release_done();  // never wait while holding a finished item
          if (!ps.have_link) ps.ln = links2[(t & 1) * n_items + (q - t * n_items)];
          if (!wait_deps(done, ps.ln, ps.ln.strips * t, dep_limit)) {
            atomicOr(status, STATUS_TIMEOUT);
            stop = 1;
          }
        }
        fence_proxy_async_global();  // the acquired stores precede this CTA's bulk reads
      } else {
        h.release_done();
      }
      s_q = q;
      s_stop = stop;
    }
    __syncthreads();
    const int q = s_q;
    if (q >= total || s_stop) return;
    const int t = q / n_items, k = q - t * n_items, par = t & 1;
    const WorkItem it = items2[par * n_items + k];
    const InstParams& P = insts[it.inst];
    float* fin = par ? slab1 : slab0;
    float* fout = par ? slab0 : slab1;
    constexpr int body = KIND == PERSIST_MIXED ? 2 : KIND == PERSIST_FULL ? 1 : 0;
    if (sweep2_item<NT, MODE_STEP, body>(fin, fout, P, it, mo, status, 0, h)) return;
    __syncthreads();  // every thread's stores of the item precede its release
    if (threadIdx.x == 0) ps.release = links2[par * n_items + k].chunk;
  }
}

}  // namespace lbm
