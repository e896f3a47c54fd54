// Host-side declarations shared by the C-ABI and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Launch the fused sweep (MODE_STEP) or the moments/diagnostics pass (MODE_MOMENTS) over
// n_items work items; nt (threads per CTA), vec (columns per thread) and, for the pair
// kernel (vec 2), full (full-width strips, see strips_for) select the instantiation.  A
// pair-kernel CTA whose instance is not of the launched kind returns at once.
template <typename S>
cudaError_t launch_sweep(int nt, int vec, int mode, int full, const S* fin, S* fout,
                         const InstParams* d_inst,
                         const WorkItem* d_items, int n_items, const MomArgs<S>& mo,
                         int* d_status, cudaStream_t st);
template <typename S>
cudaError_t launch_fill_ghosts(S* buf, const InstParams& P, cudaStream_t st);
template <typename S>
cudaError_t launch_set_pops(const double* d_fc, S* buf, const InstParams& P, cudaStream_t st);
template <typename S>
cudaError_t launch_get_pops(const S* buf, double* d_fc, const InstParams& P, cudaStream_t st);
template <typename S>
cudaError_t launch_init_eq(const double* rho, const double* ux, const double* uy, S* buf,
                           const InstParams& P, int* d_bad, cudaStream_t st);
template <typename S>
cudaError_t launch_psi(const double* d_rho, double* d_out, long long n,
                       const InstParams* d_inst, cudaStream_t st);
cudaError_t launch_diag_finalize(const double* part_sum, const float* part_max,
                                 const int* part_bad, const int* item_begin, int n_inst,
                                 double* out, cudaStream_t st);

// One droplet of lbm_init_droplets: centre, radius of the half-density circle, liquid
// density.
struct DropRec {
  double cx, cy, r_half, rho_in;
};

// Droplet fill of lbm_init_droplets: rho (ny, nx) doubles on the device; drops holds n
// records.
cudaError_t launch_fill_droplets(double* rho, int nx, int ny, const DropRec* drops, int n,
                                 double rho_v, double width, cudaStream_t st);

// u0 = -F / (2 rho) (Eq. 7 force of the density field) for a force-balanced start.
cudaError_t launch_balanced_velocity(const double* rho, const InstParams& P, double* ux,
                                     double* uy, cudaStream_t st);

// Phase sums of a dense density array (n values of type S): per block, the sum and count
// of values below vmax and above lmin, written to part[4 * block]; returns the number of
// blocks used (at most kPhaseBlocks).
constexpr int kPhaseBlocks = 152 * 4;
template <typename S>
cudaError_t launch_phase_sums(const S* rho, long long n, double vmax, double lmin, double* part,
                              cudaStream_t st);

// Discrete pressure tensor of Eq. 18 from a dense density array of one instance (plus the
// improved forcing's isotropic 2 sigma |F/psi|^2 when sigma != 0): three (ny, nx) doubles.
template <typename S>
cudaError_t launch_pressure(const S* rho, const InstParams& P, double sigma, double* pxx,
                            double* pyy, double* pxy, cudaStream_t st);

// FP32 pair kernel in its persistent form (sweep2_persist_kernel): `steps` time steps of
// one work list, from slab0 (step 0 reads it) and slab1, with `grid` CTAs.  kind is
// PERSIST_STRIP or PERSIST_FULL (every item of that kind of strip) or PERSIST_MIXED (each
// item's kind from its instance's width).  items2 and links2 hold 2 n_items entries (the
// even steps' list, then the odd steps'); queue (one int) and done (one int per chunk)
// must be zero at launch; dep_limit bounds each dependency wait (DEP_WAIT_LIMIT).
cudaError_t launch_persist(int nt, int kind, float* slab0, float* slab1,
                           const InstParams* d_inst, const WorkItem* items2,
                           const ItemLink* links2, int n_items, int steps, int* queue,
                           int* done, int* d_status, int grid, int dep_limit, cudaStream_t st);
// Resident CTAs per SM of the persistent pair kernel of width nt and that kind (at least 1).
int persist_occupancy(int nt, int kind);

// Status bit of an asynchronous initialisation whose fields failed the validity check
// (host-side status only; distinct from the kernels' STATUS_* bits).
constexpr int STATUS_BADINIT = 1 << 8;
// *status |= bit if *flag != 0 (one thread).
cudaError_t launch_flag_status(const int* flag, int* status, int bit, cudaStream_t st);

// dst[i] = (double)src[i] for n values.
cudaError_t launch_widen(const float* src, double* dst, long long n, cudaStream_t st);
// dst[i] = src[i] rounded to the nearest float, for n values.
cudaError_t launch_narrow(const double* src, float* dst, long long n, cudaStream_t st);

// dst = the transpose of src converted to D: src holds h rows of w values, dst w rows of
// h values, dst[x * h + y] = src[y * w + x] (double to float rounds to nearest).
template <typename S, typename D>
cudaError_t launch_transpose(const S* src, D* dst, int w, int h, cudaStream_t st);

// One-block kernel whose bounded mbarrier wait runs out after `polls` polls and sets
// STATUS_TIMEOUT in *status (lbm_selftest_timeout).
cudaError_t launch_wait_selftest(int* status, long long polls, cudaStream_t st);

// Resident CTAs per SM of the step kernel instantiation (at least 1).
template <typename S>
int sweep_occupancy(int nt, int vec);

// Whether a (storage type, threads per CTA, columns per thread) triple has a kernel.
inline bool cfg_supported(bool fp64, int nt, int vec) {
  if (vec == 2) return !fp64 && (nt == 32 || nt == 64 || nt == 96 || nt == 128);
  if (vec != 1) return false;
  return nt == 64 || nt == 128 || (nt == 256 && !fp64);
}

// Columns owned by one CTA of a configuration.
inline int strip_width(int nt, int vec) { return vec == 2 ? 2 * nt - 4 : nt - 4; }
// CTA strips across an instance of nx columns.  The pair kernel (vec 2) covers an
// instance with nx <= 2 nt in one full-width strip: every thread owns two columns, the
// periodic wrap in x is taken inside shared memory and the ghost columns are neither
// read nor written.  Otherwise strips of strip_width owned columns.
inline bool full_width(int nx, int nt, int vec) { return vec == 2 && nx <= 2 * nt; }
inline int strips_for(int nx, int nt, int vec) {
  if (full_width(nx, nt, vec)) return 1;
  const int W = strip_width(nt, vec);
  return (nx + W - 1) / W;
}

}  // namespace lbm
