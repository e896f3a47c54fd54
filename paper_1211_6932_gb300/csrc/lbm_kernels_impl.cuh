// Launchers of the step and helper kernels for one storage type (included once per type).
#pragma once
#include <atomic>

#include "lbm_aux.cuh"
#include "lbm_internal.h"

namespace lbm {

// Set a kernel's dynamic shared-memory limit once per device: the attribute belongs to the
// current device's context, so `done` keeps one bit per device ordinal (below 64; others
// are set on every launch).
template <typename F>
static cudaError_t ensure_smem_attr(F* fn, size_t smem, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && bit) done.fetch_or(bit);
  return e;
}

template <typename S, int NT, int MODE>
static cudaError_t launch_sweep_cfg(const S* fin, S* fout, const InstParams* d_inst,
                                    const WorkItem* d_items, int n_items, const MomArgs<S>& mo,
                                    int* d_status, cudaStream_t st) {
  constexpr size_t smem = SweepCfg<S, NT>::BYTES;
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = ensure_smem_attr(sweep_kernel<S, NT, MODE>, smem, done);
  if (e != cudaSuccess) return e;
  if (n_items <= 0) return cudaSuccess;
  sweep_kernel<S, NT, MODE><<<n_items, NT, smem, st>>>(fin, fout, d_inst, d_items, n_items,
                                                       mo, d_status);
  return cudaGetLastError();
}

template <typename S, int NT>
static cudaError_t launch_sweep_mode(int mode, const S* fin, S* fout, const InstParams* d_inst,
                                     const WorkItem* d_items, int n_items,
                                     const MomArgs<S>& mo, int* d_status, cudaStream_t st) {
  if (mode == MODE_STEP)
    return launch_sweep_cfg<S, NT, MODE_STEP>(fin, fout, d_inst, d_items, n_items, mo,
                                              d_status, st);
  return launch_sweep_cfg<S, NT, MODE_MOMENTS>(fin, fout, d_inst, d_items, n_items, mo,
                                               d_status, st);
}

// FP32 pair kernel (two columns per thread, packed float2 arithmetic), strip or
// full-width instantiation.
template <int NT, int MODE, bool FULL>
static cudaError_t launch_sweep2_cfg(const float* fin, float* fout, const InstParams* d_inst,
                                     const WorkItem* d_items, int n_items,
                                     const MomArgs<float>& mo, int* d_status, cudaStream_t st) {
  constexpr size_t smem = Sweep2Cfg<NT>::BYTES;
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = ensure_smem_attr(sweep2_kernel<NT, MODE, FULL>, smem, done);
  if (e != cudaSuccess) return e;
  if (n_items <= 0) return cudaSuccess;
  sweep2_kernel<NT, MODE, FULL><<<n_items, NT, smem, st>>>(fin, fout, d_inst, d_items, n_items,
                                                           mo, d_status);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_sweep2_mode(int mode, int full, const float* fin, float* fout,
                                      const InstParams* d_inst, const WorkItem* d_items,
                                      int n_items, const MomArgs<float>& mo, int* d_status,
                                      cudaStream_t st) {
  if (mode == MODE_STEP)
    return full ? launch_sweep2_cfg<NT, MODE_STEP, true>(fin, fout, d_inst, d_items, n_items,
                                                         mo, d_status, st)
                : launch_sweep2_cfg<NT, MODE_STEP, false>(fin, fout, d_inst, d_items, n_items,
                                                          mo, d_status, st);
  return full ? launch_sweep2_cfg<NT, MODE_MOMENTS, true>(fin, fout, d_inst, d_items, n_items,
                                                          mo, d_status, st)
              : launch_sweep2_cfg<NT, MODE_MOMENTS, false>(fin, fout, d_inst, d_items, n_items,
                                                           mo, d_status, st);
}

// Persistent pair kernel (sweep2_persist_kernel) with `grid` CTAs.
template <int NT, int KIND>
static cudaError_t launch_persist2_cfg(float* slab0, float* slab1, const InstParams* d_inst,
                                       const WorkItem* items2, const ItemLink* links2,
                                       int n_items, int steps, int* queue, int* done,
                                       int* d_status, int grid, int dep_limit,
                                       cudaStream_t st) {
  constexpr size_t smem = Sweep2Cfg<NT>::BYTES;
  static std::atomic<unsigned long long> flag{0};
  cudaError_t e = ensure_smem_attr(sweep2_persist_kernel<NT, KIND>, smem, flag);
  if (e != cudaSuccess) return e;
  if (n_items <= 0 || steps <= 0 || grid <= 0) return cudaSuccess;
  sweep2_persist_kernel<NT, KIND><<<grid, NT, smem, st>>>(slab0, slab1, d_inst, items2, links2,
                                                          n_items, steps, queue, done,
                                                          d_status, dep_limit);
  return cudaGetLastError();
}

template <int NT, int KIND>
static int persist_occupancy_cfg() {
  constexpr size_t smem = Sweep2Cfg<NT>::BYTES;
  cudaFuncSetAttribute(sweep2_persist_kernel<NT, KIND>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, sweep2_persist_kernel<NT, KIND>, NT, smem);
  return (e == cudaSuccess && occ > 0) ? occ : 1;
}

template <int NT>
static int occupancy2_cfg() {
  constexpr size_t smem = Sweep2Cfg<NT>::BYTES;
  cudaFuncSetAttribute(sweep2_kernel<NT, MODE_STEP, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, sweep2_kernel<NT, MODE_STEP, false>, NT, smem);
  return (e == cudaSuccess && occ > 0) ? occ : 1;
}

template <typename S, int NT>
static int occupancy_cfg() {
  constexpr size_t smem = SweepCfg<S, NT>::BYTES;
  cudaFuncSetAttribute(sweep_kernel<S, NT, MODE_STEP>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, sweep_kernel<S, NT, MODE_STEP>, NT, smem);
  return (e == cudaSuccess && occ > 0) ? occ : 1;
}

static inline int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

template <typename S>
cudaError_t launch_set_pops(const double* d_fc, S* buf, const InstParams& P, cudaStream_t st) {
  set_pops_kernel<S><<<grid_for((long long)P.nx * P.ny), 256, 0, st>>>(d_fc, buf, P);
  return cudaGetLastError();
}
template <typename S>
cudaError_t launch_get_pops(const S* buf, double* d_fc, const InstParams& P, cudaStream_t st) {
  get_pops_kernel<S><<<grid_for((long long)P.nx * P.ny), 256, 0, st>>>(buf, d_fc, P);
  return cudaGetLastError();
}
template <typename S>
cudaError_t launch_init_eq(const double* rho, const double* ux, const double* uy, S* buf,
                           const InstParams& P, int* d_bad, cudaStream_t st) {
  init_eq_kernel<S><<<grid_for((long long)P.nx * P.ny), 256, 0, st>>>(rho, ux, uy, buf, P,
                                                                      d_bad);
  return cudaGetLastError();
}
template <typename S>
cudaError_t launch_fill_ghosts(S* buf, const InstParams& P, cudaStream_t st) {
  fill_ghosts_kernel<S><<<grid_for((long long)Q * P.ny * 4), 256, 0, st>>>(buf, P);
  return cudaGetLastError();
}
template <typename S>
cudaError_t launch_psi(const double* d_rho, double* d_out, long long n,
                       const InstParams* d_inst, cudaStream_t st) {
  psi_kernel<S><<<grid_for(n), 256, 0, st>>>(d_rho, d_out, n, d_inst);
  return cudaGetLastError();
}

}  // namespace lbm

#define LBM_INSTANTIATE_HELPERS(S)                                                          \
  template cudaError_t lbm::launch_set_pops<S>(const double*, S*, const lbm::InstParams&,   \
                                               cudaStream_t);                               \
  template cudaError_t lbm::launch_get_pops<S>(const S*, double*, const lbm::InstParams&,   \
                                               cudaStream_t);                               \
  template cudaError_t lbm::launch_init_eq<S>(const double*, const double*, const double*,  \
                                              S*, const lbm::InstParams&, int*,             \
                                              cudaStream_t);                                \
  template cudaError_t lbm::launch_psi<S>(const double*, double*, long long,                \
                                          const lbm::InstParams*, cudaStream_t);            \
  template cudaError_t lbm::launch_fill_ghosts<S>(S*, const lbm::InstParams&, cudaStream_t);
