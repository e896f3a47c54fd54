// FP32 (deviation storage) instantiations of the step kernel and its helpers.
#include "lbm_kernels_impl.cuh"

namespace lbm {

template <>
cudaError_t launch_sweep<float>(int nt, int vec, int mode, int full, const float* fin, float* fout,
                             const InstParams* d_inst, const WorkItem* d_items, int n_items,
                             const MomArgs<float>& mo, int* d_status, cudaStream_t st) {
  if (nt == 64 && vec == 1) return launch_sweep_mode<float, 64>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 128 && vec == 1) return launch_sweep_mode<float, 128>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 256 && vec == 1) return launch_sweep_mode<float, 256>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 32 && vec == 2) return launch_sweep2_mode<32>(mode, full, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 64 && vec == 2) return launch_sweep2_mode<64>(mode, full, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 96 && vec == 2) return launch_sweep2_mode<96>(mode, full, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 128 && vec == 2) return launch_sweep2_mode<128>(mode, full, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_persist(int nt, int kind, float* slab0, float* slab1,
                           const InstParams* d_inst, const WorkItem* items2,
                           const ItemLink* links2, int n_items, int steps, int* queue,
                           int* done, int* d_status, int grid, int dep_limit,
                           cudaStream_t st) {
#define LBM_PERSIST_KIND(T, K)                                                             \
  if (nt == T && kind == K)                                                                \
    return launch_persist2_cfg<T, K>(slab0, slab1, d_inst, items2, links2, n_items, steps, \
                                     queue, done, d_status, grid, dep_limit, st);
#define LBM_PERSIST(T)                  \
  LBM_PERSIST_KIND(T, PERSIST_STRIP)    \
  LBM_PERSIST_KIND(T, PERSIST_FULL)     \
  LBM_PERSIST_KIND(T, PERSIST_MIXED)
  LBM_PERSIST(32)
  LBM_PERSIST(64)
  LBM_PERSIST(96)
  LBM_PERSIST(128)
#undef LBM_PERSIST
#undef LBM_PERSIST_KIND
  return cudaErrorInvalidValue;
}

int persist_occupancy(int nt, int kind) {
#define LBM_PERSIST_OCC(T)                                                          \
  if (nt == T)                                                                      \
    return kind == PERSIST_MIXED  ? persist_occupancy_cfg<T, PERSIST_MIXED>()       \
           : kind == PERSIST_FULL ? persist_occupancy_cfg<T, PERSIST_FULL>()        \
                                  : persist_occupancy_cfg<T, PERSIST_STRIP>();
  LBM_PERSIST_OCC(32)
  LBM_PERSIST_OCC(64)
  LBM_PERSIST_OCC(96)
  LBM_PERSIST_OCC(128)
#undef LBM_PERSIST_OCC
  return 1;
}

template <>
int sweep_occupancy<float>(int nt, int vec) {
  if (nt == 64 && vec == 1) return occupancy_cfg<float, 64>();
  if (nt == 128 && vec == 1) return occupancy_cfg<float, 128>();
  if (nt == 256 && vec == 1) return occupancy_cfg<float, 256>();
  if (nt == 32 && vec == 2) return occupancy2_cfg<32>();
  if (nt == 64 && vec == 2) return occupancy2_cfg<64>();
  if (nt == 96 && vec == 2) return occupancy2_cfg<96>();
  if (nt == 128 && vec == 2) return occupancy2_cfg<128>();
  return 1;
}

}  // namespace lbm

LBM_INSTANTIATE_HELPERS(float)
