// FP64 instantiations of the step kernel and helpers.
#include "lbm_kernels_impl.cuh"

namespace lbm {

template <>
cudaError_t launch_sweep<double>(int nt, int vec, int mode, int full, const double* fin, double* fout,
                             const InstParams* d_inst, const WorkItem* d_items, int n_items,
                             const MomArgs<double>& mo, int* d_status, cudaStream_t st) {
  if (nt == 64 && vec == 1) return launch_sweep_mode<double, 64>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 128 && vec == 1) return launch_sweep_mode<double, 128>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  return cudaErrorInvalidValue;
}

template <>
int sweep_occupancy<double>(int nt, int vec) {
  if (nt == 64 && vec == 1) return occupancy_cfg<double, 64>();
  if (nt == 128 && vec == 1) return occupancy_cfg<double, 128>();
  return 1;
}

}  // namespace lbm

LBM_INSTANTIATE_HELPERS(double)
