// FP64 instantiations of the step kernel and helpers.
#include "lbm_kernels_impl.cuh"

namespace lbm {

template <>
cudaError_t launch_sweep<double>(int nt, int mode, const double* fin, double* fout,
                             const InstParams* d_inst, const WorkItem* d_items, int n_items,
                             const MomArgs<double>& mo, int* d_status, cudaStream_t st) {
  switch (nt) {
    case 64: return launch_sweep_mode<double, 64>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
    case 128: return launch_sweep_mode<double, 128>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
    default: return cudaErrorInvalidValue;
  }
}

template <>
int sweep_occupancy<double>(int nt) {
  switch (nt) {
    case 64: return occupancy_nt<double, 64>();
    case 128: return occupancy_nt<double, 128>();
    default: return 1;
  }
}

}  // namespace lbm

LBM_INSTANTIATE_HELPERS(double)
