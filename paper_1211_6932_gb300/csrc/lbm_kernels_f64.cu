// FP64 instantiations of the step kernel and helpers.
#include "lbm_kernels_impl.cuh"

namespace lbm {

template <>
cudaError_t launch_sweep<double>(int vec, int mode, const double* fin, double* fout,
                                 const InstParams* d_inst, const WorkItem* d_items,
                                 int n_items, const MomArgs<double>& mo, int* d_status,
                                 cudaStream_t st) {
  switch (vec) {
    case 1: return launch_sweep_vec<double, 1>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
    case 2: return launch_sweep_vec<double, 2>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
    default: return cudaErrorInvalidValue;
  }
}

template <>
int sweep_occupancy<double>(int vec) {
  int occ = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (vec) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_kernel<double, 1, MODE_STEP>, NT, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_kernel<double, 2, MODE_STEP>, NT, 0); break;
    default: break;
  }
  return (e == cudaSuccess && occ > 0) ? occ : 1;
}

}  // namespace lbm

LBM_INSTANTIATE_HELPERS(double)
