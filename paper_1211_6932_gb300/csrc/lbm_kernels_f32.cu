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
