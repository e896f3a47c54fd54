// FP32 (deviation storage) instantiations of the step kernel and helpers.
#include "lbm_kernels_impl.cuh"

namespace lbm {

// Per-instance totals from the per-work-item partials, in a fixed order (deterministic).
// out: 6 doubles per instance (mass, mom_x, mom_y, max_u, dinf, nonfinite).
__global__ void diag_finalize_kernel(const double* __restrict__ part_sum,
                                     const float* __restrict__ part_max,
                                     const int* __restrict__ part_bad,
                                     const int* __restrict__ item_begin, int n_inst,
                                     double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  double m = 0, x = 0, y = 0;
  float mu = 0.f, md = 0.f;
  long long b = 0;
  for (int k = item_begin[i]; k < item_begin[i + 1]; ++k) {
    m += part_sum[3 * k];
    x += part_sum[3 * k + 1];
    y += part_sum[3 * k + 2];
    mu = fmaxf(mu, part_max[2 * k]);
    md = fmaxf(md, part_max[2 * k + 1]);
    b += part_bad[k];
  }
  out[6 * i + 0] = m;
  out[6 * i + 1] = x;
  out[6 * i + 2] = y;
  out[6 * i + 3] = mu;
  out[6 * i + 4] = md;
  out[6 * i + 5] = (double)b;
}


template <>
cudaError_t launch_sweep<float>(int nt, int vec, int mode, const float* fin, float* fout,
                             const InstParams* d_inst, const WorkItem* d_items, int n_items,
                             const MomArgs<float>& mo, int* d_status, cudaStream_t st) {
  if (nt == 64 && vec == 1) return launch_sweep_mode<float, 64>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 128 && vec == 1) return launch_sweep_mode<float, 128>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 256 && vec == 1) return launch_sweep_mode<float, 256>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 64 && vec == 2) return launch_sweep2_mode<64>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  if (nt == 128 && vec == 2) return launch_sweep2_mode<128>(mode, fin, fout, d_inst, d_items, n_items, mo, d_status, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_diag_finalize(const double* part_sum, const float* part_max,
                                 const int* part_bad, const int* item_begin, int n_inst,
                                 double* out, cudaStream_t st) {
  diag_finalize_kernel<<<(n_inst + 127) / 128, 128, 0, st>>>(part_sum, part_max, part_bad,
                                                              item_begin, n_inst, out);
  return cudaGetLastError();
}

template <>
int sweep_occupancy<float>(int nt, int vec) {
  if (nt == 64 && vec == 1) return occupancy_cfg<float, 64>();
  if (nt == 128 && vec == 1) return occupancy_cfg<float, 128>();
  if (nt == 256 && vec == 1) return occupancy_cfg<float, 256>();
  if (nt == 64 && vec == 2) return occupancy2_cfg<64>();
  if (nt == 128 && vec == 2) return occupancy2_cfg<128>();
  return 1;
}

}  // namespace lbm

LBM_INSTANTIATE_HELPERS(float)
