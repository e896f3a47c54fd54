// Small device kernels outside the step: the per-instance diagnostics totals, the
// float-to-double widening and double-to-float narrowing of host transfers, and the
// bounded-wait self-test.
#include "lbm_kernels_impl.cuh"

namespace lbm {

// Per-instance totals from the per-work-item partials.  One block per instance; thread t
// takes items t, t + 256, ... and the block combines them in a fixed tree order, so the
// result does not depend on scheduling.
// out: 6 doubles per instance (mass, mom_x, mom_y, max_u, dinf, nonfinite).
__global__ void __launch_bounds__(256) diag_finalize_kernel(const double* __restrict__ part_sum,
                                                            const float* __restrict__ part_max,
                                                            const int* __restrict__ part_bad,
                                                            const int* __restrict__ item_begin,
                                                            int n_inst, double* __restrict__ out) {
  __shared__ double sd[3][256];
  __shared__ float sf[2][256];
  __shared__ long long sb[256];
  const int i = blockIdx.x, t = threadIdx.x;
  if (i >= n_inst) return;
  double m = 0, x = 0, y = 0;
  float mu = 0.f, md = 0.f;
  long long b = 0;
  for (int k = item_begin[i] + t; k < item_begin[i + 1]; k += 256) {
    m += part_sum[3 * k];
    x += part_sum[3 * k + 1];
    y += part_sum[3 * k + 2];
    mu = fmaxf(mu, part_max[2 * k]);
    md = fmaxf(md, part_max[2 * k + 1]);
    b += part_bad[k];
  }
  sd[0][t] = m;
  sd[1][t] = x;
  sd[2][t] = y;
  sf[0][t] = mu;
  sf[1][t] = md;
  sb[t] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) {
      sd[0][t] += sd[0][t + w];
      sd[1][t] += sd[1][t + w];
      sd[2][t] += sd[2][t + w];
      sf[0][t] = fmaxf(sf[0][t], sf[0][t + w]);
      sf[1][t] = fmaxf(sf[1][t], sf[1][t + w]);
      sb[t] += sb[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[6 * i + 0] = sd[0][0];
    out[6 * i + 1] = sd[1][0];
    out[6 * i + 2] = sd[2][0];
    out[6 * i + 3] = sf[0][0];
    out[6 * i + 4] = sf[1][0];
    out[6 * i + 5] = (double)sb[0];
  }
}

// Failure-detection check: thread 0 waits on an mbarrier that nothing arrives at, with
// the step kernels' bounded-wait helper and a caller-given poll limit, and reports the
// timeout through the same status word.  No copy is in flight, so giving up is clean.
__global__ void wait_selftest_kernel(int* __restrict__ status, long long polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_polls(&bar, 0u, polls)) atomicOr(status, STATUS_TIMEOUT);
}

// float -> double copy on the device (host reads of FP32 fields land as doubles).
__global__ void __launch_bounds__(256) widen_kernel(const float* __restrict__ src,
                                                    double* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

cudaError_t launch_widen(const float* src, double* dst, long long n, cudaStream_t st) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  widen_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// double -> float (round to nearest) on the device, for float host reads of FP64 fields.
__global__ void __launch_bounds__(256) narrow_kernel(const double* __restrict__ src,
                                                     float* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

cudaError_t launch_narrow(const double* src, float* dst, long long n, cudaStream_t st) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  narrow_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// Transpose through 32 x 32 tiles in shared memory (row-wise reads and writes); block
// (32, 8), grid (tiles across w, up to 65535 tile rows, looped over the rest of h).
template <typename S, typename D>
__global__ void __launch_bounds__(256) transpose_kernel(const S* __restrict__ src,
                                                        D* __restrict__ dst, int w, int h) {
  __shared__ D tile[32][33];
  const int bx = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int by = blockIdx.y * 32; by < h; by += gridDim.y * 32) {
    for (int k = ty; k < 32; k += 8) {
      const int x = bx + tx, y = by + k;
      if (x < w && y < h) tile[k][tx] = (D)src[(long long)y * w + x];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      const int x = bx + k, y = by + tx;  // dst row x, column y
      if (x < w && y < h) dst[(long long)x * h + y] = tile[tx][k];
    }
    __syncthreads();
  }
}

template <typename S, typename D>
cudaError_t launch_transpose(const S* src, D* dst, int w, int h, cudaStream_t st) {
  if (w <= 0 || h <= 0) return cudaSuccess;
  const int gx = (w + 31) / 32, gy = std::min((h + 31) / 32, 65535);
  transpose_kernel<S, D><<<dim3(gx, gy), dim3(32, 8), 0, st>>>(src, dst, w, h);
  return cudaGetLastError();
}

template cudaError_t launch_transpose<float, double>(const float*, double*, int, int,
                                                     cudaStream_t);
template cudaError_t launch_transpose<double, double>(const double*, double*, int, int,
                                                      cudaStream_t);
template cudaError_t launch_transpose<float, float>(const float*, float*, int, int,
                                                    cudaStream_t);
template cudaError_t launch_transpose<double, float>(const double*, float*, int, int,
                                                     cudaStream_t);

__global__ void flag_status_kernel(const int* __restrict__ flag, int* __restrict__ status,
                                   int bit) {
  if (*flag != 0) atomicOr(status, bit);
}

cudaError_t launch_flag_status(const int* flag, int* status, int bit, cudaStream_t st) {
  flag_status_kernel<<<1, 1, 0, st>>>(flag, status, bit);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* status, long long polls, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status, polls);
  return cudaGetLastError();
}

cudaError_t launch_diag_finalize(const double* part_sum, const float* part_max,
                                 const int* part_bad, const int* item_begin, int n_inst,
                                 double* out, cudaStream_t st) {
  diag_finalize_kernel<<<n_inst, 256, 0, st>>>(part_sum, part_max, part_bad, item_begin,
                                                n_inst, out);
  return cudaGetLastError();
}

}  // namespace lbm
