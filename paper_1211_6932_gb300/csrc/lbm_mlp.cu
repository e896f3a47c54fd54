// Warm-start network (declared in include/lbm_mlp.h): forward, backward and Adam kernels
// for a 4 -> 64 -> 64 -> 5 GELU perceptron with BF16 weights and FP32 accumulation.
//
// The network is far too small for tensor cores to pay off (4805 parameters, a few
// hundred rows), so it runs on the CUDA cores:
//   mlp_rows_kernel   one warp per row: lane l owns hidden units l and l + 32; weights
//                     staged in shared memory as floats (rows padded to avoid bank
//                     conflicts); forward, and in training mode the backward pass down to
//                     the per-row deltas, which are written to row-major scratch.
//   mlp_param_kernel  32 parameters per block, one per lane, and the rows split over the
//                     block's 8 warps (warp w sums rows w, w + 8, ... in order); the 8
//                     partial sums are added in warp order (deterministic), then the
//                     Adam update of the FP32 master weight, its moments and its BF16
//                     copy.  Block 0 also reduces the loss in a fixed order.  (One thread
//                     per parameter summing all rows left one warp per SM waiting on its
//                     loads: 34 us of a 49 us update under ncu, against 18.6 us.  With 32
//                     row slices the Adam trajectory of 60 updates left 1.4 % of the
//                     parameters more than 1e-5 from the oracle's, against 1 % allowed:
//                     the summation order moves parameters whose second moment is tiny.)
// Runs of training updates are replayed from a captured CUDA graph.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lbm_mlp.h"

namespace {

constexpr int NI = LBM_MLP_IN, NH = LBM_MLP_HIDDEN, NO = LBM_MLP_OUT, NP = LBM_MLP_NPARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH;
static_assert(OFF_B3 + NO == NP, "parameter packing");
constexpr int W1S = NI + 1;  // padded row strides in shared memory
constexpr int W2S = NH + 1;
constexpr int ROWS_PER_BLOCK = 8;  // warps per block in the rows kernel
constexpr int PARAM_THREADS = 256;
constexpr int PARAM_SLICES = PARAM_THREADS / 32;  // row slices (warps) per parameter
constexpr int PARAM_BLOCKS = (NP + 31) / 32;      // 32 parameters per block
constexpr int kGraphUpdates = 50;
constexpr int kLossHistory = 1 << 16;

struct Scaling {
  float in_mean[NI], in_scale[NI], out_mean[NO], out_scale[NO];
};

// Per-row scratch (row-major, n rows each).
struct RowBufs {
  float* xn;   // n x 4, standardised inputs
  float* h1;   // n x 64
  float* h2;   // n x 64
  float* dz1;  // n x 64, dL/dz1
  float* dz2;  // n x 64, dL/dz2
  float* dy;   // n x 5, dL/dy (standardised outputs)
  float* lrow; // n, sum over outputs of the squared error
};

struct AdamArgs {
  float lr, beta1, beta2, eps;
};

__device__ __forceinline__ float norm_cdf(float z) {
  return 0.5f * erfcf(-z * 0.70710678118654752f);
}
__device__ __forceinline__ float gelu(float z) { return z * norm_cdf(z); }
__device__ __forceinline__ float gelu_grad(float z) {
  return norm_cdf(z) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ float warp_sum(float v) {
  // xor butterfly: a + b == b + a exactly, so every lane ends with the same value
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

enum { ROWS_PREDICT = 0, ROWS_TRAIN = 1 };

template <int MODE>
__global__ void __launch_bounds__(ROWS_PER_BLOCK * 32) mlp_rows_kernel(
    const __nv_bfloat16* __restrict__ w, const float* __restrict__ x,
    const float* __restrict__ t, int n, Scaling sc, RowBufs rb, double* __restrict__ y_out,
    long long* __restrict__ update_counter) {
  __shared__ float sW1[NH * W1S], sB1[NH], sW2[NH * W2S], sB2[NH], sW3[NO * NH], sB3[NO];
  __shared__ float sBuf[ROWS_PER_BLOCK][NH];
  const int tid = threadIdx.x;
  for (int i = tid; i < NP; i += blockDim.x) {
    const float v = __bfloat162float(w[i]);
    if (i < OFF_B1) sW1[(i / NI) * W1S + i % NI] = v;
    else if (i < OFF_W2) sB1[i - OFF_B1] = v;
    else if (i < OFF_B2) sW2[((i - OFF_W2) / NH) * W2S + (i - OFF_W2) % NH] = v;
    else if (i < OFF_W3) sB2[i - OFF_B2] = v;
    else if (i < OFF_B3) sW3[i - OFF_W3] = v;
    else sB3[i - OFF_B3] = v;
  }
  __syncthreads();
  if (MODE == ROWS_TRAIN && update_counter && blockIdx.x == 0 && tid == 0) ++*update_counter;
  const int warp = tid >> 5, lane = tid & 31;
  const int row = blockIdx.x * ROWS_PER_BLOCK + warp;
  if (row >= n) return;
  float* buf = sBuf[warp];

  float xn[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) xn[i] = (x[(size_t)row * NI + i] - sc.in_mean[i]) / sc.in_scale[i];

  // layer 1
  float z1[2], h1[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float z = sB1[j];
#pragma unroll
    for (int i = 0; i < NI; ++i) z = fmaf(sW1[j * W1S + i], xn[i], z);
    z1[u] = z;
    h1[u] = gelu(z);
    buf[j] = h1[u];
  }
  __syncwarp();
  // layer 2
  float z2[2], h2[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float z = sB2[j];
#pragma unroll 16
    for (int k = 0; k < NH; ++k) z = fmaf(sW2[j * W2S + k], buf[k], z);
    z2[u] = z;
    h2[u] = gelu(z);
  }
  // output layer
  float y[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    const float part = fmaf(sW3[o * NH + lane], h2[0], sW3[o * NH + lane + 32] * h2[1]);
    y[o] = sB3[o] + warp_sum(part);
  }

  if (MODE == ROWS_PREDICT) {
    if (lane < NO) {
      float yo = y[0];
#pragma unroll
      for (int o = 1; o < NO; ++o)
        if (lane == o) yo = y[o];
      y_out[(size_t)row * NO + lane] = (double)sc.out_mean[lane] + (double)sc.out_scale[lane] * yo;
    }
    return;
  }

  // backward: loss = sum over rows and outputs of e^2 / (n * NO), e = y - t_n
  const float inv = 2.0f / ((float)n * (float)NO);
  float dy[NO], l2 = 0.f;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    const float tn = (t[(size_t)row * NO + o] - sc.out_mean[o]) / sc.out_scale[o];
    const float e = y[o] - tn;
    l2 = fmaf(e, e, l2);
    dy[o] = inv * e;
  }
  float dz2[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float d = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o) d = fmaf(sW3[o * NH + j], dy[o], d);
    dz2[u] = d * gelu_grad(z2[u]);
  }
  __syncwarp();  // every lane has finished reading h1 from buf
  buf[lane] = dz2[0];
  buf[lane + 32] = dz2[1];
  __syncwarp();
  float dz1[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    float d = 0.f;
#pragma unroll 16
    for (int j = 0; j < NH; ++j) d = fmaf(sW2[j * W2S + k], buf[j], d);
    dz1[u] = d * gelu_grad(z1[u]);
  }
  const size_t rh = (size_t)row * NH;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    rb.h1[rh + j] = h1[u];
    rb.h2[rh + j] = h2[u];
    rb.dz1[rh + j] = dz1[u];
    rb.dz2[rh + j] = dz2[u];
  }
  if (lane < NI) {
    float v = xn[0];
#pragma unroll
    for (int i = 1; i < NI; ++i)
      if (lane == i) v = xn[i];
    rb.xn[(size_t)row * NI + lane] = v;
  }
  if (lane < NO) {
    float v = dy[0];
#pragma unroll
    for (int o = 1; o < NO; ++o)
      if (lane == o) v = dy[o];
    rb.dy[(size_t)row * NO + lane] = v;
  }
  if (lane == 0) rb.lrow[row] = l2;
}

enum { PARAM_GRAD = 0, PARAM_ADAM = 1 };

__global__ void __launch_bounds__(PARAM_THREADS) mlp_param_kernel(
    RowBufs rb, int n, float* __restrict__ master, __nv_bfloat16* __restrict__ w,
    float* __restrict__ m1, float* __restrict__ m2, float* __restrict__ grad_out, AdamArgs a,
    int mode, const long long* __restrict__ update_counter, float* __restrict__ loss_hist,
    float* __restrict__ loss_out) {
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) {
    // loss: fixed partition of the rows over the threads, then a fixed tree
    __shared__ float red[PARAM_THREADS];
    float s = 0.f;
    for (int r = tid; r < n; r += PARAM_THREADS) s += rb.lrow[r];
    red[tid] = s;
    __syncthreads();
    for (int h = PARAM_THREADS / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) {
      const float L = red[0] / ((float)n * (float)NO);
      if (loss_out) *loss_out = L;
      if (mode == PARAM_ADAM && loss_hist)
        loss_hist[(*update_counter - 1) & (kLossHistory - 1)] = L;
    }
  }
  const int lane = tid & 31, slice = tid >> 5;
  const int p = blockIdx.x * 32 + lane;
  __shared__ float part[PARAM_SLICES][32];
  // dL/dp = sum over rows of (delta of the output unit) x (input value): warp `slice` sums
  // rows slice, slice + PARAM_SLICES, ... in order, lane l for parameter p
  const float* da = nullptr;
  const float* xb = nullptr;
  int sa, ia, sb = 0, ib = 0;
  if (p < OFF_B1) {
    da = rb.dz1; sa = NH; ia = p / NI; xb = rb.xn; sb = NI; ib = p % NI;
  } else if (p < OFF_W2) {
    da = rb.dz1; sa = NH; ia = p - OFF_B1;
  } else if (p < OFF_B2) {
    da = rb.dz2; sa = NH; ia = (p - OFF_W2) / NH; xb = rb.h1; sb = NH; ib = (p - OFF_W2) % NH;
  } else if (p < OFF_W3) {
    da = rb.dz2; sa = NH; ia = p - OFF_B2;
  } else if (p < OFF_B3) {
    da = rb.dy; sa = NO; ia = (p - OFF_W3) / NH; xb = rb.h2; sb = NH; ib = (p - OFF_W3) % NH;
  } else {
    da = rb.dy; sa = NO; ia = p - OFF_B3;
  }
  float g = 0.f;
  if (p < NP) {
    if (xb) {
#pragma unroll 4
      for (int r = slice; r < n; r += PARAM_SLICES)
        g = fmaf(da[(size_t)r * sa + ia], xb[(size_t)r * sb + ib], g);
    } else {
#pragma unroll 4
      for (int r = slice; r < n; r += PARAM_SLICES) g += da[(size_t)r * sa + ia];
    }
  }
  part[slice][lane] = g;
  __syncthreads();
  if (slice != 0 || p >= NP) return;
  g = part[0][lane];
#pragma unroll
  for (int k = 1; k < PARAM_SLICES; ++k) g += part[k][lane];
  if (grad_out) grad_out[p] = g;
  if (mode != PARAM_ADAM) return;
  // Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 master weight
  const float k = (float)*update_counter;
  const float mm = fmaf(a.beta1, m1[p], (1.f - a.beta1) * g);
  const float vv = fmaf(a.beta2, m2[p], (1.f - a.beta2) * g * g);
  const float mhat = mm / (1.f - powf(a.beta1, k));
  const float vhat = vv / (1.f - powf(a.beta2, k));
  const float pm = master[p] - a.lr * mhat / (sqrtf(vhat) + a.eps);
  m1[p] = mm;
  m2[p] = vv;
  master[p] = pm;
  w[p] = __float2bfloat16_rn(pm);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}
__global__ void from_bf16_kernel(const __nv_bfloat16* __restrict__ src, float* __restrict__ dst,
                                 int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __bfloat162float(src[i]);
}

}  // namespace

struct lbm_mlp {
  int device = -1;
  int max_rows = 0;
  int n = 0;  // rows of the uploaded training set
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  float* master = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* w = nullptr;
  float* x = nullptr;   // training inputs
  float* t = nullptr;   // training targets
  float* xp = nullptr;  // inputs of the last predict call
  double* y = nullptr;
  RowBufs rb{};
  float* scratch = nullptr;
  long long* counter = nullptr;
  float* loss_hist = nullptr;
  float* loss_one = nullptr;
  long long updates = 0;
  Scaling sc{};
  AdamArgs graph_args{};
  int graph_n = 0;
  cudaGraphExec_t graph = nullptr;
  std::string err;
};

namespace {

thread_local std::string g_mlp_err;

int mset_err(lbm_mlp* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  (h ? h->err : g_mlp_err) = buf;
  return code;
}

#define MCK(h, call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return mset_err(h, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct MlpDeviceGuard {
  explicit MlpDeviceGuard(const lbm_mlp* h) {
    if (h && h->device >= 0) cudaSetDevice(h->device);
  }
};

void free_all(lbm_mlp* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  void* ptrs[] = {h->master, h->m1, h->m2, h->grad, h->w, h->x, h->t, h->xp, h->y, h->scratch,
                  h->counter, h->loss_hist, h->loss_one};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

int launch_rows(lbm_mlp* h, int mode, int n, double* y_out, long long* counter,
                cudaStream_t st) {
  const int blocks = (n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
  if (mode == ROWS_TRAIN)
    mlp_rows_kernel<ROWS_TRAIN><<<blocks, ROWS_PER_BLOCK * 32, 0, st>>>(h->w, h->x, h->t, n, h->sc,
                                                                       h->rb, y_out, counter);
  else
    mlp_rows_kernel<ROWS_PREDICT><<<blocks, ROWS_PER_BLOCK * 32, 0, st>>>(
        h->w, h->xp, nullptr, n, h->sc, h->rb, y_out, counter);
  MCK(h, cudaGetLastError());
  return LBM_OK;
}

int launch_update(lbm_mlp* h, const AdamArgs& a, cudaStream_t st) {
  int rc = launch_rows(h, ROWS_TRAIN, h->n, nullptr, h->counter, st);
  if (rc) return rc;
  mlp_param_kernel<<<PARAM_BLOCKS, PARAM_THREADS, 0, st>>>(
      h->rb, h->n, h->master, h->w, h->m1, h->m2, nullptr, a, PARAM_ADAM, h->counter,
      h->loss_hist, nullptr);
  MCK(h, cudaGetLastError());
  return LBM_OK;
}

int capture(lbm_mlp* h, const AdamArgs& a) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  MCK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBM_OK;
  for (int k = 0; k < kGraphUpdates && rc == LBM_OK; ++k) rc = launch_update(h, a, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess)
    return mset_err(h, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return mset_err(h, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  h->graph_args = a;
  h->graph_n = h->n;
  return LBM_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int upload_rows(lbm_mlp* h, float* dst, const double* src, int n, int cols) {
  std::vector<float> tmp((size_t)n * cols);
  for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = (float)src[i];
  MCK(h, cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice,
                         h->stream));
  MCK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_mlp_create(lbm_mlp** out, const float* params, int max_rows, void* stream, int device) {
  if (!out || !params) return mset_err(nullptr, LBM_EINVAL, "out and params must not be NULL");
  *out = nullptr;
  if (max_rows < 1) return mset_err(nullptr, LBM_EINVAL, "max_rows must be >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return mset_err(nullptr, LBM_ECUDA, "no usable CUDA device");
  }
  if (device >= ndev) return mset_err(nullptr, LBM_EINVAL, "device %d out of range", device);
  lbm_mlp* h = new lbm_mlp();
  if (device < 0) cudaGetDevice(&device);
  h->device = device;
  MlpDeviceGuard guard(h);
  h->max_rows = max_rows;
  h->stream = (cudaStream_t)stream;
  for (int i = 0; i < NI; ++i) h->sc.in_scale[i] = 1.f;
  for (int o = 0; o < NO; ++o) h->sc.out_scale[o] = 1.f;
  auto fail = [&](const char* what, cudaError_t e) {
    int rc = mset_err(nullptr, LBM_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
    free_all(h);
    delete h;
    return rc;
  };
  cudaError_t e;
  const size_t R = (size_t)max_rows;
  const size_t scratch_floats = R * (NI + 4 * NH + NO + 1);
  if ((e = cudaMalloc(&h->master, NP * sizeof(float))) ||
      (e = cudaMalloc(&h->m1, NP * sizeof(float))) ||
      (e = cudaMalloc(&h->m2, NP * sizeof(float))) ||
      (e = cudaMalloc(&h->grad, NP * sizeof(float))) ||
      (e = cudaMalloc(&h->w, NP * sizeof(__nv_bfloat16))) ||
      (e = cudaMalloc(&h->x, R * NI * sizeof(float))) ||
      (e = cudaMalloc(&h->t, R * NO * sizeof(float))) ||
      (e = cudaMalloc(&h->xp, R * NI * sizeof(float))) ||
      (e = cudaMalloc(&h->y, R * NO * sizeof(double))) ||
      (e = cudaMalloc(&h->scratch, scratch_floats * sizeof(float))) ||
      (e = cudaMalloc(&h->counter, sizeof(long long))) ||
      (e = cudaMalloc(&h->loss_hist, kLossHistory * sizeof(float))) ||
      (e = cudaMalloc(&h->loss_one, sizeof(float))) ||
      (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)))
    return fail("device allocation", e);
  float* s = h->scratch;
  h->rb.xn = s; s += R * NI;
  h->rb.h1 = s; s += R * NH;
  h->rb.h2 = s; s += R * NH;
  h->rb.dz1 = s; s += R * NH;
  h->rb.dz2 = s; s += R * NH;
  h->rb.dy = s; s += R * NO;
  h->rb.lrow = s;
  if ((e = cudaMemcpyAsync(h->master, params, NP * sizeof(float), cudaMemcpyHostToDevice,
                           h->stream)) ||
      (e = cudaMemsetAsync(h->m1, 0, NP * sizeof(float), h->stream)) ||
      (e = cudaMemsetAsync(h->m2, 0, NP * sizeof(float), h->stream)) ||
      (e = cudaMemsetAsync(h->counter, 0, sizeof(long long), h->stream)) ||
      (e = cudaMemsetAsync(h->loss_hist, 0, kLossHistory * sizeof(float), h->stream)))
    return fail("initial upload", e);
  to_bf16_kernel<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->master, h->w, NP);
  if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(h->stream)))
    return fail("weight conversion", e);
  *out = h;
  return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* h) {
  if (!h) return;
  MlpDeviceGuard guard(h);
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

const char* lbm_mlp_last_error(const lbm_mlp* h) {
  return h ? h->err.c_str() : g_mlp_err.c_str();
}

int lbm_mlp_set_scaling(lbm_mlp* h, const double in_mean[4], const double in_scale[4],
                        const double out_mean[5], const double out_scale[5]) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!in_mean || !in_scale || !out_mean || !out_scale)
    return mset_err(h, LBM_EINVAL, "scaling arrays must not be NULL");
  for (int i = 0; i < NI; ++i)
    if (!std::isfinite(in_mean[i]) || !finite_pos(in_scale[i]))
      return mset_err(h, LBM_EINVAL, "input scaling %d is not finite and positive", i);
  for (int o = 0; o < NO; ++o)
    if (!std::isfinite(out_mean[o]) || !finite_pos(out_scale[o]))
      return mset_err(h, LBM_EINVAL, "output scaling %d is not finite and positive", o);
  for (int i = 0; i < NI; ++i) {
    h->sc.in_mean[i] = (float)in_mean[i];
    h->sc.in_scale[i] = (float)in_scale[i];
  }
  for (int o = 0; o < NO; ++o) {
    h->sc.out_mean[o] = (float)out_mean[o];
    h->sc.out_scale[o] = (float)out_scale[o];
  }
  h->graph_n = 0;  // the scaling is a kernel argument: re-capture
  return LBM_OK;
}

int lbm_mlp_fit_scaling(lbm_mlp* h, const double* x, const double* t, int n) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!x || !t || n < 1) return mset_err(h, LBM_EINVAL, "need x, t and n >= 1");
  auto stats = [&](const double* a, int cols, int c, double* mu, double* sd) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += a[(size_t)r * cols + c];
    const double m = s / n;
    double q = 0.0;
    for (int r = 0; r < n; ++r) {
      const double d = a[(size_t)r * cols + c] - m;
      q += d * d;
    }
    const double v = std::sqrt(q / n);
    *mu = m;
    *sd = v > 0.0 ? v : 1.0;
  };
  double im[NI], is[NI], om[NO], os[NO];
  for (int i = 0; i < NI; ++i) stats(x, NI, i, &im[i], &is[i]);
  for (int o = 0; o < NO; ++o) stats(t, NO, o, &om[o], &os[o]);
  return lbm_mlp_set_scaling(h, im, is, om, os);
}

int lbm_mlp_set_data(lbm_mlp* h, const double* x, const double* t, int n) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!x || !t) return mset_err(h, LBM_EINVAL, "x and t must not be NULL");
  if (n < 1 || n > h->max_rows)
    return mset_err(h, LBM_EINVAL, "row count %d not in [1, %d]", n, h->max_rows);
  MlpDeviceGuard guard(h);
  int rc = upload_rows(h, h->x, x, n, NI);
  if (!rc) rc = upload_rows(h, h->t, t, n, NO);
  if (rc) return rc;
  h->n = n;
  h->graph_n = 0;
  return LBM_OK;
}

int lbm_mlp_train(lbm_mlp* h, int steps, const lbm_adam* opt, float* losses) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!opt || steps < 0) return mset_err(h, LBM_EINVAL, "need optimiser settings and steps >= 0");
  if (h->n < 1) return mset_err(h, LBM_EINVAL, "no training data uploaded");
  if (!(opt->lr > 0.0) || !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) ||
      !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) || !(opt->eps >= 0.0))
    return mset_err(h, LBM_EINVAL, "Adam settings out of range");
  MlpDeviceGuard guard(h);
  const AdamArgs a{(float)opt->lr, (float)opt->beta1, (float)opt->beta2, (float)opt->eps};
  const long long start = h->updates;
  int left = steps;
  while (left > 0) {
    if (left >= kGraphUpdates) {
      const bool same = h->graph && h->graph_n == h->n && h->graph_args.lr == a.lr &&
                        h->graph_args.beta1 == a.beta1 && h->graph_args.beta2 == a.beta2 &&
                        h->graph_args.eps == a.eps;
      if (!same) {
        MCK(h, cudaStreamSynchronize(h->stream));
        int rc = capture(h, a);
        if (rc) return rc;
      }
      MCK(h, cudaGraphLaunch(h->graph, h->stream));
      left -= kGraphUpdates;
    } else {
      int rc = launch_update(h, a, h->stream);
      if (rc) return rc;
      --left;
    }
  }
  h->updates += steps;
  MCK(h, cudaStreamSynchronize(h->stream));
  if (losses && steps > 0) {
    // losses of updates start+1 .. start+steps live at (index - 1) mod the history size
    std::vector<float> hist(kLossHistory);
    MCK(h, cudaMemcpy(hist.data(), h->loss_hist, kLossHistory * sizeof(float),
                      cudaMemcpyDeviceToHost));
    for (int k = 0; k < steps; ++k) {
      const long long idx = start + k;
      losses[k] = (steps - k <= kLossHistory) ? hist[idx & (kLossHistory - 1)] : NAN;
    }
  }
  return LBM_OK;
}

int lbm_mlp_gradient(lbm_mlp* h, float* grad, float* loss) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (h->n < 1) return mset_err(h, LBM_EINVAL, "no training data uploaded");
  MlpDeviceGuard guard(h);
  int rc = launch_rows(h, ROWS_TRAIN, h->n, nullptr, nullptr, h->stream);
  if (rc) return rc;
  mlp_param_kernel<<<PARAM_BLOCKS, PARAM_THREADS, 0, h->stream>>>(
      h->rb, h->n, h->master, h->w, h->m1, h->m2, h->grad, AdamArgs{}, PARAM_GRAD, nullptr,
      nullptr, h->loss_one);
  MCK(h, cudaGetLastError());
  if (grad)
    MCK(h, cudaMemcpyAsync(grad, h->grad, NP * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  float L = 0.f;
  MCK(h, cudaMemcpyAsync(&L, h->loss_one, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  MCK(h, cudaStreamSynchronize(h->stream));
  if (loss) *loss = L;
  return LBM_OK;
}

int lbm_mlp_predict(lbm_mlp* h, const double* x, int n, double* y) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!x || !y) return mset_err(h, LBM_EINVAL, "x and y must not be NULL");
  if (n < 1 || n > h->max_rows)
    return mset_err(h, LBM_EINVAL, "row count %d not in [1, %d]", n, h->max_rows);
  MlpDeviceGuard guard(h);
  int rc = upload_rows(h, h->xp, x, n, NI);
  if (rc) return rc;
  rc = launch_rows(h, ROWS_PREDICT, n, h->y, nullptr, h->stream);
  if (rc) return rc;
  MCK(h, cudaMemcpyAsync(y, h->y, (size_t)n * NO * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
  MCK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mlp_get_params(lbm_mlp* h, int which, float* out) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!out || which < 0 || which > 3) return mset_err(h, LBM_EINVAL, "bad arguments");
  MlpDeviceGuard guard(h);
  if (which == 1) {
    from_bf16_kernel<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->w, h->grad, NP);
    MCK(h, cudaGetLastError());
  }
  const float* src = which == 0 ? h->master : which == 1 ? h->grad : which == 2 ? h->m1 : h->m2;
  MCK(h, cudaMemcpyAsync(out, src, NP * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  MCK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp* h, int which, const float* in) {
  if (!h) return mset_err(nullptr, LBM_EINVAL, "handle is NULL");
  if (!in || which < 0 || which > 3 || which == 1)
    return mset_err(h, LBM_EINVAL, "bad arguments (the BF16 copy is read only)");
  MlpDeviceGuard guard(h);
  float* dst = which == 0 ? h->master : which == 2 ? h->m1 : h->m2;
  MCK(h, cudaMemcpyAsync(dst, in, NP * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  if (which == 0) {
    to_bf16_kernel<<<(NP + 255) / 256, 256, 0, h->stream>>>(h->master, h->w, NP);
    MCK(h, cudaGetLastError());
  }
  MCK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

long long lbm_mlp_update_count(const lbm_mlp* h) { return h ? h->updates : -1; }

}  // extern "C"
