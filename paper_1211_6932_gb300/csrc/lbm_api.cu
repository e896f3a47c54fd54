// C ABI of the D2Q9 improved-MRT pseudopotential library (declared in include/lbm.h).
//
// Every lattice, single or batched, is an instance of one Batch: the populations of all
// instances live in two slabs (ping-pong), each instance with its own padded planes; one
// launch of the fused sweep kernel advances every active instance by one step (one launch
// per kernel width under per-instance tiling, the widths as parallel graph branches), and
// runs of steps are replayed from a captured CUDA graph.
#include <cuda.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "../../include/lbm_warm.h"
#include "lbm_internal.h"

using lbm::InstParams;
using lbm::MomArgs;
using lbm::ItemLink;
using lbm::WorkItem;

namespace {

constexpr int kGraphSteps = 64;  // even, so a replay returns to the same slab
thread_local std::string g_thread_err;

struct Batch {
  bool fp64 = false;
  size_t esz = 4;
  int n_inst = 0;
  std::vector<InstParams> inst;  // storage dimensions (axes exchanged where tr[i])
  std::vector<char> tr;          // instance stored transposed (lbm_instance.layout)
  std::vector<int> active;
  std::vector<long long> steps;
  std::vector<char> dinf_valid;
  InstParams* d_inst = nullptr;
  std::vector<WorkItem> items;  // active instances only
  WorkItem* d_items = nullptr;
  int n_items = 0, cap_items = 0;
  // Persistent stepping (FP32 pair kernel, sweep2_persist_kernel): one launch over every
  // step item (both launch groups of one kernel width, as kind PERSIST_MIXED); the even and
  // odd steps' work lists and their dependency links (2 n_items entries each), the queue
  // counter at d_sync[0] followed by the chunk counters (persist_sync ints), the grid.
  bool persist = false;
  bool persist_off = false;  // the autotuner measured one launch per step faster
  int persist_kind = 0, persist_sync = 0, persist_grid = 0;
  WorkItem* d_items2 = nullptr;
  ItemLink* d_links2 = nullptr;
  int* d_sync = nullptr;
  int cap_items2 = 0, cap_sync = 0;
  std::vector<WorkItem> all_items;  // every instance, for diagnostics
  WorkItem* d_all_items = nullptr;
  int n_all = 0, cap_all = 0;
  std::vector<int> item_begin;  // per instance, into all_items
  int* d_item_begin = nullptr;
  void* slab[2] = {nullptr, nullptr};
  size_t slab_elems = 0;
  int cur = 0;
  size_t dense_elems = 0;
  void* rho_prev = nullptr;
  void* fields[3] = {nullptr, nullptr, nullptr};
  double* staging = nullptr;  // 3 x (largest instance) doubles: host uploads and downloads
  size_t staging_elems = 0;
  float* staging32 = nullptr;  // 3 x (largest instance) floats: float host transfers
  double* staging_t = nullptr;  // 3 x (largest transposed instance) doubles
  size_t staging_t_elems = 0;
  int* d_flag = nullptr;      // one int for the initialisation's validity check
  // Asynchronous host transfers (lbm_init_fields_async, lbm_moments_async): copy streams
  // and the events that order them with the handle's stream.
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  cudaEvent_t ev_uploaded = nullptr;      // up_stream: the last upload is on the device
  cudaEvent_t ev_staging_free = nullptr;  // stream: the last initialisation read its staging
  cudaEvent_t ev_fields_ready = nullptr;  // stream: the last asynchronous moments pass ended
  cudaEvent_t ev_fields_free = nullptr;   // down_stream: its read-back left the fields
  double* d_part_sum = nullptr;
  float* d_part_max = nullptr;
  int* d_part_bad = nullptr;
  double* d_diag = nullptr;
  int* d_status = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  int nt = 0, vec = 0, rows_req = 0, rows = 0;  // threads and columns/thread per CTA, rows per sweep
  // Step launches: group g runs items [grp_begin[g], grp_begin[g+1]) with grp_nt[g]
  // threads, in full-width strips if grp_full[g] (pair kernel).  One group per kernel
  // width (one width, unless nt == LBM_TILE_PER_INSTANCE: then each instance has the width
  // inst_nt[i]), split into strip and full-width instances.
  static constexpr int kMaxWidths = 4;
  static constexpr int kMaxGroups = 2 * kMaxWidths;
  std::vector<int> inst_nt;
  int n_groups = 0;
  int grp_nt[kMaxGroups] = {};
  int grp_full[kMaxGroups] = {};
  int grp_begin[kMaxGroups + 1] = {};
  cudaStream_t grp_stream[kMaxGroups - 1] = {};  // graph branches
  cudaEvent_t grp_fork = nullptr, grp_join[kMaxGroups - 1] = {};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // Buffers allocated with guard bands (lbm_check_guards): base pointer, user bytes, name.
  struct Guarded {
    char* base;
    size_t bytes;
    const char* name;
  };
  std::vector<Guarded> guarded;
  std::string err;
  int sms = 0;
  int device = -1;
};

// Makes the batch's device current for the duration of a public call.
struct DeviceGuard {
  explicit DeviceGuard(const Batch* b) {
    if (b && b->device >= 0) cudaSetDevice(b->device);
  }
};

int set_err(std::string& dst, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  dst = buf;
  return code;
}

#define CK(b, call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return set_err((b)->err, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, \
                     "%s failed: %s", #call, cudaGetErrorString(e_));                  \
  } while (0)

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

// Fault injection (lbm_debug_fail_alloc): while >= 0, the number of device allocations
// that still succeed before one fails.
std::atomic<int> g_fail_after{-1};
std::atomic<long long> g_live_allocs{0};  // device allocations not yet released

// Every device allocation of the lattice and batch handles goes through here.
cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  int n = g_fail_after.load();
  while (n >= 0 && !g_fail_after.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
// ... and every release.
void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  g_live_allocs.fetch_sub(1);
}

// Guard bands: this many bytes of kCanary before and after each guarded buffer.
constexpr size_t kGuard = 4096;
constexpr unsigned char kCanary = 0xA5;

// NVTX range over a public call (shown by Nsight Systems / Compute when attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Default kernel configuration per precision (threads per CTA, columns per thread).
int default_threads(bool) { return 128; }  // best measured for both precisions
int default_vec(bool fp64) { return fp64 ? 1 : 2; }

template <typename R>
void fill_mirror(lbm::PhysParams<R>& m, const InstParams& P) {
  m.b4 = (R)P.b4;
  m.RT = (R)P.RT;
  m.a = (R)P.a;
  m.two_over_G = (R)P.two_over_G;
  m.G = (R)P.G;
  m.s1 = (R)P.s[1];
  m.s2 = (R)P.s[2];
  m.s4 = (R)P.s[4];
  m.s6 = (R)P.s[6];
  m.s7 = (R)P.s[7];
  m.s8 = (R)P.s[8];
  m.c1 = (R)(1.0 - 0.5 * P.s[1]);
  m.c2 = (R)(1.0 - 0.5 * P.s[2]);
  m.c4 = (R)(1.0 - 0.5 * P.s[4]);
  m.c6 = (R)(1.0 - 0.5 * P.s[6]);
  m.c7 = (R)(1.0 - 0.5 * P.s[7]);
  m.c8 = (R)(1.0 - 0.5 * P.s[8]);
  m.sig12_e = (R)P.sig12_e;
  m.sig12_z = (R)P.sig12_z;
  m.tau_l = (R)P.tau_l;
  m.tau_v = (R)P.tau_v;
  m.dtau = (R)(P.tau_l - P.tau_v);
  m.rho_c = (R)P.rho_c;
  m.rho_v = (R)P.rho_v;
  m.inv_drho_lv = P.rho_l != P.rho_v ? (R)(1.0 / (P.rho_l - P.rho_v)) : (R)0;
  m.rho_ref = (R)P.rho_ref;
  m.g1 = (R)(-P.G / 3.0);
  m.g2 = (R)(-P.G / 12.0);
  m.k1s = (R)(P.s[1] / 36.0);
  m.k1v = (R)((1.0 - 0.5 * P.s[1]) / 6.0);
  m.k1f = (R)(P.sig12_e / 36.0);
  m.k2s = (R)(P.s[2] / 36.0);
  m.k2v = (R)((1.0 - 0.5 * P.s[2]) / 6.0);
  m.k2f = (R)(P.sig12_z / 36.0);
  m.k4s = (R)(P.s[4] / 12.0);
  m.k4f = (R)((1.0 - 0.5 * P.s[4]) / 12.0);
  m.k6s = (R)(P.s[6] / 12.0);
  m.k6f = (R)((1.0 - 0.5 * P.s[6]) / 12.0);
  m.k7s = (R)(P.s[7] / 4.0);
  m.k7v = (R)((1.0 - 0.5 * P.s[7]) / 2.0);
  m.k8s = (R)(P.s[8] / 4.0);
  m.k8v = (R)((1.0 - 0.5 * P.s[8]) / 4.0);
}

template <typename T>
void free_dev(T*& p) {
  dev_free((void*)p);
  p = nullptr;
}

// Device buffer of `bytes` with kGuard bytes of kCanary on each side; *p is the user part.
int guarded_alloc(Batch* b, void** p, size_t bytes, const char* name) {
  char* base = nullptr;
  CK(b, dev_malloc(&base, bytes + 2 * kGuard));
  b->guarded.push_back({base, bytes, name});  // freed by destroy_batch from here on
  CK(b, cudaMemsetAsync(base, kCanary, kGuard, b->stream));
  CK(b, cudaMemsetAsync(base + kGuard + bytes, kCanary, kGuard, b->stream));
  *p = base + kGuard;
  return LBM_OK;
}

void free_guarded(Batch* b) {
  for (auto& g : b->guarded) dev_free(g.base);
  b->guarded.clear();
}

// LBM_ECORRUPT if a byte of any guard band changed (a write outside its buffer).
int check_guards(Batch* b) {
  CK(b, cudaStreamSynchronize(b->stream));
  std::vector<unsigned char> h(2 * kGuard);
  for (const auto& g : b->guarded) {
    CK(b, cudaMemcpy(h.data(), g.base, kGuard, cudaMemcpyDeviceToHost));
    CK(b, cudaMemcpy(h.data() + kGuard, g.base + kGuard + g.bytes, kGuard,
                     cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < 2 * kGuard; ++k)
      if (h[k] != kCanary)
        return set_err(b->err, LBM_ECORRUPT, "%s: guard byte %s the buffer overwritten (%s %zu)",
                       g.name, k < kGuard ? "before" : "after",
                       k < kGuard ? "offset -" : "offset +",
                       k < kGuard ? kGuard - k : k - kGuard);
  }
  return LBM_OK;
}

void drop_graphs(Batch* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void destroy_batch(Batch* b) {
  if (!b) return;
  DeviceGuard g(b);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (cudaStream_t s : {b->up_stream, b->down_stream})  // copies may still use buffers
    if (s) cudaStreamSynchronize(s);
  drop_graphs(b);
  free_dev(b->d_inst);
  free_dev(b->d_items);
  free_dev(b->d_items2);
  free_dev(b->d_links2);
  free_dev(b->d_sync);
  free_dev(b->d_all_items);
  free_dev(b->d_item_begin);
  b->slab[0] = b->slab[1] = nullptr;  // guarded buffers
  b->rho_prev = nullptr;
  for (auto& f : b->fields) f = nullptr;
  b->staging = nullptr;
  b->staging32 = nullptr;
  b->staging_t = nullptr;
  free_guarded(b);
  free_dev(b->d_part_sum);
  free_dev(b->d_part_max);
  free_dev(b->d_part_bad);
  free_dev(b->d_diag);
  free_dev(b->d_status);
  free_dev(b->d_flag);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto& st : b->grp_stream)
    if (st) cudaStreamDestroy(st);
  for (auto& ev : b->grp_join)
    if (ev) cudaEventDestroy(ev);
  if (b->grp_fork) cudaEventDestroy(b->grp_fork);
  for (cudaStream_t s : {b->up_stream, b->down_stream})
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t ev : {b->ev_uploaded, b->ev_staging_free, b->ev_fields_ready, b->ev_fields_free})
    if (ev) cudaEventDestroy(ev);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  b->stream = nullptr;
}

bool per_instance(const Batch* b) { return b->nt == LBM_TILE_PER_INSTANCE; }

// Whether a tiling request is available for a precision.
bool tiling_ok(bool fp64, int nt, int vec) {
  if (nt == LBM_TILE_PER_INSTANCE) return !fp64 && vec == 2;
  return lbm::cfg_supported(fp64, nt, vec);
}

// Threads per CTA of the moments/diagnostics pass (one uniform tiling over all instances).
int mom_nt(const Batch* b) { return per_instance(b) ? 128 : b->nt; }

constexpr int kPairThreads[Batch::kMaxWidths] = {32, 64, 96, 128};
constexpr int kRowFixedCols = 57;  // per-row work of a strip row, in computed columns

// Pair-kernel width for an instance of nx columns: the least strip time, where a strip row
// of 2 nt - 4 owned columns costs its 2 nt computed columns plus a fixed 57
// column-equivalents (the per-row work that does not scale with width: copy issue,
// barrier, halo columns, the instance's ghost columns; fitted to batches of equal
// instances that fill their strips exactly, 60, 124 and 252 columns wide, at 45.9, 64.1
// and 74.4 GLUPS).  Ties go to the wider CTA.
int pair_threads_for(int nx) {
  int best = 128;
  long long best_cost = -1;
  for (int g = Batch::kMaxWidths - 1; g >= 0; --g) {
    const int nt = kPairThreads[g];
    const long long cost = (long long)lbm::strips_for(nx, nt, 2) * (2 * nt + kRowFixedCols);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = nt;
    }
  }
  return best;
}

// Modelled time of one lattice row of nx columns at a tiling (threads nt, columns per
// thread vec, or the per-instance pair width): its strips' computed columns plus the fixed
// per-row work of each strip.
long long row_cost(int nx, int nt, int vec) {
  if (nt == LBM_TILE_PER_INSTANCE) {
    nt = pair_threads_for(nx);
    vec = 2;
  }
  return (long long)lbm::strips_for(nx, nt, vec) * (nt * vec + kRowFixedCols);
}

// Orientation of an instance: LBM_LAYOUT_AUTO stores a periodic instance of at least 8 x 8
// nodes transposed when its ny-column rows cost less in total than its nx-column rows
// (ties keep the given orientation).  The update is symmetric under x <-> y only without
// walls, which are along y.
bool transposed_layout(const lbm_instance& in, int nt, int vec) {
  if (in.layout == LBM_LAYOUT_TRANSPOSED) return true;
  if (in.layout != LBM_LAYOUT_AUTO || in.bc != LBM_BC_PERIODIC || in.nx < 8 || in.ny < 8)
    return false;
  return row_cost(in.ny, nt, vec) * in.nx < row_cost(in.nx, nt, vec) * in.ny;
}

// Step-kernel threads per CTA of instance i under the current tiling.
int step_nt(const Batch* b, int i) { return per_instance(b) ? b->inst_nt[i] : b->nt; }

// LBM_PERSISTENT in the environment: 0 never steps persistently, 2 whenever the
// dependency rule allows (even with few items per step; for tests), anything else (the
// default) when there are enough items per step.
int persist_env() {
  const char* env = std::getenv("LBM_PERSISTENT");
  return env ? std::atoi(env) : 1;
}

// Whether persistent stepping may be used at all: FP32 pair tilings, unless switched off
// (by the environment, or by the autotuner's choice for the tiling in use).
bool persist_allowed(const Batch* b) {
  return !b->fp64 && b->vec == 2 && persist_env() != 0 && !b->persist_off;
}

// Kind of persistent launch (sweep2_persist_kernel) the active instances allow: all of
// one kernel width, swept in strips (PERSIST_STRIP), in full-width strips (PERSIST_FULL)
// or both (PERSIST_MIXED, the two launch groups in one launch); -1 with several widths
// (per-instance tilings) or no active instance.  *nt receives the width.
int persist_kind(const Batch* b, int* nt_out = nullptr) {
  int nt = 0;
  bool strip = false, full = false;
  for (int i = 0; i < b->n_inst; ++i)
    if (b->active[i]) {
      const int w = step_nt(b, i);
      if (nt != 0 && w != nt) return -1;
      nt = w;
      (lbm::full_width(b->inst[i].nx, nt, b->vec) ? full : strip) = true;
    }
  if (nt_out) *nt_out = nt;
  if (nt == 0) return -1;
  return strip && full ? lbm::PERSIST_MIXED : full ? lbm::PERSIST_FULL : lbm::PERSIST_STRIP;
}

// Whether chunks of `rows` rows give the active instances at least two waves of step items
// (resident persistent CTAs): with fewer, a step's first items would wait on the previous
// step's last ones, since the odd steps' lists start only half a step further on (the
// 1024^2 ellipse, 640 items per step against 760 resident CTAs, stepped at 48 against 53
// GLUPS persistently).
bool persist_items_ok(const Batch* b, int rows) {
  int nt = 0;
  const int kind = persist_kind(b, &nt);
  if (kind < 0) return false;
  long long items = 0;
  for (int i = 0; i < b->n_inst; ++i)
    if (b->active[i])
      items += (long long)lbm::strips_for(b->inst[i].nx, nt, b->vec) *
               ((b->inst[i].ny + rows - 1) / rows);
  return items >= 2LL * lbm::persist_occupancy(nt, kind) * std::max(b->sms, 1);
}

// Rows per CTA sweep: about six waves of resident CTAs (measured best on 4096^2: fewer
// rows cost halo re-reads and row-loop start-up, more rows leave SMs idle in the tail),
// clamped to [8, 64] for FP32 and [1, 64] for FP64, whose rows are FP64-pipe bound: on a
// 128^2 FP64 lattice one-row chunks spread the work over 4x more SMs (1.0 against 0.27
// GLUPS), while FP32 lattices of 1M nodes lose 20-40 % below 8 rows.  With per-instance
// widths each strip row counts as 1 / (resident CTAs of its width) of an SM.
int default_rows(const Batch* b) {
  double sm_rows = 0.0;
  for (int i = 0; i < b->n_inst; ++i)
    if (b->active[i]) {
      const int nt = step_nt(b, i);
      const int occ = b->fp64 ? lbm::sweep_occupancy<double>(nt, b->vec)
                              : lbm::sweep_occupancy<float>(nt, b->vec);
      sm_rows += (double)lbm::strips_for(b->inst[i].nx, nt, b->vec) * b->inst[i].ny /
                 std::max(occ, 1);
    }
  const long long lo = b->fp64 ? 1 : 8;
  auto clamp = [&](long long r) { return (int)std::min<long long>(64, std::max(lo, r)); };
  const int r6 = clamp((long long)std::ceil(sm_rows / ((double)std::max(b->sms, 1) * 6.0)));
  // Persistent stepping has no drain between steps, so fewer, taller chunks (fewer halo
  // rows) win: about three waves, rounded up to a multiple of four rows (32 rows at 4096^2,
  // 87.5 against 84.0 GLUPS at 16 rows per step), if that still gives the two waves of
  // items per step that persistent stepping needs (persist_items_ok).
  if (persist_allowed(b) && persist_kind(b) >= 0) {
    const long long r3 = (long long)std::ceil(sm_rows / ((double)std::max(b->sms, 1) * 3.0));
    const int rp = clamp((r3 + 3) / 4 * 4);
    if (persist_items_ok(b, rp)) return rp;
  }
  return r6;
}

// Work items of instance i: strips of W owned columns by chunks of `rows` rows.
void append_items(const InstParams& P, int i, int nt, int vec, int rows,
                  std::vector<WorkItem>& out) {
  const int W = lbm::strip_width(nt, vec);
  const int strips = lbm::strips_for(P.nx, nt, vec);
  const int chunks = (P.ny + rows - 1) / rows;
  for (int c = 0; c < chunks; ++c)
    for (int s = 0; s < strips; ++s) {
      WorkItem w{};
      w.inst = i;
      w.x0 = s * W;
      w.y0 = c * rows;
      w.y1 = std::min(P.ny, (c + 1) * rows);
      w.dir = (c & 1) ? -1 : 1;
      out.push_back(w);
    }
}

// Step items of the active instances, grouped by kernel width and, within a width, by
// strip and full-width instances (b->items, b->grp_*).
void make_step_items(Batch* b) {
  b->items.clear();
  b->n_groups = 0;
  b->grp_begin[0] = 0;
  for (int g = 0; g < Batch::kMaxWidths; ++g) {
    const int nt = per_instance(b) ? kPairThreads[g] : b->nt;
    for (int full = 0; full < 2; ++full) {
      const size_t before = b->items.size();
      for (int i = 0; i < b->n_inst; ++i)
        if (b->active[i] && step_nt(b, i) == nt &&
            (int)lbm::full_width(b->inst[i].nx, nt, b->vec) == full)
          append_items(b->inst[i], i, nt, b->vec, b->rows, b->items);
      if (b->items.size() > before) {
        b->grp_nt[b->n_groups] = nt;
        b->grp_full[b->n_groups] = full;
        b->grp_begin[++b->n_groups] = (int)b->items.size();
      }
    }
    if (!per_instance(b)) break;
  }
}

// Items of every instance for the moments/diagnostics pass, with per-instance ranges.
void make_all_items(const Batch* b, std::vector<WorkItem>& out, std::vector<int>& begin) {
  out.clear();
  begin.assign(1, 0);
  for (int i = 0; i < b->n_inst; ++i) {
    append_items(b->inst[i], i, mom_nt(b), b->vec, b->rows, out);
    begin.push_back((int)out.size());
  }
}

// Work lists of the persistent step kernel (sweep2_persist_kernel) for the current step
// items: the even steps' list (the step items in their order), the odd steps' (each
// instance's chunk rows from the middle one on, wrapping), the dependency links, the
// counters and the grid (the resident CTAs).  Used for FP32 pair tilings of one kernel
// width (persist_kind: a batch's strip and full-width launch groups share the launch) and
// at least two waves of items per step (persist_items_ok), unless switched off
// (persist_env), and only when every item depends on at most four chunks (chunks of two
// rows or more, but for a short last one); otherwise steps are one launch per group each.
// (Several groups, each persistent with its share of the CTAs, ran at 58.9 against 67.3
// GLUPS as per-step graph branches on the 256-instance batch.)
// Persistent work lists of the step items [lo, hi) of `items` (an instance's items
// consecutive, chunk rows in order of `rows` rows each, `strips` items per chunk row) into
// items2 / links2 (2 (hi - lo) entries: the even steps' list, then the odd steps', which
// visits each instance's chunk rows from the middle one on).  Chunk ids count from 0 over
// the instances of the range; *n_chunks receives their number, rowwork (may be NULL) the
// rows its items load.  False if an item would depend on more than four chunks (chunks of
// one row): the items then cannot step persistently.  Host code only.
bool plan_persist_list(const std::vector<WorkItem>& items, int lo, int hi,
                        const std::vector<InstParams>& inst, int rows, WorkItem* items2,
                        ItemLink* links2, int* n_chunks, double* rowwork) {
  const int ng = hi - lo;
  int chunk0 = 0;  // id of the first chunk of the current instance
  double work = 0.0;
  for (int k = lo; k < hi;) {
    const int i = items[k].inst;
    const InstParams& P = inst[i];
    int e = k, strips = 0;
    while (e < hi && items[e].inst == i) ++e;
    while (k + strips < e && items[k + strips].y0 == items[k].y0) ++strips;
    const int nch = (e - k) / strips;
    if (nch * strips != e - k) return false;
    for (int c = 0; c < nch; ++c) {
      const int co = (c + nch / 2) % nch;  // the odd steps' c-th chunk row
      for (int sx = 0; sx < strips; ++sx) {
        const int pos = k + c * strips + sx - lo;
        for (int par = 0; par < 2; ++par) {
          const int cc = par ? co : c;
          const WorkItem& w = items[k + cc * strips + sx];
          ItemLink ln{};
          ln.chunk = chunk0 + cc;
          ln.strips = strips;
          int nd = 0;
          // the chunks holding the rows it reads: its own and two beyond each end
          // (wrapped, or clamped at walls); by symmetry also those that read its rows
          for (int r = w.y0 - 2; r <= w.y1 + 1; ++r) {
            const int rr = P.walls ? std::min(std::max(r, 0), P.ny - 1)
                                   : ((r % P.ny) + P.ny) % P.ny;
            const int d = chunk0 + std::min(rr / rows, nch - 1);
            bool seen = false;
            for (int j = 0; j < nd; ++j) seen |= ln.dep[j] == d;
            if (seen) continue;
            if (nd == 4) return false;
            ln.dep[nd++] = d;
          }
          for (int j = nd; j < 4; ++j) ln.dep[j] = ln.dep[0];
          items2[(size_t)par * ng + pos] = w;
          links2[(size_t)par * ng + pos] = ln;
        }
        work += items[k + c * strips + sx].y1 - items[k + c * strips + sx].y0 + 4;
      }
    }
    chunk0 += nch;
    k = e;
  }
  *n_chunks = chunk0;
  if (rowwork) *rowwork = work;
  return true;
}

int build_persist(Batch* b) {
  b->persist = false;
  int nt = 0;
  const int kind = persist_kind(b, &nt);
  if (!persist_allowed(b) || b->n_items == 0 || kind < 0 ||
      (persist_env() != 2 && !persist_items_ok(b, b->rows)))
    return LBM_OK;
  const int n = b->n_items;
  std::vector<WorkItem> items2(2 * (size_t)n);
  std::vector<ItemLink> links2(2 * (size_t)n);
  int nch = 0;
  if (!plan_persist_list(b->items, 0, n, b->inst, b->rows, items2.data(), links2.data(), &nch,
                         nullptr))
    return LBM_OK;  // too many dependencies: no persistent stepping
  const int sync = 1 + nch;  // the queue counter, then the chunk counters
  b->persist_kind = kind;
  b->persist_sync = sync;
  b->persist_grid =
      std::max(1, std::min(lbm::persist_occupancy(nt, kind) * std::max(b->sms, 1), n));
  if (2 * n > b->cap_items2 || !b->d_items2) {
    free_dev(b->d_items2);
    free_dev(b->d_links2);
    b->cap_items2 = 0;
    CK(b, dev_malloc(&b->d_items2, sizeof(WorkItem) * 2 * n));
    CK(b, dev_malloc(&b->d_links2, sizeof(ItemLink) * 2 * n));
    b->cap_items2 = 2 * n;
  }
  if (sync > b->cap_sync || !b->d_sync) {
    free_dev(b->d_sync);
    b->cap_sync = 0;
    CK(b, dev_malloc(&b->d_sync, sizeof(int) * sync));
    b->cap_sync = sync;
  }
  CK(b, cudaMemcpy(b->d_items2, items2.data(), sizeof(WorkItem) * 2 * n, cudaMemcpyHostToDevice));
  CK(b, cudaMemcpy(b->d_links2, links2.data(), sizeof(ItemLink) * 2 * n, cudaMemcpyHostToDevice));
  b->persist = true;
  return LBM_OK;
}

// Rebuild and upload the work lists (after a tiling change or a retirement).
int rebuild_items(Batch* b) {
  drop_graphs(b);
  if (b->stream) CK(b, cudaStreamSynchronize(b->stream));
  if (per_instance(b)) {
    b->inst_nt.resize(b->n_inst);
    for (int i = 0; i < b->n_inst; ++i) b->inst_nt[i] = pair_threads_for(b->inst[i].nx);
  }
  b->rows = b->rows_req > 0 ? b->rows_req : default_rows(b);
  make_step_items(b);
  make_all_items(b, b->all_items, b->item_begin);
  b->n_items = (int)b->items.size();
  const int n_all = (int)b->all_items.size();
  if (n_all > b->cap_all || !b->d_all_items) {
    free_dev(b->d_all_items);
    free_dev(b->d_part_sum);
    free_dev(b->d_part_max);
    free_dev(b->d_part_bad);
    b->cap_all = 0;
    CK(b, dev_malloc(&b->d_all_items, sizeof(WorkItem) * std::max(n_all, 1)));
    CK(b, dev_malloc(&b->d_part_sum, sizeof(double) * 3 * std::max(n_all, 1)));
    CK(b, dev_malloc(&b->d_part_max, sizeof(float) * 2 * std::max(n_all, 1)));
    CK(b, dev_malloc(&b->d_part_bad, sizeof(int) * std::max(n_all, 1)));
    b->cap_all = n_all;
  }
  // Step items can outnumber the moments items (narrower strips under per-instance widths).
  if (b->n_items > b->cap_items || !b->d_items) {
    free_dev(b->d_items);
    b->cap_items = 0;
    CK(b, dev_malloc(&b->d_items, sizeof(WorkItem) * std::max(b->n_items, 1)));
    b->cap_items = b->n_items;
  }
  b->n_all = n_all;
  CK(b, cudaMemcpy(b->d_all_items, b->all_items.data(), sizeof(WorkItem) * n_all,
                   cudaMemcpyHostToDevice));
  if (b->n_items)
    CK(b, cudaMemcpy(b->d_items, b->items.data(), sizeof(WorkItem) * b->n_items,
                     cudaMemcpyHostToDevice));
  if (!b->d_item_begin) CK(b, dev_malloc(&b->d_item_begin, sizeof(int) * (b->n_inst + 1)));
  CK(b, cudaMemcpy(b->d_item_begin, b->item_begin.data(), sizeof(int) * (b->n_inst + 1),
                   cudaMemcpyHostToDevice));
  {
    int rc = build_persist(b);
    if (rc) return rc;
  }
  // Full-width strips of the pair kernel neither read nor write the ghost columns, so
  // after steps under one set of work lists they may be stale; a pass under the new lists
  // may use strips that read them.
  if (!b->fp64 && b->slab[b->cur])
    for (int i = 0; i < b->n_inst; ++i)
      CK(b, lbm::launch_fill_ghosts<float>((float*)b->slab[b->cur], b->inst[i], b->stream));
  return LBM_OK;
}

// Fill the device parameters of one instance; validates the physical arguments.
int fill_params(std::string& err, InstParams& P, const lbm_instance& in, bool fp64,
                int psi_fp64) {
  if (in.nx < 1 || in.ny < 1) return set_err(err, LBM_EINVAL, "nx, ny must be >= 1");
  if (!(in.eos.a > 0) || !(in.eos.b > 0) || !(in.eos.R > 0) || !(in.eos.T > 0))
    return set_err(err, LBM_EINVAL, "EOS parameters a, b, R, T must be positive");
  if (!(in.G != 0) || !std::isfinite(in.G)) return set_err(err, LBM_EINVAL, "G must be nonzero");
  if (!std::isfinite(in.sigma)) return set_err(err, LBM_EINVAL, "sigma must be finite");
  for (int i = 0; i < 9; ++i)
    if (!(in.s[i] > 0 && in.s[i] < 2))
      return set_err(err, LBM_EINVAL, "s[%d] = %g is not in (0, 2)", i, in.s[i]);
  if (in.visc_mode < LBM_VISC_CONST || in.visc_mode > LBM_VISC_LINEAR)
    return set_err(err, LBM_EINVAL, "unknown viscosity mode %d", in.visc_mode);
  if (in.visc_mode != LBM_VISC_CONST && !(in.nu_l > 0 && in.nu_v > 0))
    return set_err(err, LBM_EINVAL, "nu_l and nu_v must be positive for this viscosity mode");
  if (in.bc != LBM_BC_PERIODIC && in.bc != LBM_BC_WALLS_Y)
    return set_err(err, LBM_EINVAL, "unknown boundary %d", in.bc);
  std::memset(&P, 0, sizeof P);
  P.nx = in.nx;
  P.ny = in.ny;
  P.pitch = (int)round_up((size_t)in.nx + 2 * lbm::GHOST, 8);
  P.plane = (long long)in.ny * P.pitch;
  P.walls = in.bc == LBM_BC_WALLS_Y;
  P.visc_mode = in.visc_mode;
  P.psi_fp64 = fp64 ? 0 : psi_fp64;
  P.b4 = in.eos.b / 4.0;
  P.RT = in.eos.R * in.eos.T;
  P.a = in.eos.a;
  P.two_over_G = 2.0 / in.G;
  P.G = in.G;
  for (int i = 0; i < 9; ++i) P.s[i] = in.s[i];
  P.sig12_e = 12.0 * in.sigma * in.s[1];
  P.sig12_z = 12.0 * in.sigma * in.s[2];
  P.tau_l = 3.0 * in.nu_l + 0.5;
  P.tau_v = 3.0 * in.nu_v + 0.5;
  P.rho_c = in.rho_c > 0 ? in.rho_c : 0.5218 / in.eos.b;
  double rl = in.rho_l, rv = in.rho_v;
  const bool need_maxwell = (in.visc_mode == LBM_VISC_LINEAR && (rl <= 0 || rv <= 0)) ||
                            (!fp64 && in.rho_ref < 0);
  double ml = 0, mv = 0;
  const bool have_maxwell = need_maxwell && lbm_maxwell(in.eos, &ml, &mv) == LBM_OK;
  if (in.visc_mode == LBM_VISC_LINEAR) {
    if (rl <= 0 || rv <= 0) {
      if (!have_maxwell)
        return set_err(err, LBM_EINVAL,
                       "LINEAR viscosity needs rho_l, rho_v (no Maxwell solution at this T)");
      rl = ml;
      rv = mv;
    }
    if (!(rl > rv)) return set_err(err, LBM_EINVAL, "LINEAR viscosity needs rho_l > rho_v");
  }
  P.rho_l = rl;
  P.rho_v = rv;
  P.rho_ref = fp64 ? 0.0 : (in.rho_ref >= 0 ? in.rho_ref : (have_maxwell ? mv : 0.0));
  fill_mirror(P.pf, P);
  fill_mirror(P.pd, P);
  return LBM_OK;
}


int create_batch(Batch* b, int n, const lbm_instance* in, bool fp64, int psi_fp64,
                 void* stream, int device, int nt, int vec, int rows) {
  if (n < 1 || !in) return set_err(b->err, LBM_EINVAL, "need at least one instance");
  const int nt_ = nt ? nt : default_threads(fp64), vec_ = vec ? vec : default_vec(fp64);
  if (!tiling_ok(fp64, nt_, vec_))
    return set_err(b->err, LBM_EINVAL,
                   "tile_threads %d with tile_vec %d is not available for this precision", nt_,
                   vec_);
  if (rows < 0) return set_err(b->err, LBM_EINVAL, "tile_rows must be >= 0");
  b->fp64 = fp64;
  b->esz = fp64 ? sizeof(double) : sizeof(float);
  b->n_inst = n;
  b->inst.resize(n);
  b->tr.assign(n, 0);
  b->active.assign(n, 1);
  b->steps.assign(n, 0);
  b->dinf_valid.assign(n, 0);
  size_t off = 0, dense = 0;
  for (int i = 0; i < n; ++i) {
    lbm_instance li = in[i];
    if (li.layout < LBM_LAYOUT_AUTO || li.layout > LBM_LAYOUT_TRANSPOSED)
      return set_err(b->err, LBM_EINVAL, "instance %d: unknown layout %d", i, li.layout);
    if (li.layout == LBM_LAYOUT_TRANSPOSED && li.bc != LBM_BC_PERIODIC)
      return set_err(b->err, LBM_EINVAL,
                     "instance %d: an instance with walls cannot be stored transposed", i);
    if (transposed_layout(li, nt_, vec_)) {
      std::swap(li.nx, li.ny);
      b->tr[i] = 1;
    }
    int rc = fill_params(b->err, b->inst[i], li, fp64, psi_fp64);
    if (rc) return rc;
    b->inst[i].off = (long long)off;
    b->inst[i].dense_off = (long long)dense;
    // Keep every instance's block 256-byte aligned.
    off += round_up((size_t)9 * (size_t)b->inst[i].plane, 64);
    dense += (size_t)in[i].nx * (size_t)in[i].ny;
  }
  b->slab_elems = off;
  b->dense_elems = dense;
  b->nt = nt_;
  b->vec = vec_;
  b->rows_req = rows;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
    return set_err(b->err, LBM_ECUDA, "no CUDA device available");
  int dev = 0;
  if (device >= 0) {
    if (device >= dev_count) return set_err(b->err, LBM_EINVAL, "device %d out of range", device);
    CK(b, cudaSetDevice(device));
  }
  CK(b, cudaGetDevice(&dev));
  b->device = dev;
  CK(b, cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    CK(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  CK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    int rc = guarded_alloc(b, &b->slab[k], b->slab_elems * b->esz,
                           k == 0 ? "population slab 0" : "population slab 1");
    if (rc) return rc;
    CK(b, cudaMemsetAsync(b->slab[k], 0, b->slab_elems * b->esz, b->stream));
  }
  {
    int rc = guarded_alloc(b, &b->rho_prev, std::max<size_t>(b->dense_elems, 1) * b->esz,
                           "previous density");
    if (rc) return rc;
  }
  CK(b, dev_malloc(&b->d_inst, sizeof(InstParams) * n));
  CK(b, cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(InstParams) * n,
                        cudaMemcpyHostToDevice, b->stream));
  CK(b, dev_malloc(&b->d_diag, sizeof(double) * 6 * n));
  CK(b, dev_malloc(&b->d_status, sizeof(int)));
  CK(b, cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  return rebuild_items(b);
}

// One step of the instances of launch group g, from slab c into slab c ^ 1.
int launch_group(Batch* b, int g, int c, cudaStream_t st) {
  const WorkItem* items = b->d_items + b->grp_begin[g];
  const int n = b->grp_begin[g + 1] - b->grp_begin[g];
  cudaError_t e;
  if (b->fp64) {
    MomArgs<double> mo{};
    e = lbm::launch_sweep<double>(b->grp_nt[g], b->vec, lbm::MODE_STEP, 0,
                                  (const double*)b->slab[c], (double*)b->slab[c ^ 1], b->d_inst,
                                  items, n, mo, b->d_status, st);
  } else {
    MomArgs<float> mo{};
    e = lbm::launch_sweep<float>(b->grp_nt[g], b->vec, lbm::MODE_STEP, b->grp_full[g],
                                 (const float*)b->slab[c], (float*)b->slab[c ^ 1], b->d_inst,
                                 items, n, mo, b->d_status, st);
  }
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "step kernel launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// n steps (at most kGraphSteps) of every active instance from slab c as one persistent
// launch on st, after zeroing the queue and chunk counters.
int launch_persist_steps(Batch* b, int c, int n, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(int) * b->persist_sync, st);
  if (e == cudaSuccess)
    e = lbm::launch_persist(b->grp_nt[0], b->persist_kind, (float*)b->slab[c],
                            (float*)b->slab[c ^ 1], b->d_inst, b->d_items2, b->d_links2,
                            b->n_items, n, b->d_sync, b->d_sync + 1, b->d_status,
                            b->persist_grid, lbm::DEP_WAIT_LIMIT, st);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "persistent step launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// One step of every active instance: the launch groups one after another on st.
int launch_step(Batch* b, cudaStream_t st) {
  for (int g = 0; g < b->n_groups; ++g) {
    int rc = launch_group(b, g, b->cur, st);
    if (rc) return rc;
  }
  b->cur ^= 1;
  return LBM_OK;
}

// Streams and events that fork the launch groups into parallel graph branches.
int ensure_branches(Batch* b) {
  for (int g = 0; g + 1 < b->n_groups; ++g) {
    if (!b->grp_stream[g])
      CK(b, cudaStreamCreateWithFlags(&b->grp_stream[g], cudaStreamNonBlocking));
    if (!b->grp_join[g])
      CK(b, cudaEventCreateWithFlags(&b->grp_join[g], cudaEventDisableTiming));
  }
  if (!b->grp_fork) CK(b, cudaEventCreateWithFlags(&b->grp_fork, cudaEventDisableTiming));
  return LBM_OK;
}

// n steps queued on st.  With several launch groups (which touch disjoint instances) each
// group runs its chain of n launches on its own stream, forked from st and joined back,
// so the groups overlap on the GPU and fill each other's tails.  b->cur is unchanged.
int queue_steps(Batch* b, int n, cudaStream_t st) {
  const int start = b->cur;
  if (b->persist) return n > 0 ? launch_persist_steps(b, start, n, st) : LBM_OK;
  if (b->n_groups <= 1) {
    int rc = LBM_OK;
    for (int k = 0; k < n && rc == LBM_OK; ++k) rc = launch_step(b, st);
    b->cur = start;
    return rc;
  }
  int rc = ensure_branches(b);
  if (rc) return rc;
  cudaError_t e = cudaEventRecord(b->grp_fork, st);
  for (int k = 0; k + 1 < b->n_groups && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->grp_stream[k], b->grp_fork, 0);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "stream fork failed: %s", cudaGetErrorString(e));
  for (int gi = 0; gi < b->n_groups && rc == LBM_OK; ++gi) {
    cudaStream_t sg = gi == 0 ? st : b->grp_stream[gi - 1];
    for (int k = 0; k < n && rc == LBM_OK; ++k) rc = launch_group(b, gi, start ^ (k & 1), sg);
  }
  // Join every branch that was forked, even after a failed launch.
  for (int k = 0; k + 1 < b->n_groups; ++k) {
    e = cudaEventRecord(b->grp_join[k], b->grp_stream[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->grp_join[k], 0);
    if (e != cudaSuccess && rc == LBM_OK)
      rc = set_err(b->err, LBM_ECUDA, "stream join failed: %s", cudaGetErrorString(e));
  }
  return rc;
}

// Capture kGraphSteps consecutive steps that start from slab `start` (one branch per
// launch group).
int capture_graph(Batch* b, int start) {
  const int saved = b->cur;
  if (b->n_groups > 1) {
    int rc = ensure_branches(b);  // created outside the capture
    if (rc) return rc;
  }
  b->cur = start;
  cudaGraph_t g = nullptr;
  CK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = queue_steps(b, kGraphSteps, b->cap_stream);
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  b->cur = saved;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph[start] = nullptr;
    return set_err(b->err, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  return LBM_OK;
}

int do_steps(Batch* b, long long n) {
  if (n < 0) return set_err(b->err, LBM_EINVAL, "step count must be >= 0");
  if (b->n_items == 0) return LBM_OK;
  const long long n0 = n;
  while (n > 0) {
    if (n >= kGraphSteps) {
      if (!b->graph[b->cur]) {
        int rc = capture_graph(b, b->cur);
        if (rc) return rc;
      }
      CK(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
      n -= kGraphSteps;
    } else {
      int rc = queue_steps(b, (int)n, b->stream);
      if (rc) return rc;
      b->cur ^= (int)(n & 1);
      n = 0;
    }
  }
  for (int i = 0; i < b->n_inst; ++i)
    if (b->active[i]) b->steps[i] += n0;
  return LBM_OK;
}

int sync_status(Batch* b) {
  CK(b, cudaStreamSynchronize(b->stream));
  if (b->up_stream) CK(b, cudaStreamSynchronize(b->up_stream));
  if (b->down_stream) CK(b, cudaStreamSynchronize(b->down_stream));
  int st = 0;
  CK(b, cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & lbm::STATUS_BADINIT)
    return set_err(b->err, LBM_EINVAL,
                   "the last initialisation had nodes with a density outside (0, 4/b), a "
                   "negative psi^2 (Eq. 24) or a non-finite velocity");
  if (st & lbm::STATUS_BOUNDS)
    return set_err(b->err, LBM_ECORRUPT,
                   "a kernel index check failed (bounds-check build): an access outside its "
                   "buffer was skipped");
  if (st & lbm::STATUS_TIMEOUT)
    return set_err(b->err, LBM_ETIMEOUT,
                   "a bounded wait for a shared-memory copy ran out in the step kernel");
  if (st & lbm::STATUS_NONFINITE)
    return set_err(b->err, LBM_EUNSTABLE,
                   "a density became non-finite or non-positive during stepping");
  return LBM_OK;
}

// Device scratch of `bytes`, freed by the caller.
int dev_alloc(Batch* b, void** p, size_t bytes) {
  CK(b, dev_malloc(p, std::max<size_t>(bytes, 16)));
  return LBM_OK;
}

// Device doubles for 3 fields of the largest instance, kept for the handle's lifetime
// (host transfers go through it without per-call allocation).
int ensure_staging(Batch* b) {
  if (b->staging) return LBM_OK;
  size_t m = 1;
  for (const auto& P : b->inst) m = std::max(m, (size_t)P.nx * P.ny);
  int rc = guarded_alloc(b, (void**)&b->staging, 3 * m * sizeof(double), "staging");
  if (rc) return rc;
  b->staging_elems = m;
  return LBM_OK;
}

// Device floats for 3 fields of the largest instance (float host transfers).
int ensure_staging32(Batch* b) {
  if (b->staging32) return LBM_OK;
  int rc = ensure_staging(b);  // sets staging_elems
  if (rc) return rc;
  return guarded_alloc(b, (void**)&b->staging32, 3 * b->staging_elems * sizeof(float),
                       "float staging");
}

// Device doubles for 3 fields of the largest transposed instance (its initialisation
// fields in the stored orientation).
int ensure_staging_t(Batch* b) {
  if (b->staging_t) return LBM_OK;
  size_t m = 1;
  for (int i = 0; i < b->n_inst; ++i)
    if (b->tr[i]) m = std::max(m, (size_t)b->inst[i].nx * b->inst[i].ny);
  int rc = guarded_alloc(b, (void**)&b->staging_t, 3 * m * sizeof(double),
                         "transposed staging");
  if (rc) return rc;
  b->staging_t_elems = m;
  return LBM_OK;
}

int ensure_flag(Batch* b) {
  if (!b->d_flag) CK(b, dev_malloc(&b->d_flag, sizeof(int)));
  return LBM_OK;
}

int init_instance(Batch* b, int i, const double* rho, const double* ux, const double* uy,
                  bool device_ptrs) {
  if (i < 0 || i >= b->n_inst) return set_err(b->err, LBM_EINVAL, "instance %d out of range", i);
  if (!rho) return set_err(b->err, LBM_EINVAL, "rho must not be NULL");
  const InstParams& P = b->inst[i];
  const size_t N = (size_t)P.nx * P.ny;
  const double *dr = rho, *du = ux, *dv = uy;
  int rc = ensure_flag(b);
  if (rc) return rc;
  int* dbad = b->d_flag;
  if (!device_ptrs) {
    rc = ensure_staging(b);
    if (rc) return rc;
    double* t = b->staging;
    cudaMemcpyAsync(t, rho, N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    dr = t;
    t += N;
    if (ux) {
      cudaMemcpyAsync(t, ux, N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      du = t;
      t += N;
    }
    if (uy) {
      cudaMemcpyAsync(t, uy, N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      dv = t;
    }
  }
  if (b->tr[i]) {
    // Fields in the given orientation (P.nx rows of P.ny values) into the stored one; the
    // stored x velocity is the given y velocity and vice versa.
    rc = ensure_staging_t(b);
    if (rc) return rc;
    double* t = b->staging_t;
    const double* src[3] = {dr, dv, du};
    const double* dst[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
      if (!src[k]) continue;
      double* d = t + k * b->staging_t_elems;
      CK(b, (lbm::launch_transpose<double, double>(src[k], d, P.ny, P.nx, b->stream)));
      dst[k] = d;
    }
    dr = dst[0];
    du = dst[1];
    dv = dst[2];
  }
  cudaMemsetAsync(dbad, 0, sizeof(int), b->stream);
  cudaError_t e;
  if (b->fp64)
    e = lbm::launch_init_eq<double>(dr, du, dv, (double*)b->slab[b->cur], P, dbad, b->stream);
  else
    e = lbm::launch_init_eq<float>(dr, du, dv, (float*)b->slab[b->cur], P, dbad, b->stream);
  if (e == cudaSuccess)
    e = b->fp64 ? lbm::launch_fill_ghosts<double>((double*)b->slab[b->cur], P, b->stream)
                : lbm::launch_fill_ghosts<float>((float*)b->slab[b->cur], P, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
  // Nothing is copied into the other slab: the next step of an active instance writes
  // every column it later reads there (the interior and the ghost pairs), and an instance
  // is copied into both slabs when it is frozen (lbm_batch_run_to_equilibrium).
  b->steps[i] = 0;
  b->dinf_valid[i] = 0;
  if (!b->active[i]) {
    b->active[i] = 1;
    rc = rebuild_items(b);
    if (rc) return rc;
  }
  if (bad)
    return set_err(b->err, LBM_EINVAL,
                   "%d nodes have a density outside (0, 4/b), a negative psi^2 (Eq. 24) or "
                   "a non-finite velocity", bad);
  return LBM_OK;
}

// init_instance from host floats: one transfer of floats per field, widened to double on
// the device, then the double path.
int init_instance_f32(Batch* b, int i, const float* rho, const float* ux, const float* uy) {
  if (i < 0 || i >= b->n_inst) return set_err(b->err, LBM_EINVAL, "instance %d out of range", i);
  if (!rho) return set_err(b->err, LBM_EINVAL, "rho must not be NULL");
  int rc = ensure_staging32(b);
  if (rc) return rc;
  const size_t N = (size_t)b->inst[i].nx * b->inst[i].ny;
  const float* in[3] = {rho, ux, uy};
  const double* dev[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    float* f = b->staging32 + k * b->staging_elems;
    double* d = b->staging + k * b->staging_elems;
    CK(b, cudaMemcpyAsync(f, in[k], N * sizeof(float), cudaMemcpyHostToDevice, b->stream));
    CK(b, lbm::launch_widen(f, d, (long long)N, b->stream));
    dev[k] = d;
  }
  return init_instance(b, i, dev[0], dev[1], dev[2], true);
}

int set_pops(Batch* b, int i, const double* f) {
  if (!f) return set_err(b->err, LBM_EINVAL, "f must not be NULL");
  const InstParams& P = b->inst[i];
  const size_t N = (size_t)P.nx * P.ny;
  void* tmp = nullptr;
  int rc = dev_alloc(b, &tmp, 9 * N * sizeof(double));
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(tmp, f, 9 * N * sizeof(double), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess)
    e = b->fp64 ? lbm::launch_set_pops<double>((double*)tmp, (double*)b->slab[b->cur], P, b->stream)
                : lbm::launch_set_pops<float>((double*)tmp, (float*)b->slab[b->cur], P, b->stream);
  if (e == cudaSuccess)
    e = b->fp64 ? lbm::launch_fill_ghosts<double>((double*)b->slab[b->cur], P, b->stream)
                : lbm::launch_fill_ghosts<float>((float*)b->slab[b->cur], P, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((char*)b->slab[b->cur ^ 1] + P.off * b->esz,
                        (char*)b->slab[b->cur] + P.off * b->esz, 9 * P.plane * b->esz,
                        cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(tmp);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "set populations failed: %s", cudaGetErrorString(e));
  b->steps[i] = 0;
  b->dinf_valid[i] = 0;
  return LBM_OK;
}

// Direction of D2Q9 velocity q with its components exchanged (x <-> y): 1 <-> 2, 3 <-> 4,
// 6 <-> 8.
constexpr int kSwapXY[9] = {0, 2, 1, 4, 3, 5, 8, 7, 6};

int get_pops(Batch* b, int i, double* f) {
  if (!f) return set_err(b->err, LBM_EINVAL, "f must not be NULL");
  const InstParams& P = b->inst[i];
  const size_t N = (size_t)P.nx * P.ny;
  const bool t = b->tr[i];
  void* tmp = nullptr;
  int rc = dev_alloc(b, &tmp, (t ? 18 : 9) * N * sizeof(double));
  if (rc) return rc;
  cudaError_t e = b->fp64
      ? lbm::launch_get_pops<double>((const double*)b->slab[b->cur], (double*)tmp, P, b->stream)
      : lbm::launch_get_pops<float>((const float*)b->slab[b->cur], (double*)tmp, P, b->stream);
  const double* out = (const double*)tmp;
  if (t) {
    // plane q of the given orientation is the stored plane of q's mirror image, transposed
    double* g = (double*)tmp + 9 * N;
    for (int q = 0; q < 9 && e == cudaSuccess; ++q)
      e = lbm::launch_transpose<double, double>((const double*)tmp + kSwapXY[q] * N, g + q * N,
                                                P.nx, P.ny, b->stream);
    out = g;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f, out, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(tmp);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "get populations failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Launch the moments/diagnostics kernel over a device list of n items on the batch's
// stream.  The pair kernel has strip and full-width instantiations: both are launched over
// the whole list, and each CTA works only on an item of its own kind.
template <typename S>
cudaError_t launch_moments(const Batch* b, const WorkItem* d_items, int n,
                           const MomArgs<S>& mo) {
  bool kind[2] = {false, false};  // strips, full-width strips present
  for (int i = 0; i < b->n_inst; ++i)
    kind[lbm::full_width(b->inst[i].nx, mom_nt(b), b->vec) ? 1 : 0] = true;
  cudaError_t e = cudaSuccess;
  for (int full = 0; full < 2 && e == cudaSuccess; ++full)
    if (kind[full])
      e = lbm::launch_sweep<S>(mom_nt(b), b->vec, lbm::MODE_MOMENTS, full,
                               (const S*)b->slab[b->cur], nullptr, b->d_inst, d_items, n, mo,
                               b->d_status, b->stream);
  return e;
}

// Moments/diagnostics pass over `items` (device list of n entries).
template <typename S>
int moments_pass(Batch* b, const WorkItem* d_items, int n, MomArgs<S> mo) {
  mo.part_sum = b->d_part_sum;
  mo.part_max = b->d_part_max;
  mo.part_bad = b->d_part_bad;
  cudaError_t e = launch_moments<S>(b, d_items, n, mo);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "moments kernel launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int ensure_fields(Batch* b) {
  for (auto& f : b->fields)
    if (!f) {
      int rc = guarded_alloc(b, &f, std::max<size_t>(b->dense_elems, 1) * b->esz,
                             "moment field");
      if (rc) return rc;
    }
  return LBM_OK;
}

// Fields of instance i into device arrays (storage type) at the instance's dense offset
// (or, with direct pointers, at offset 0 of the caller's arrays).
int moments_device(Batch* b, int i, void* rho, void* ux, void* uy, bool caller_ptrs) {
  const int lo = b->item_begin[i], hi = b->item_begin[i + 1];
  if (b->ev_fields_free && !caller_ptrs)  // an asynchronous read-back may still read them
    CK(b, cudaStreamWaitEvent(b->stream, b->ev_fields_free, 0));
  const long long shift = caller_ptrs ? b->inst[i].dense_off : 0;
  if (b->fp64) {
    MomArgs<double> mo{};
    mo.rho = rho ? (double*)rho - shift : nullptr;
    mo.ux = ux ? (double*)ux - shift : nullptr;
    mo.uy = uy ? (double*)uy - shift : nullptr;
    mo.flags = lbm::MOM_FIELDS;
    return moments_pass<double>(b, b->d_all_items + lo, hi - lo, mo);
  }
  MomArgs<float> mo{};
  mo.rho = rho ? (float*)rho - shift : nullptr;
  mo.ux = ux ? (float*)ux - shift : nullptr;
  mo.uy = uy ? (float*)uy - shift : nullptr;
  mo.flags = lbm::MOM_FIELDS;
  return moments_pass<float>(b, b->d_all_items + lo, hi - lo, mo);
}

// Stored field of each host output (rho, ux, uy) of instance i: a transposed instance's
// x velocity is its stored y velocity.
void stored_fields(const Batch* b, int i, int sk[3]) {
  sk[0] = 0;
  sk[1] = b->tr[i] ? 2 : 1;
  sk[2] = b->tr[i] ? 1 : 2;
}

// moments_device into the batch's own fields for the requested host outputs.
int moments_for_outputs(Batch* b, int i, const void* const outs[3], int sk[3]) {
  stored_fields(b, i, sk);
  void* want[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k)
    if (outs[k]) want[sk[k]] = b->fields[sk[k]];
  return moments_device(b, i, want[0], want[1], want[2], false);
}

int moments_host(Batch* b, int i, double* rho, double* ux, double* uy) {
  int rc = ensure_fields(b);
  if (rc) return rc;
  double* outs[3] = {rho, ux, uy};
  const void* const req[3] = {rho, ux, uy};
  int sk[3];
  rc = moments_for_outputs(b, i, req, sk);
  if (rc) return rc;
  const InstParams& P = b->inst[i];
  const size_t N = (size_t)P.nx * P.ny;
  const bool t = b->tr[i];
  if (!b->fp64 || t) {
    rc = ensure_staging(b);
    if (rc) return rc;
  }
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    const char* src = (const char*)b->fields[sk[k]] + P.dense_off * b->esz;
    if (t) {
      // back to the given orientation (P.ny rows of P.nx values stored), as doubles
      double* w = b->staging + k * b->staging_elems;
      if (b->fp64)
        CK(b, (lbm::launch_transpose<double, double>((const double*)src, w, P.nx, P.ny,
                                                    b->stream)));
      else
        CK(b, (lbm::launch_transpose<float, double>((const float*)src, w, P.nx, P.ny,
                                                   b->stream)));
      CK(b, cudaMemcpyAsync(outs[k], w, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    } else if (b->fp64) {
      CK(b, cudaMemcpyAsync(outs[k], src, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    } else {
      // widen on the device, then one transfer of doubles into the caller's buffer
      double* w = b->staging + k * b->staging_elems;
      CK(b, lbm::launch_widen((const float*)src, w, (long long)N, b->stream));
      CK(b, cudaMemcpyAsync(outs[k], w, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    }
  }
  CK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

// moments_host into host floats: FP32 fields are transferred as stored, FP64 fields are
// rounded to float on the device first.
int moments_host_f32(Batch* b, int i, float* rho, float* ux, float* uy) {
  int rc = ensure_fields(b);
  if (rc) return rc;
  float* outs[3] = {rho, ux, uy};
  const void* const req[3] = {rho, ux, uy};
  int sk[3];
  rc = moments_for_outputs(b, i, req, sk);
  if (rc) return rc;
  const bool t = b->tr[i];
  if (b->fp64 || t) {
    rc = ensure_staging32(b);
    if (rc) return rc;
  }
  const InstParams& P = b->inst[i];
  const size_t N = (size_t)P.nx * P.ny;
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    const char* src = (const char*)b->fields[sk[k]] + P.dense_off * b->esz;
    const float* f = (const float*)src;
    if (t) {
      // back to the given orientation, as floats
      float* w = b->staging32 + k * b->staging_elems;
      if (b->fp64)
        CK(b, (lbm::launch_transpose<double, float>((const double*)src, w, P.nx, P.ny,
                                                   b->stream)));
      else
        CK(b, (lbm::launch_transpose<float, float>(f, w, P.nx, P.ny, b->stream)));
      f = w;
    } else if (b->fp64) {
      float* w = b->staging32 + k * b->staging_elems;
      CK(b, lbm::launch_narrow((const double*)src, w, (long long)N, b->stream));
      f = w;
    }
    CK(b, cudaMemcpyAsync(outs[k], f, N * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
  }
  CK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

// Copy streams and events of the asynchronous host transfers (created on first use).
int ensure_async(Batch* b) {
  for (cudaStream_t* s : {&b->up_stream, &b->down_stream})
    if (!*s) CK(b, cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
  for (cudaEvent_t* ev : {&b->ev_uploaded, &b->ev_staging_free, &b->ev_fields_ready,
                          &b->ev_fields_free})
    if (!*ev) CK(b, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  return LBM_OK;
}

// Instance 0 initialised from host fields of the storage type, uploaded on up_stream; the
// initialisation itself (FP32: widening, then the double path of init_instance) is queued
// on the handle's stream, and its validity check sets STATUS_BADINIT.
int init_async(Batch* b, const void* rho, const void* ux, const void* uy) {
  if (!rho) return set_err(b->err, LBM_EINVAL, "rho must not be NULL");
  int rc = ensure_async(b);
  if (rc == LBM_OK) rc = ensure_flag(b);
  if (rc == LBM_OK) rc = b->fp64 ? ensure_staging(b) : ensure_staging32(b);
  if (rc) return rc;
  const InstParams& P = b->inst[0];
  const size_t N = (size_t)P.nx * P.ny;
  const void* in[3] = {rho, ux, uy};
  const double* dev[3] = {nullptr, nullptr, nullptr};
  CK(b, cudaStreamWaitEvent(b->up_stream, b->ev_staging_free, 0));
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    void* dst = b->fp64 ? (void*)(b->staging + k * b->staging_elems)
                        : (void*)(b->staging32 + k * b->staging_elems);
    CK(b, cudaMemcpyAsync(dst, in[k], N * b->esz, cudaMemcpyHostToDevice, b->up_stream));
  }
  CK(b, cudaEventRecord(b->ev_uploaded, b->up_stream));
  CK(b, cudaStreamWaitEvent(b->stream, b->ev_uploaded, 0));
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    double* d = b->staging + k * b->staging_elems;
    if (!b->fp64)
      CK(b, lbm::launch_widen(b->staging32 + k * b->staging_elems, d, (long long)N, b->stream));
    dev[k] = d;
  }
  CK(b, cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream));
  CK(b, cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  cudaError_t e =
      b->fp64 ? lbm::launch_init_eq<double>(dev[0], dev[1], dev[2], (double*)b->slab[b->cur], P,
                                            b->d_flag, b->stream)
              : lbm::launch_init_eq<float>(dev[0], dev[1], dev[2], (float*)b->slab[b->cur], P,
                                           b->d_flag, b->stream);
  if (e == cudaSuccess)
    e = b->fp64 ? lbm::launch_fill_ghosts<double>((double*)b->slab[b->cur], P, b->stream)
                : lbm::launch_fill_ghosts<float>((float*)b->slab[b->cur], P, b->stream);
  if (e == cudaSuccess)
    e = lbm::launch_flag_status(b->d_flag, b->d_status, lbm::STATUS_BADINIT, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_staging_free, b->stream);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
  b->steps[0] = 0;
  b->dinf_valid[0] = 0;
  return LBM_OK;
}

// Moments of instance 0 into the handle's fields on its stream, copied to host arrays of
// the storage type on down_stream.
int moments_async(Batch* b, void* rho, void* ux, void* uy) {
  if (!rho && !ux && !uy) return LBM_OK;
  int rc = ensure_async(b);
  if (rc == LBM_OK) rc = ensure_fields(b);
  if (rc) return rc;
  void* outs[3] = {rho, ux, uy};
  rc = moments_device(b, 0, rho ? b->fields[0] : nullptr, ux ? b->fields[1] : nullptr,
                      uy ? b->fields[2] : nullptr, false);  // waits for the last read-back
  if (rc) return rc;
  const InstParams& P = b->inst[0];
  const size_t N = (size_t)P.nx * P.ny;
  CK(b, cudaEventRecord(b->ev_fields_ready, b->stream));
  CK(b, cudaStreamWaitEvent(b->down_stream, b->ev_fields_ready, 0));
  for (int k = 0; k < 3; ++k)
    if (outs[k])
      CK(b, cudaMemcpyAsync(outs[k], (const char*)b->fields[k] + P.dense_off * b->esz,
                            N * b->esz, cudaMemcpyDeviceToHost, b->down_stream));
  CK(b, cudaEventRecord(b->ev_fields_free, b->down_stream));
  return LBM_OK;
}

// Diagnostics of every instance (out: n_inst entries).
int diagnostics(Batch* b, lbm_diag* out) {
  int rc;
  if (b->fp64) {
    MomArgs<double> mo{};
    mo.rho_prev = (double*)b->rho_prev;
    mo.flags = lbm::MOM_DIAG | lbm::MOM_UPDATE_PREV;
    rc = moments_pass<double>(b, b->d_all_items, b->n_all, mo);
  } else {
    MomArgs<float> mo{};
    mo.rho_prev = (float*)b->rho_prev;
    mo.flags = lbm::MOM_DIAG | lbm::MOM_UPDATE_PREV;
    rc = moments_pass<float>(b, b->d_all_items, b->n_all, mo);
  }
  if (rc) return rc;
  cudaError_t e = lbm::launch_diag_finalize(b->d_part_sum, b->d_part_max, b->d_part_bad,
                                            b->d_item_begin, b->n_inst, b->d_diag, b->stream);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "diagnostics reduction failed: %s", cudaGetErrorString(e));
  std::vector<double> h(6 * (size_t)b->n_inst);
  CK(b, cudaMemcpyAsync(h.data(), b->d_diag, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                        b->stream));
  CK(b, cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n_inst; ++i) {
    out[i].mass = h[6 * i];
    out[i].mom_x = h[6 * i + (b->tr[i] ? 2 : 1)];  // stored axes of a transposed instance
    out[i].mom_y = h[6 * i + (b->tr[i] ? 1 : 2)];
    out[i].max_u = h[6 * i + 3];
    out[i].dinf = b->dinf_valid[i] ? h[6 * i + 4] : -1.0;
    out[i].nonfinite = (long long)h[6 * i + 5];
    out[i].step = b->steps[i];
    b->dinf_valid[i] = 1;
  }
  return LBM_OK;
}

// Stop stepping instance i; both slabs then hold its state.
int freeze(Batch* b, int i) {
  const InstParams& P = b->inst[i];
  CK(b, cudaMemcpyAsync((char*)b->slab[b->cur ^ 1] + P.off * b->esz,
                        (char*)b->slab[b->cur] + P.off * b->esz, 9 * P.plane * b->esz,
                        cudaMemcpyDeviceToDevice, b->stream));
  b->active[i] = 0;
  return LBM_OK;
}

int eval_psi(Batch* b, const double* rho, double* psi, size_t n) {
  if (!rho || !psi) return set_err(b->err, LBM_EINVAL, "rho and psi must not be NULL");
  if (n == 0) return LBM_OK;
  void* tmp = nullptr;
  int rc = dev_alloc(b, &tmp, 2 * n * sizeof(double));
  if (rc) return rc;
  double* dr = (double*)tmp;
  double* dp = dr + n;
  cudaError_t e = cudaMemcpyAsync(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = b->fp64 ? lbm::launch_psi<double>(dr, dp, (long long)n, b->d_inst, b->stream)
                : lbm::launch_psi<float>(dr, dp, (long long)n, b->d_inst, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(psi, dp, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(tmp);
  if (e != cudaSuccess) return set_err(b->err, LBM_ECUDA, "psi evaluation failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// CRC-32 (IEEE 802.3 polynomial, reflected), bytewise.
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  const unsigned char* p = (const unsigned char*)data;
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

struct FileHeader {
  char magic[8];
  uint32_t version, precision;
  int32_t nx, ny, pitch, walls;
  int64_t step;
  uint64_t payload_bytes;
  InstParams params;
};

// ---------------------------------------------------------------------------------------
// Autotuner

struct TileChoice {
  int nt = 0, vec = 0, rows = 0;
  double ms = -1.0;
  int persist = 1;  // 0: one launch per step measured faster than persistent stepping
};

std::string tune_key(const Batch* b) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  unsigned long long hsh = 1469598103934665603ULL;  // FNV-1a over the instance sizes/walls
  long long nodes = 0;
  for (int i = 0; i < b->n_inst; ++i) {
    if (!b->active[i]) continue;
    const long long v[3] = {b->inst[i].nx, b->inst[i].ny, b->inst[i].walls};
    for (long long x : v)
      for (int k = 0; k < 8; ++k) hsh = (hsh ^ ((x >> (8 * k)) & 0xff)) * 1099511628211ULL;
    nodes += (long long)b->inst[i].nx * b->inst[i].ny;
  }
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%d|%s|%d|%lld|%016llx", b->fp64 ? "fp64" : "fp32", b->n_inst,
           name.c_str(), prop.multiProcessorCount, nodes, hsh);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, TileChoice& c) {
  if (!path) return false;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return false;
  char line[512], k[300];
  bool found = false;
  while (std::fgets(line, sizeof line, fp)) {
    TileChoice t;
    const int got =
        std::sscanf(line, "%299s %d %d %d %lf %d", k, &t.nt, &t.vec, &t.rows, &t.ms, &t.persist);
    if (got >= 5 && key == k) {  // entries without the persistence field allow it
      c = t;  // the last entry for a key wins
      found = true;
    }
  }
  std::fclose(fp);
  return found;
}

void cache_store(const char* path, const std::string& key, const TileChoice& c) {
  if (!path) return;
  FILE* fp = std::fopen(path, "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d %d %d %.6f %d\n", key.c_str(), c.nt, c.vec, c.rows, c.ms, c.persist);
  std::fclose(fp);
}

int apply_tiling(Batch* b, int nt, int vec, int rows, bool persist = true) {
  if (!tiling_ok(b->fp64, nt, vec))
    return set_err(b->err, LBM_EINVAL, "tiling %d threads x %d columns not available", nt, vec);
  b->nt = nt;
  b->vec = vec;
  b->rows_req = rows;
  b->persist_off = !persist;
  return rebuild_items(b);
}

int autotune(Batch* b, int steps, const char* cache_path, TileChoice& best) {
  if (steps < 2) return set_err(b->err, LBM_EINVAL, "autotune needs steps >= 2");
  if (const char* env = std::getenv("LBM_TILE")) {
    TileChoice t;
    if (std::sscanf(env, "%d,%d,%d", &t.nt, &t.vec, &t.rows) != 3)
      return set_err(b->err, LBM_EINVAL, "LBM_TILE must be threads,vec,rows");
    int rc = apply_tiling(b, t.nt, t.vec, t.rows);
    if (rc) return rc;
    best = t;
    return LBM_OK;
  }
  const std::string key = tune_key(b);
  TileChoice hit;
  if (cache_lookup(cache_path, key, hit) && tiling_ok(b->fp64, hit.nt, hit.vec)) {
    best = hit;
    return apply_tiling(b, hit.nt, hit.vec, hit.rows, hit.persist != 0);
  }
  if (b->n_items == 0) return set_err(b->err, LBM_ESTATE, "no active instance to tune on");
  // Save the state (both slabs agree for frozen instances; the current one for the rest).
  // Errors below are recorded in rc and the loop left, so the copy and the events are
  // always released and the state always restored.
  void* backup = nullptr;
  const size_t bytes = b->slab_elems * b->esz;
  CK(b, dev_malloc(&backup, bytes));
  int rc = LBM_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == LBM_OK)
      rc = set_err(b->err, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                   "%s failed: %s", what, cudaGetErrorString(e));
    return rc == LBM_OK;
  };
  const int saved_cur = b->cur;
  const std::vector<long long> saved_steps = b->steps;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool saved =
      cu(cudaMemcpyAsync(backup, b->slab[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream),
         "state backup");  // nothing is stepped unless the copy was queued
  cu(cudaEventCreate(&e0), "cudaEventCreate");
  cu(cudaEventCreate(&e1), "cudaEventCreate");
  const int nts[] = {32, 64, 96, 128, 256, LBM_TILE_PER_INSTANCE};
  const int vecs[] = {1, 2};
  // Chunk heights: the best one depends on how the CTA count falls into waves of resident
  // CTAs, which moves the step time by several per cent between neighbouring heights.
  // Heights below 8 are for small grids, where more (shorter) chunks fill more SMs.
  const int rows_c[] = {1, 2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64};
  best = TileChoice();
  for (int vec : vecs) {
    for (int nt : nts) {
      if (!tiling_ok(b->fp64, nt, vec)) continue;
      for (int rows : rows_c) {
        // A tiling that steps persistently is timed that way and with one launch per step.
        for (int persist = 1; persist >= 0 && rc == LBM_OK; --persist) {
          rc = apply_tiling(b, nt, vec, rows, persist != 0);
          if (rc) break;
          const bool persistent = b->persist;
          // Timed as stepping runs (graph replays for each kGraphSteps); an even count
          // returns to the same slab, so the warm-up run captures the graph the timed run
          // replays.
          const int n_t = steps + (steps & 1);
          rc = do_steps(b, n_t);  // warm-up
          if (rc) break;
          double per = -1.0;  // the better of two timed runs
          for (int rep = 0; rep < 2; ++rep) {
            if (!cu(cudaEventRecord(e0, b->stream), "cudaEventRecord")) break;
            rc = do_steps(b, n_t);
            if (rc) break;
            if (!cu(cudaEventRecord(e1, b->stream), "cudaEventRecord")) break;
            if (!cu(cudaEventSynchronize(e1), "cudaEventSynchronize")) break;
            float ms = 0.f;
            if (!cu(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime")) break;
            if (per < 0 || ms / n_t < per) per = ms / n_t;
          }
          if (rc) break;
          if (best.ms < 0 || per < best.ms) {
            best.nt = nt;
            best.vec = vec;
            best.rows = rows;
            best.ms = per;
            best.persist = persist;
          }
          if (!persistent) break;  // the tiling does not step persistently: timed once
        }
        if (rc) break;
      }
      if (rc) break;
    }
    if (rc) break;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // Restore the state into both slabs and the bookkeeping.
  if (saved) {
    cudaMemcpyAsync(b->slab[0], backup, bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->slab[1], backup, bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  }
  cudaStreamSynchronize(b->stream);
  dev_free(backup);
  b->cur = saved_cur;
  b->steps = saved_steps;
  if (rc) return rc;
  rc = apply_tiling(b, best.nt, best.vec, best.rows, best.persist != 0);
  if (rc) return rc;
  cache_store(cache_path, key, best);
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Allocation-free diagnostics: the per-work-item partials live in this fixed device array
// instead of handle-owned buffers.  Layout: 3 doubles (sums) per item, then 2 floats
// (maxima) per item, then 1 int (non-finite count) per item.
namespace {

constexpr size_t kNoAllocItemBytes = 3 * sizeof(double) + 2 * sizeof(float) + sizeof(int);
static __device__ __align__(256) unsigned char
    g_noalloc_partials[(size_t)LBM_NOALLOC_MAX_ITEMS * kNoAllocItemBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
// Per device ordinal: the context that was current when the address was looked up, and
// the address.  A device reset (cudaDeviceReset) destroys the primary context and a later
// call runs in a new one, where the module is loaded again and the array may sit
// elsewhere: a different current context triggers a fresh lookup.
struct NoAllocSlot {
  CUcontext ctx;
  void* addr;
};
NoAllocSlot g_noalloc_slot[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (no link against libcuda);
// it only reads the calling thread's current context and enqueues no work.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

int current_context(Batch* b, CUcontext* ctx) {
  static std::once_flag once;
  static CtxGetCurrentFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  if (!fn) return set_err(b->err, LBM_ECUDA, "cuCtxGetCurrent is not available");
  if (fn(ctx) != CUDA_SUCCESS) return set_err(b->err, LBM_ECUDA, "cuCtxGetCurrent failed");
  return LBM_OK;
}

// Device address of the array on the current device, looked up once per device (and
// again in a new context after a device reset).  Host code must never use the symbol's
// name as a device pointer: it is a host-side stand-in.
int noalloc_partials(Batch* b, unsigned char** out) {
  int dev = 0;
  CK(b, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_err(b->err, LBM_EINVAL, "device %d beyond the %d supported", dev, kMaxDevices);
  CUcontext ctx = nullptr;
  int rc = current_context(b, &ctx);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocSlot& slot = g_noalloc_slot[dev];
  if (!slot.addr || slot.ctx != ctx) {
    void* p = nullptr;
    CK(b, cudaGetSymbolAddress(&p, g_noalloc_partials));
    slot.addr = p;
    slot.ctx = ctx;
  }
  *out = (unsigned char*)slot.addr;
  return LBM_OK;
}

template <typename S>
int noalloc_diag_pass(Batch* b, double* part_sum, float* part_max, int* part_bad) {
  MomArgs<S> mo{};
  mo.part_sum = part_sum;
  mo.part_max = part_max;
  mo.part_bad = part_bad;
  mo.flags = lbm::MOM_DIAG;  // no fields, no reference density
  cudaError_t e = launch_moments<S>(b, b->d_all_items, b->n_all, mo);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "diagnostics pass launch failed: %s",
                   cudaGetErrorString(e));
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Single-lattice handle

struct lbm_handle {
  Batch b;
};
struct lbm_batch {
  Batch b;
};

extern "C" {

void lbm_options_default(lbm_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = LBM_FP32_DEV;
  o->visc_mode = -1;
  o->bc = LBM_BC_PERIODIC;
  o->psi_fp64 = 0;
  o->rho_ref = -1.0;
  o->rho_c = 0.0;
  o->rho_l = 0.0;
  o->rho_v = 0.0;
  o->stream = nullptr;
  o->device = -1;
  o->tile_threads = 0;
  o->tile_vec = 0;
  o->tile_rows = 0;
}

int lbm_create(lbm_handle** out, int nx, int ny, lbm_eos eos, double G, double sigma,
               const double s[9], double nu_l, double nu_v, const lbm_options* opt) {
  Range r_("lbm_create");
  if (!out || !s) return set_err(g_thread_err, LBM_EINVAL, "out and s must not be NULL");
  *out = nullptr;
  lbm_options o;
  lbm_options_default(&o);
  if (opt) o = *opt;
  if (o.precision != LBM_FP64 && o.precision != LBM_FP32_DEV)
    return set_err(g_thread_err, LBM_EINVAL, "unknown precision %d", o.precision);
  lbm_instance in{};
  in.nx = nx;
  in.ny = ny;
  in.eos = eos;
  in.G = G;
  in.sigma = sigma;
  for (int i = 0; i < 9; ++i) in.s[i] = s[i];
  in.nu_l = nu_l;
  in.nu_v = nu_v;
  in.visc_mode = o.visc_mode >= 0 ? o.visc_mode
                                  : ((nu_l > 0 && nu_v > 0) ? LBM_VISC_STEP : LBM_VISC_CONST);
  in.bc = o.bc;
  in.rho_c = o.rho_c;
  in.rho_l = o.rho_l;
  in.rho_v = o.rho_v;
  in.rho_ref = o.rho_ref;
  in.layout = LBM_LAYOUT_ROWS;  // a lattice handle is never transposed
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return set_err(g_thread_err, LBM_ENOMEM, "out of host memory");
  int rc = create_batch(&h->b, 1, &in, o.precision == LBM_FP64, o.psi_fp64, o.stream,
                        o.device, o.tile_threads, o.tile_vec, o.tile_rows);
  if (rc) {
    g_thread_err = h->b.err;
    destroy_batch(&h->b);
    delete h;
    return rc;
  }
  g_thread_err.clear();
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  destroy_batch(&h->b);
  delete h;
}

const char* lbm_last_error(const lbm_handle* h) {
  DeviceGuard g_(h ? &h->b : nullptr);
  return h ? h->b.err.c_str() : g_thread_err.c_str();
}

int lbm_init_fields(lbm_handle* h, const double* rho, const double* ux, const double* uy) {
  Range r_("lbm_init_fields");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return init_instance(&h->b, 0, rho, ux, uy, false);
}

int lbm_init_fields_device(lbm_handle* h, const double* rho, const double* ux,
                           const double* uy) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return init_instance(&h->b, 0, rho, ux, uy, true);
}

int lbm_set_populations(lbm_handle* h, const double* f) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return set_pops(&h->b, 0, f);
}

int lbm_get_populations(lbm_handle* h, double* f) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  int rc = get_pops(&h->b, 0, f);
  if (rc) return rc;
  return sync_status(&h->b);
}

int lbm_step(lbm_handle* h, int n) {
  Range r_("lbm_step");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return do_steps(&h->b, n);
}

int lbm_sync(lbm_handle* h) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return sync_status(&h->b);
}

int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy) {
  Range r_("lbm_moments");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  int rc = moments_host(&h->b, 0, rho, ux, uy);
  if (rc) return rc;
  return sync_status(&h->b);
}

int lbm_init_fields_async(lbm_handle* h, const void* rho, const void* ux, const void* uy) {
  Range r_("lbm_init_fields_async");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return init_async(&h->b, rho, ux, uy);
}

int lbm_moments_async(lbm_handle* h, void* rho, void* ux, void* uy) {
  Range r_("lbm_moments_async");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  if (!rho) return set_err(h->b.err, LBM_EINVAL, "rho must not be NULL");
  return moments_async(&h->b, rho, ux, uy);
}

int lbm_moments_device(lbm_handle* h, void* rho, void* ux, void* uy) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return moments_device(&h->b, 0, rho, ux, uy, true);
}

int lbm_init_fields_f32(lbm_handle* h, const float* rho, const float* ux, const float* uy) {
  Range r_("lbm_init_fields_f32");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return init_instance_f32(&h->b, 0, rho, ux, uy);
}

int lbm_moments_f32(lbm_handle* h, float* rho, float* ux, float* uy) {
  Range r_("lbm_moments_f32");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return moments_host_f32(&h->b, 0, rho, ux, uy);
}

int lbm_diagnostics(lbm_handle* h, lbm_diag* out) {
  Range r_("lbm_diagnostics");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h || !out) return h ? set_err(h->b.err, LBM_EINVAL, "out must not be NULL") : LBM_EINVAL;
  return diagnostics(&h->b, out);
}

int lbm_pressure_tensor(lbm_handle* h, double* pxx, double* pyy, double* pxy,
                        int include_sigma) {
  Range r_("lbm_pressure_tensor");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  if (!pxx || !pyy || !pxy) return set_err(b->err, LBM_EINVAL, "outputs must not be NULL");
  int rc = ensure_fields(b);
  if (!rc) rc = moments_device(b, 0, b->fields[0], nullptr, nullptr, false);
  if (rc) return rc;
  const InstParams& P = b->inst[0];
  const size_t N = (size_t)P.nx * P.ny;
  // sigma back from the per-instance constant 12 sigma s_e (s_e > 0 is checked at create)
  const double sigma = include_sigma ? P.sig12_e / (12.0 * P.s[1]) : 0.0;
  double* d = nullptr;
  rc = dev_alloc(b, (void**)&d, 3 * N * sizeof(double));
  if (rc) return rc;
  cudaError_t e =
      b->fp64 ? lbm::launch_pressure<double>((const double*)b->fields[0] + P.dense_off, P, sigma,
                                             d, d + N, d + 2 * N, b->stream)
              : lbm::launch_pressure<float>((const float*)b->fields[0] + P.dense_off, P, sigma, d,
                                            d + N, d + 2 * N, b->stream);
  double* outs[3] = {pxx, pyy, pxy};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(outs[k], d + k * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(d);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "pressure tensor failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_selftest_timeout(lbm_handle* h, long long polls) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  if (polls < 1 || polls > (1LL << 20))
    return set_err(h->b.err, LBM_EINVAL, "polls must be in [1, 2^20]");
  cudaError_t e = lbm::launch_wait_selftest(h->b.d_status, polls, h->b.stream);
  if (e != cudaSuccess)
    return set_err(h->b.err, LBM_ECUDA, "self-test launch failed: %s", cudaGetErrorString(e));
  return sync_status(&h->b);
}

int lbm_selftest_dep_timeout(lbm_handle* h, int polls) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  if (polls < 1 || polls > (1 << 20))
    return set_err(b->err, LBM_EINVAL, "polls must be in [1, 2^20]");
  if (b->fp64 || b->vec != 2 || b->n_items < 1 || b->n_groups < 1)
    return set_err(b->err, LBM_EINVAL, "the self-test needs an FP32 lattice with tile_vec 2");
  // One item, two steps: step 0 runs and releases chunk 0; step 1 waits for chunk 1, which
  // no item has, so its wait runs out.
  WorkItem items2[2] = {b->items[0], b->items[0]};
  ItemLink links2[2];
  for (ItemLink& l : links2) {
    l = ItemLink{};
    l.chunk = 0;
    l.strips = 1;
    for (int& d : l.dep) d = 1;
  }
  void* buf = nullptr;
  int rc = dev_alloc(b, &buf, sizeof(items2) + sizeof(links2) + 4 * sizeof(int));
  if (rc) return rc;
  char* p = (char*)buf;
  WorkItem* d_items2 = (WorkItem*)p;
  ItemLink* d_links2 = (ItemLink*)(p + sizeof(items2));
  int* sync = (int*)(p + sizeof(items2) + sizeof(links2));
  cudaError_t e = cudaMemcpyAsync(d_items2, items2, sizeof(items2), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_links2, links2, sizeof(links2), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sync, 0, 4 * sizeof(int), b->stream);
  if (e == cudaSuccess)
    e = lbm::launch_persist(b->grp_nt[0],
                            b->grp_full[0] ? lbm::PERSIST_FULL : lbm::PERSIST_STRIP,
                            (float*)b->slab[b->cur], (float*)b->slab[b->cur ^ 1], b->d_inst,
                            d_items2, d_links2, 1, 2,
                            sync, sync + 1, b->d_status, 1, polls, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(buf);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "self-test launch failed: %s", cudaGetErrorString(e));
  return sync_status(b);
}

int lbm_init_droplets(lbm_handle* h, const lbm_droplet* drops, int n, const lbm_warm_params* p,
                      int flags) {
  Range r_("lbm_init_droplets");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  if (!drops || !p) return set_err(b->err, LBM_EINVAL, "drops and params must not be NULL");
  if (n < 1 || n > 65536) return set_err(b->err, LBM_EINVAL, "droplet count %d not in [1, 65536]", n);
  if (flags & ~(LBM_WARM_CURVATURE | LBM_WARM_BALANCED))
    return set_err(b->err, LBM_EINVAL, "unknown flags %d", flags);
  if (!(p->width > 0.0) || !std::isfinite(p->width) || !(p->rho_v > 0.0) ||
      !(p->rho_l > p->rho_v) || !std::isfinite(p->rho_l) || !std::isfinite(p->shift))
    return set_err(b->err, LBM_EINVAL, "warm-start parameters out of range");
  const InstParams& P = b->inst[0];
  const lbm_eos eos{P.a, 4.0 * P.b4, 1.0, P.RT};  // p depends on R and T through R T only
  double kappa = 0.0;
  for (int k = 0; k < n; ++k) {
    const lbm_droplet& d = drops[k];
    if (!std::isfinite(d.cx) || !std::isfinite(d.cy) || !(d.radius > 0.0))
      return set_err(b->err, LBM_EINVAL, "droplet %d: bad centre or radius", k);
    kappa += 1.0 / d.radius;
  }
  kappa /= n;
  double rin = p->rho_l, rout = p->rho_v;
  if ((flags & LBM_WARM_CURVATURE) && lbm_curved_densities(eos, p, kappa, &rin, &rout) != LBM_OK)
    return set_err(b->err, LBM_EINVAL, "no curved-interface densities for these parameters");
  if (!(rin > rout)) return set_err(b->err, LBM_EINVAL, "liquid density not above the vapour's");
  std::vector<lbm::DropRec> recs(n);
  for (int k = 0; k < n; ++k)
    recs[k] = lbm::DropRec{drops[k].cx, drops[k].cy, drops[k].radius + p->shift, rin};
  const size_t N = (size_t)P.nx * P.ny;
  const bool balanced = (flags & LBM_WARM_BALANCED) != 0;
  double* d_rho = nullptr;
  lbm::DropRec* d_drops = nullptr;
  int rc = dev_alloc(b, (void**)&d_rho, (balanced ? 3 : 1) * N * sizeof(double));
  if (!rc) rc = dev_alloc(b, (void**)&d_drops, n * sizeof(lbm::DropRec));
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(d_drops, recs.data(), n * sizeof(lbm::DropRec),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = lbm::launch_fill_droplets(d_rho, P.nx, P.ny, d_drops, n, rout, p->width, b->stream);
    if (e == cudaSuccess && balanced)
      e = lbm::launch_balanced_velocity(d_rho, P, d_rho + N, d_rho + 2 * N, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
      rc = set_err(b->err, LBM_ECUDA, "droplet fill failed: %s", cudaGetErrorString(e));
  }
  if (!rc)
    rc = init_instance(b, 0, d_rho, balanced ? d_rho + N : nullptr,
                       balanced ? d_rho + 2 * N : nullptr, true);
  dev_free(d_rho);
  dev_free(d_drops);
  return rc;
}

int lbm_phase_stats(lbm_handle* h, double rho_vap_max, double rho_liq_min, double out[4]) {
  Range r_("lbm_phase_stats");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  if (!out) return set_err(b->err, LBM_EINVAL, "out must not be NULL");
  int rc = ensure_fields(b);
  if (!rc) rc = moments_device(b, 0, b->fields[0], nullptr, nullptr, false);
  if (rc) return rc;
  const InstParams& P = b->inst[0];
  const long long N = (long long)P.nx * P.ny;
  double* d_part = nullptr;
  rc = dev_alloc(b, (void**)&d_part, lbm::kPhaseBlocks * 4 * sizeof(double));
  if (rc) return rc;
  std::vector<double> part(lbm::kPhaseBlocks * 4);
  cudaError_t e =
      b->fp64 ? lbm::launch_phase_sums<double>((const double*)b->fields[0] + P.dense_off, N,
                                               rho_vap_max, rho_liq_min, d_part, b->stream)
              : lbm::launch_phase_sums<float>((const float*)b->fields[0] + P.dense_off, N,
                                              rho_vap_max, rho_liq_min, d_part, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), d_part, part.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(d_part);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "phase sums failed: %s", cudaGetErrorString(e));
  double sv = 0.0, cv = 0.0, sl = 0.0, cl = 0.0;
  for (int k = 0; k < lbm::kPhaseBlocks; ++k) {
    sv += part[4 * k];
    cv += part[4 * k + 1];
    sl += part[4 * k + 2];
    cl += part[4 * k + 3];
  }
  out[0] = cv > 0 ? sv / cv : 0.0;
  out[1] = cv;
  out[2] = cl > 0 ? sl / cl : 0.0;
  out[3] = cl;
  return LBM_OK;
}

int lbm_diagnostics_noalloc(lbm_handle* h, double* out_dev) {
  Range r_("lbm_diagnostics_noalloc");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  if (!out_dev) return set_err(b->err, LBM_EINVAL, "out_dev must not be NULL");
  if (b->n_all > LBM_NOALLOC_MAX_ITEMS)
    return set_err(b->err, LBM_EINVAL,
                   "lbm_diagnostics_noalloc: this lattice needs %d work items, the fixed "
                   "array holds %d; use lbm_diagnostics or larger tiles",
                   b->n_all, LBM_NOALLOC_MAX_ITEMS);
  unsigned char* base = nullptr;
  int rc = noalloc_partials(b, &base);
  if (rc) return rc;
  const size_t cap = LBM_NOALLOC_MAX_ITEMS;
  double* part_sum = (double*)base;
  float* part_max = (float*)(base + 3 * sizeof(double) * cap);
  int* part_bad = (int*)(base + (3 * sizeof(double) + 2 * sizeof(float)) * cap);
  const size_t n = (size_t)b->n_all;
  // Clear the part this call uses: an item that returned early must not leave an earlier
  // call's partials behind.
  CK(b, cudaMemsetAsync(part_sum, 0, 3 * sizeof(double) * n, b->stream));
  CK(b, cudaMemsetAsync(part_max, 0, 2 * sizeof(float) * n, b->stream));
  CK(b, cudaMemsetAsync(part_bad, 0, sizeof(int) * n, b->stream));
  rc = b->fp64 ? noalloc_diag_pass<double>(b, part_sum, part_max, part_bad)
               : noalloc_diag_pass<float>(b, part_sum, part_max, part_bad);
  if (rc) return rc;
  cudaError_t e = lbm::launch_diag_finalize(part_sum, part_max, part_bad, b->d_item_begin,
                                            b->n_inst, out_dev, b->stream);
  if (e != cudaSuccess)
    return set_err(b->err, LBM_ECUDA, "diagnostics reduction failed: %s",
                   cudaGetErrorString(e));
  return LBM_OK;
}

long long lbm_step_count(const lbm_handle* h) { return h ? h->b.steps[0] : -1; }

int lbm_eval_psi(lbm_handle* h, const double* rho, double* psi, size_t n) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return eval_psi(&h->b, rho, psi, n);
}

int lbm_get_tiling(const lbm_handle* h, int* threads, int* vec, int* rows) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  if (threads) *threads = h->b.nt;
  if (vec) *vec = h->b.vec;
  if (rows) *rows = h->b.rows;
  return LBM_OK;
}

int lbm_set_tiling(lbm_handle* h, int threads, int vec, int rows) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  const int nt_ = threads ? threads : default_threads(b->fp64);
  const int vec_ = vec ? vec : default_vec(b->fp64);
  if (!tiling_ok(b->fp64, nt_, vec_))
    return set_err(b->err, LBM_EINVAL,
                   "tile_threads %d with tile_vec %d is not available for this precision", nt_,
                   vec_);
  if (rows < 0) return set_err(b->err, LBM_EINVAL, "tile_rows must be >= 0");
  b->nt = nt_;
  b->vec = vec_;
  b->rows_req = rows;
  b->persist_off = false;
  return rebuild_items(b);
}

void* lbm_stream(const lbm_handle* h) { return h ? (void*)h->b.stream : nullptr; }

int lbm_autotune(lbm_handle* h, int steps, const char* cache_path, int* threads, int* vec,
                 int* rows, double* ms_per_step) {
  Range r_("lbm_autotune");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  TileChoice c;
  int rc = autotune(&h->b, steps, cache_path, c);
  if (rc) return rc;
  if (threads) *threads = h->b.nt;
  if (vec) *vec = h->b.vec;
  if (rows) *rows = h->b.rows;
  if (ms_per_step) *ms_per_step = c.ms;
  return LBM_OK;
}

int lbm_save(lbm_handle* h, const char* path) {
  Range r_("lbm_save");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h || !path) return LBM_EINVAL;
  Batch* b = &h->b;
  const InstParams& P = b->inst[0];
  const size_t bytes = 9 * (size_t)P.plane * b->esz;
  std::vector<char> buf(bytes);
  CK(b, cudaMemcpyAsync(buf.data(), (char*)b->slab[b->cur] + P.off * b->esz, bytes,
                        cudaMemcpyDeviceToHost, b->stream));
  CK(b, cudaStreamSynchronize(b->stream));
  FileHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "LBMSTATE", 8);
  hd.version = 1;
  hd.precision = b->fp64 ? LBM_FP64 : LBM_FP32_DEV;
  hd.nx = P.nx;
  hd.ny = P.ny;
  hd.pitch = P.pitch;
  hd.walls = P.walls;
  hd.step = b->steps[0];
  hd.payload_bytes = bytes;
  hd.params = P;
  uint32_t crc = crc32_update(0, &hd, sizeof hd);
  crc = crc32_update(crc, buf.data(), bytes);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return set_err(b->err, LBM_EIO, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 &&
            std::fwrite(buf.data(), 1, bytes, fp) == bytes &&
            std::fwrite(&crc, sizeof crc, 1, fp) == 1;
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? LBM_OK : set_err(b->err, LBM_EIO, "short write to %s", path);
}

int lbm_load(lbm_handle* h, const char* path) {
  Range r_("lbm_load");
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h || !path) return LBM_EINVAL;
  Batch* b = &h->b;
  const InstParams& P = b->inst[0];
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return set_err(b->err, LBM_EIO, "cannot open %s", path);
  FileHeader hd;
  if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, "LBMSTATE", 8) != 0) {
    std::fclose(fp);
    return set_err(b->err, LBM_EIO, "%s is not a state file", path);
  }
  if (hd.nx != P.nx || hd.ny != P.ny || hd.pitch != P.pitch ||
      (int)hd.precision != (b->fp64 ? LBM_FP64 : LBM_FP32_DEV) ||
      hd.payload_bytes != 9 * (uint64_t)P.plane * b->esz) {
    std::fclose(fp);
    return set_err(b->err, LBM_EINVAL, "state file does not match this handle's size/precision");
  }
  std::vector<char> buf(hd.payload_bytes);
  uint32_t crc_file = 0;
  const bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size() &&
                  std::fread(&crc_file, sizeof crc_file, 1, fp) == 1;
  std::fclose(fp);
  if (!ok) return set_err(b->err, LBM_EIO, "short read from %s", path);
  uint32_t crc = crc32_update(0, &hd, sizeof hd);
  crc = crc32_update(crc, buf.data(), buf.size());
  if (crc != crc_file) return set_err(b->err, LBM_EIO, "checksum mismatch in %s", path);
  for (int k = 0; k < 2; ++k)
    CK(b, cudaMemcpyAsync((char*)b->slab[k] + P.off * b->esz, buf.data(), buf.size(),
                          cudaMemcpyHostToDevice, b->stream));
  // A state saved after full-width sweeps carries stale ghost columns; this handle's
  // tiling may sweep the lattice in strips, which read them.
  CK(b, b->fp64 ? lbm::launch_fill_ghosts<double>((double*)b->slab[b->cur], P, b->stream)
                : lbm::launch_fill_ghosts<float>((float*)b->slab[b->cur], P, b->stream));
  CK(b, cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  CK(b, cudaStreamSynchronize(b->stream));
  b->steps[0] = hd.step;
  b->dinf_valid[0] = 0;
  return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Batches

int lbm_batch_create(lbm_batch** out, int n, const lbm_instance* inst, int precision,
                     void* stream, int device, int tile_threads, int tile_vec,
                     int tile_rows) {
  Range r_("lbm_batch_create");
  if (!out) return set_err(g_thread_err, LBM_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (precision != LBM_FP64 && precision != LBM_FP32_DEV)
    return set_err(g_thread_err, LBM_EINVAL, "unknown precision %d", precision);
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return set_err(g_thread_err, LBM_ENOMEM, "out of host memory");
  int rc = create_batch(&b->b, n, inst, precision == LBM_FP64, 0, stream, device,
                        tile_threads, tile_vec, tile_rows);
  if (rc) {
    g_thread_err = b->b.err;
    destroy_batch(&b->b);
    delete b;
    return rc;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  destroy_batch(&b->b);
  delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
  DeviceGuard g_(b ? &b->b : nullptr);
  return b ? b->b.err.c_str() : g_thread_err.c_str();
}

int lbm_batch_init_fields(lbm_batch* b, int i, const double* rho, const double* ux,
                          const double* uy) {
  Range r_("lbm_batch_init_fields");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  return init_instance(&b->b, i, rho, ux, uy, false);
}

int lbm_batch_step(lbm_batch* b, int n) {
  Range r_("lbm_batch_step");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  return do_steps(&b->b, n);
}

int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy) {
  Range r_("lbm_batch_moments");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  if (i < 0 || i >= b->b.n_inst) return set_err(b->b.err, LBM_EINVAL, "instance out of range");
  return moments_host(&b->b, i, rho, ux, uy);
}

int lbm_batch_init_fields_f32(lbm_batch* b, int i, const float* rho, const float* ux,
                              const float* uy) {
  Range r_("lbm_batch_init_fields_f32");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  return init_instance_f32(&b->b, i, rho, ux, uy);
}

int lbm_batch_moments_f32(lbm_batch* b, int i, float* rho, float* ux, float* uy) {
  Range r_("lbm_batch_moments_f32");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  if (i < 0 || i >= b->b.n_inst) return set_err(b->b.err, LBM_EINVAL, "instance out of range");
  return moments_host_f32(&b->b, i, rho, ux, uy);
}

int lbm_batch_get_populations(lbm_batch* b, int i, double* f) {
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  if (i < 0 || i >= b->b.n_inst) return set_err(b->b.err, LBM_EINVAL, "instance out of range");
  return get_pops(&b->b, i, f);
}

int lbm_batch_diagnostics(lbm_batch* b, lbm_diag* out) {
  Range r_("lbm_batch_diagnostics");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b || !out) return LBM_EINVAL;
  return diagnostics(&b->b, out);
}

int lbm_batch_active(const lbm_batch* b) {
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  int n = 0;
  for (int a : b->b.active) n += a;
  return n;
}

int lbm_debug_persist_plan(int n_inst, const int* nx, const int* ny, const int* walls,
                           int threads, int rows, int* n_items, int* items_out,
                           int* links_out) {
  if (n_inst < 1 || !nx || !ny || !n_items || rows < 1) return LBM_EINVAL;
  if (threads != 32 && threads != 64 && threads != 96 && threads != 128) return LBM_EINVAL;
  std::vector<InstParams> inst(n_inst);
  std::vector<WorkItem> items;
  for (int i = 0; i < n_inst; ++i) {
    if (nx[i] < 1 || ny[i] < 1) return LBM_EINVAL;
    std::memset(&inst[i], 0, sizeof(InstParams));
    inst[i].nx = nx[i];
    inst[i].ny = ny[i];
    inst[i].walls = walls && walls[i] ? 1 : 0;
    append_items(inst[i], i, threads, 2, rows, items);
  }
  const int n = (int)items.size();
  *n_items = n;
  std::vector<WorkItem> items2(2 * (size_t)n);
  std::vector<ItemLink> links2(2 * (size_t)n);
  int nch = 0;
  if (!plan_persist_list(items, 0, n, inst, rows, items2.data(), links2.data(), &nch,
                         nullptr))
    return 1;
  for (int k = 0; k < 2 * n; ++k) {
    if (items_out) {
      const WorkItem& w = items2[k];
      const int v[5] = {w.inst, w.x0, w.y0, w.y1, w.dir};
      std::memcpy(items_out + 5 * (size_t)k, v, sizeof v);
    }
    if (links_out) {
      const ItemLink& l = links2[k];
      const int v[6] = {l.chunk, l.strips, l.dep[0], l.dep[1], l.dep[2], l.dep[3]};
      std::memcpy(links_out + 6 * (size_t)k, v, sizeof v);
    }
  }
  return LBM_OK;
}

int lbm_persistent(const lbm_handle* h) { return h ? (h->b.persist ? 1 : 0) : LBM_EINVAL; }

int lbm_batch_persistent(const lbm_batch* b) { return b ? (b->b.persist ? 1 : 0) : LBM_EINVAL; }

int lbm_batch_instance_transposed(const lbm_batch* b, int i) {
  if (!b || i < 0 || i >= b->b.n_inst) return LBM_EINVAL;
  return b->b.tr[i] ? 1 : 0;
}

int lbm_batch_instance_active(const lbm_batch* b, int i) {
  if (!b || i < 0 || i >= b->b.n_inst) return LBM_EINVAL;
  return b->b.active[i] ? 1 : 0;
}

int lbm_batch_retire(lbm_batch* bb, int i) {
  Range r_("lbm_batch_retire");
  DeviceGuard g_(bb ? &bb->b : nullptr);
  if (!bb) return LBM_EINVAL;
  Batch* b = &bb->b;
  if (i < 0 || i >= b->n_inst) return set_err(b->err, LBM_EINVAL, "instance %d out of range", i);
  if (!b->active[i]) return LBM_OK;
  int rc = freeze(b, i);
  if (rc) return rc;
  return rebuild_items(b);
}

int lbm_batch_retire_nonfinite(lbm_batch* bb, int* retired) {
  Range r_("lbm_batch_retire_nonfinite");
  DeviceGuard g_(bb ? &bb->b : nullptr);
  if (!bb) return LBM_EINVAL;
  Batch* b = &bb->b;
  if (retired)
    for (int i = 0; i < b->n_inst; ++i) retired[i] = 0;
  std::vector<lbm_diag> d(b->n_inst);
  int rc = diagnostics(b, d.data());
  if (rc) return rc;
  int n = 0;
  for (int i = 0; i < b->n_inst; ++i) {
    if (!b->active[i] || d[i].nonfinite == 0) continue;
    rc = freeze(b, i);
    if (rc) return rc;
    if (retired) retired[i] = 1;
    ++n;
  }
  if (n) {
    rc = rebuild_items(b);
    if (rc) return rc;
  }
  return n;
}

int lbm_batch_autotune(lbm_batch* b, int steps, const char* cache_path, int* threads,
                       int* vec, int* rows, double* ms_per_step) {
  Range r_("lbm_batch_autotune");
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  TileChoice c;
  int rc = autotune(&b->b, steps, cache_path, c);
  if (rc) return rc;
  if (threads) *threads = b->b.nt;
  if (vec) *vec = b->b.vec;
  if (rows) *rows = b->b.rows;
  if (ms_per_step) *ms_per_step = c.ms;
  return LBM_OK;
}

int lbm_batch_get_tiling(const lbm_batch* b, int* threads, int* vec, int* rows) {
  if (!b) return LBM_EINVAL;
  if (threads) *threads = b->b.nt;
  if (vec) *vec = b->b.vec;
  if (rows) *rows = b->b.rows;
  return LBM_OK;
}

int lbm_check_guards(lbm_handle* h) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  return check_guards(&h->b);
}

int lbm_batch_check_guards(lbm_batch* b) {
  DeviceGuard g_(b ? &b->b : nullptr);
  if (!b) return LBM_EINVAL;
  return check_guards(&b->b);
}

int lbm_debug_fail_alloc(int n) { return g_fail_after.exchange(n < 0 ? -1 : n); }

long long lbm_debug_live_allocs(void) { return g_live_allocs.load(); }

int lbm_bounds_checked(void) {
#ifdef LBM_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

int lbm_debug_corrupt_guard(lbm_handle* h, int which) {
  DeviceGuard g_(h ? &h->b : nullptr);
  if (!h) return LBM_EINVAL;
  Batch* b = &h->b;
  const void* user = which == 0 ? b->slab[0] : which == 1 ? b->slab[1]
                   : which == 2 ? b->rho_prev : nullptr;
  for (const auto& g : b->guarded)
    if (user && g.base + kGuard == user) {
      const unsigned char bad = (unsigned char)~kCanary;
      CK(b, cudaMemcpyAsync(g.base + kGuard + g.bytes, &bad, 1, cudaMemcpyHostToDevice,
                            b->stream));
      CK(b, cudaStreamSynchronize(b->stream));
      return LBM_OK;
    }
  return set_err(b->err, LBM_EINVAL, "no guarded buffer %d", which);
}

int lbm_batch_launches_per_step(const lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  return b->b.n_items > 0 ? (b->b.persist ? 1 : b->b.n_groups) : 0;
}

int lbm_batch_run_to_equilibrium(lbm_batch* bb, double tol, int check_every,
                                 long long max_steps, long long* steps_out) {
  Range r_("lbm_batch_run_to_equilibrium");
  DeviceGuard g_(bb ? &bb->b : nullptr);
  if (!bb) return LBM_EINVAL;
  Batch* b = &bb->b;
  if (!(tol > 0) || check_every < 1 || max_steps < 0)
    return set_err(b->err, LBM_EINVAL, "need tol > 0, check_every >= 1, max_steps >= 0");
  std::vector<lbm_diag> d(b->n_inst);
  if (steps_out)
    for (int i = 0; i < b->n_inst; ++i) steps_out[i] = -1;
  int rc = diagnostics(b, d.data());  // seeds the dinf reference
  if (rc) return rc;
  long long taken = 0;
  while (taken < max_steps && b->n_items > 0) {
    const long long k = std::min<long long>(check_every, max_steps - taken);
    rc = do_steps(b, k);
    if (rc) return rc;
    taken += k;
    rc = diagnostics(b, d.data());
    if (rc) return rc;
    bool changed = false;
    for (int i = 0; i < b->n_inst; ++i) {
      if (!b->active[i]) continue;
      const bool bad = d[i].nonfinite > 0;
      const bool conv = !bad && d[i].dinf >= 0 && d[i].dinf < tol && k == check_every;
      if (conv || bad) {
        if (conv && steps_out) steps_out[i] = b->steps[i];
        rc = freeze(b, i);
        if (rc) return rc;
        changed = true;
      }
    }
    if (changed) {
      rc = rebuild_items(b);
      if (rc) return rc;
    }
  }
  int left = 0;
  for (int a : b->active) left += a;
  return left;
}

}  // extern "C"
