// Batched ensembles: n independent lattices (own size, parameters, obstacle
// mask and state) advanced together.  The paper has no counterpart; every
// replica runs the fused step of lb_kernels.cuh unchanged.
//
// Work list: one item per (replica, tile); a replica table in the workspace
// holds each replica's kernel constants and buffer pointers.  Two schedules:
//   0  per-step: one launch per time step over all items (grid = items),
//      replayed from a CUDA graph of kBatchGraphLen steps;
//   1  persistent: one cooperative launch of co-resident CTAs runs K steps;
//      CTA b owns items b, b + G, b + 2G, ... and runs them back to back,
//      then meets every other CTA at a grid-wide barrier before the next
//      step.  The barrier is a generation counter: each CTA reads the
//      generation, arrives with one atom.add.acq_rel on the arrival count
//      (after a CTA barrier, so the release covers all its threads' stores),
//      and the last arriver resets the count and releases the next
//      generation, which the others wait for with ld.acquire, bounded by a
//      clock budget.  The barrier orders every read of a buffer after all
//      of the previous step's writes to it and every write after all of the
//      previous step's reads, so the step's loads may go through L1: no
//      load of a buffer is in flight across the barrier that orders its
//      writes.  A wait that runs out sets an error word; every CTA then
//      leaves, and the host reports LB_ETIMEOUT.
// The schedule and the tile shape are picked by lb_batch_autotune.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lb_host.h"
#include "lb_kernels.cuh"

using namespace tlb;

namespace tlb {

template <class S> struct ReplicaDesc {
  KParams<S> kp;
  S* buf[2];
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <class S, bool SHIFT, int TX, int TY, int BY, int MB>
__global__ void __launch_bounds__(TX * BY, MB)
lb_batch_step_kernel(const ReplicaDesc<S>* __restrict__ reps, const int4* __restrict__ items, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileSmem<S, TX, TY, false>*>(smem_raw);
  const int4 it = items[blockIdx.x];
  const ReplicaDesc<S>& rd = reps[it.x];  // read-only table: uniform cached loads
  double acc[kObsSlots];
  tile_step<S, S, SHIFT, MODE_STEP, TX, TY, BY, false>(rd.buf[parity], rd.buf[parity ^ 1], rd.kp, it.y, it.z, sm,
                                                       nullptr, acc);
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch (bar[0] arrivals, bar[1] generation); false when a wait ran
// out or another CTA reported one (the caller then leaves).
__device__ __forceinline__ bool grid_barrier(int* bar, int* err, long long budget, int tid) {
  __shared__ int s_ok;
  __syncthreads();
  if (tid == 0) {
    int ok = 1;
    const int g = ld_relaxed_gpu(bar + 1);
    if (atom_add_acq_rel_gpu(bar, 1) == (int)gridDim.x - 1) {
      st_relaxed_gpu(bar, 0);
      st_release_gpu(bar + 1, g + 1);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu(bar + 1) == g) {
        if (ld_relaxed_gpu(err) != 0) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > budget) {
          atomicCAS(err, 0, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class S, bool SHIFT, int TX, int TY, int BY, int MB>
__global__ void __launch_bounds__(TX * BY, MB)
lb_batch_persistent_kernel(const ReplicaDesc<S>* __restrict__ reps, const int4* __restrict__ items, int* bar, int* err,
                           int n_items, int parity0, int n_steps, long long budget, int withhold) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileSmem<S, TX, TY, false>*>(smem_raw);
  const int tid = threadIdx.y * TX + threadIdx.x;
  // failure-detection hook: CTA `withhold` (mod the grid) leaves before the first step barrier
  const bool withheld = withhold >= 0 && withhold % (int)gridDim.x == (int)blockIdx.x;
  double acc[kObsSlots];
  for (int s = 0; s < n_steps; ++s) {
    const int parity = (parity0 + s) & 1;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
      const int4 it = items[item];
      const ReplicaDesc<S>& rd = reps[it.x];
      tile_step<S, S, SHIFT, MODE_STEP, TX, TY, BY>(rd.buf[parity], rd.buf[parity ^ 1], rd.kp, it.y, it.z, sm, nullptr,
                                                    acc);
      __syncthreads();  // the next item's phase A rewrites the shared memory
    }
    if (s + 1 == n_steps) break;  // the launch boundary orders the last step
    if (withheld) return;
    if (!grid_barrier(bar, err, budget, tid)) return;
  }
}

struct BatchArgs {
  const void* reps;
  const int4* items;
  int* counters;
  int* err;
  int n_items;
  int parity;
  int n_steps;
  long long budget;
  int withhold;
};

using BatchStepFn = cudaError_t (*)(const BatchArgs&, cudaStream_t);
using BatchPersFn = cudaError_t (*)(const BatchArgs&, int grid, cudaStream_t);
using BatchOccFn = cudaError_t (*)(int* blocks_per_sm);

template <class S, bool SHIFT, int TX, int TY, int BY, int MB> struct BatchKernels {
  static constexpr size_t kSmem = sizeof(TileSmem<S, TX, TY, false>);

  static cudaError_t set_attr(const void* fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  }
  static cudaError_t step(const BatchArgs& a, cudaStream_t s) {
    auto k = lb_batch_step_kernel<S, SHIFT, TX, TY, BY, MB>;
    cudaError_t e = set_attr((const void*)k);
    if (e != cudaSuccess) return e;
    k<<<a.n_items, dim3(TX, BY, 1), kSmem, s>>>(static_cast<const ReplicaDesc<S>*>(a.reps), a.items, a.parity);
    return cudaGetLastError();
  }
  static cudaError_t occupancy(int* blocks) {
    auto k = lb_batch_persistent_kernel<S, SHIFT, TX, TY, BY, MB>;
    cudaError_t e = set_attr((const void*)k);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, TX * BY, kSmem);
  }
  static cudaError_t persistent(const BatchArgs& a, int grid, cudaStream_t s) {
    auto k = lb_batch_persistent_kernel<S, SHIFT, TX, TY, BY, MB>;
    cudaError_t e = set_attr((const void*)k);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(TX, BY, 1);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<const ReplicaDesc<S>*>(a.reps), a.items, a.counters, a.err,
                              a.n_items, a.parity, a.n_steps, a.budget, a.withhold);
  }
};

struct BatchCand {
  TileChoice t;
  BatchStepFn step;
  BatchPersFn persistent;
  BatchOccFn occupancy;
};

#define TLB_BATCH_CAND(S, SH, TX, TY, BY, MB)                                                 \
  {{TX, TY, BY, MB}, BatchKernels<S, SH, TX, TY, BY, MB>::step, BatchKernels<S, SH, TX, TY, BY, MB>::persistent, \
   BatchKernels<S, SH, TX, TY, BY, MB>::occupancy}

const BatchCand kBatchF32[] = {
    TLB_BATCH_CAND(float, true, 64, 8, 4, 4),
    TLB_BATCH_CAND(float, true, 64, 16, 4, 3),
    TLB_BATCH_CAND(float, true, 32, 16, 8, 3),
    TLB_BATCH_CAND(float, true, 128, 16, 2, 3),
    TLB_BATCH_CAND(float, true, 32, 8, 8, 4),
};
const BatchCand kBatchF64[] = {
    TLB_BATCH_CAND(double, false, 32, 16, 8, 2),
    TLB_BATCH_CAND(double, false, 64, 16, 4, 2),
};

}  // namespace tlb

namespace {

constexpr int kBatchGraphLen = 16;
constexpr int kMinTileX = 32, kMinTileY = 8;  // smallest batch tile: sizes the item tables
thread_local char g_batch_err[512] = "no error";

const BatchCand* cands(int precision, int* n) {
  if (precision == LB_FP64) {
    *n = (int)(sizeof kBatchF64 / sizeof kBatchF64[0]);
    return kBatchF64;
  }
  *n = (int)(sizeof kBatchF32 / sizeof kBatchF32[0]);
  return kBatchF32;
}

}  // namespace

struct lb_batch {
  int n = 0, precision = 0;
  std::vector<lb_params> p;
  std::vector<Layout> L;
  std::vector<size_t> base;
  std::vector<StepCfg> cfg;
  unsigned char* ws = nullptr;
  size_t reps_off = 0, items_off = 0, counters_off = 0, err_off = 0;
  int max_items = 0, n_items = 0;
  int schedule = 0, tile = 0, steps_per_launch = 64, grid = 0;
  int parity = 0;
  long long step = 0;
  long long budget = 4000000000LL;  // SM clock cycles a persistent wait may spin (about 2 s)
  int withhold = -1;
  int graphs_ok = 1;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  char err[512] = "no error";
};

namespace {

int bfail(lb_batch* b, int code, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define BCUDA(b, call)                                                                            \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return bfail((b), LB_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int tiles_of(const lb_params& p, int tx, int ty) { return ((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty); }

size_t desc_bytes(int precision) {
  return precision == LB_FP64 ? sizeof(ReplicaDesc<double>) : sizeof(ReplicaDesc<float>);
}

// Offsets of every replica and of the batch tables.
size_t batch_layout(const lb_params* reps, int n, const int* has_mask, std::vector<Layout>* L, std::vector<size_t>* base,
                    size_t* reps_off, size_t* items_off, size_t* counters_off, size_t* err_off,
                    int* max_items) {
  size_t off = 0;
  int items = 0;
  for (int r = 0; r < n; ++r) {
    const Layout l = layout_for(&reps[r], has_mask ? has_mask[r] : 0);
    if (L) L->push_back(l);
    if (base) base->push_back(off);
    off += round_up(l.total, kAlign);
    items += tiles_of(reps[r], kMinTileX, kMinTileY);
  }
  *reps_off = off;
  off += round_up((size_t)n * desc_bytes(reps[0].precision), kAlign);
  *items_off = off;
  off += round_up((size_t)items * sizeof(int4), kAlign);
  *counters_off = off;  // persistent schedule: step barrier (arrivals, generation)
  off += kAlign;
  *err_off = off;
  off += kAlign;
  *max_items = items;
  return off;
}

// Work list for tile candidate k; uploads it and sizes the persistent grid.
int configure(lb_batch* b, int schedule, int tile, int steps_per_launch) {
  int nc = 0;
  const BatchCand* cs = cands(b->precision, &nc);
  if (tile < 0 || tile >= nc) return bfail(b, LB_EINVAL, "tile candidate out of range");
  if (schedule != 0 && schedule != 1) return bfail(b, LB_EINVAL, "schedule must be 0 (per-step) or 1 (persistent)");
  if (steps_per_launch < 2 || (steps_per_launch & 1)) return bfail(b, LB_EINVAL, "steps_per_launch must be even, >= 2");
  const TileChoice t = cs[tile].t;
  std::vector<int4> items;
  for (int r = 0; r < b->n; ++r) {
    const lb_params& p = b->p[r];
    const int ntx = (p.nx + t.tx - 1) / t.tx, nty = (p.ny + t.ty - 1) / t.ty;
    for (int ty = 0; ty < nty; ++ty)
      for (int tx = 0; tx < ntx; ++tx) items.push_back(make_int4(r, tx * t.tx, ty * t.ty, 0));
  }
  if ((int)items.size() > b->max_items) return bfail(b, LB_EINVAL, "work list larger than its table");
  BCUDA(b, cudaStreamSynchronize(b->stream));
  BCUDA(b, cudaMemcpy(b->ws + b->items_off, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  int occ = 0, dev = 0, sms = 0;
  BCUDA(b, cs[tile].occupancy(&occ));
  BCUDA(b, cudaGetDevice(&dev));
  BCUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (occ < 1) return bfail(b, LB_EINVAL, "persistent kernel cannot be resident");
  b->n_items = (int)items.size();
  b->grid = b->n_items < occ * sms ? b->n_items : occ * sms;
  for (auto& g : b->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  b->schedule = schedule;
  b->tile = tile;
  b->steps_per_launch = steps_per_launch;
  return LB_OK;
}

BatchArgs args_for(const lb_batch* b, int parity, int n_steps) {
  BatchArgs a;
  a.reps = b->ws + b->reps_off;
  a.items = reinterpret_cast<const int4*>(b->ws + b->items_off);
  a.counters = reinterpret_cast<int*>(b->ws + b->counters_off);
  a.err = reinterpret_cast<int*>(b->ws + b->err_off);
  a.n_items = b->n_items;
  a.parity = parity;
  a.n_steps = n_steps;
  a.budget = b->budget;
  a.withhold = b->withhold;
  return a;
}

// Enqueue `steps` steps starting at buffer parity `parity` on stream s (no graphs).
cudaError_t enqueue(const lb_batch* b, int parity, int steps, cudaStream_t s) {
  int nc = 0;
  const BatchCand& c = cands(b->precision, &nc)[b->tile];
  if (b->schedule == 0) {
    for (int k = 0; k < steps; ++k) {
      cudaError_t e = c.step(args_for(b, (parity + k) & 1, 1), s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaMemsetAsync(b->ws + b->counters_off, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  return c.persistent(args_for(b, parity, steps), b->grid, s);
}

int graph_len(const lb_batch* b) { return b->schedule == 0 ? kBatchGraphLen : b->steps_per_launch; }

int build_graph(lb_batch* b, int parity) {
  cudaGraph_t g = nullptr;
  BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue(b, parity, graph_len(b), b->cap);
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->gexec[parity] = nullptr;
    return LB_ECUDA;
  }
  return LB_OK;
}

int do_steps(lb_batch* b, int n) {
  const int L = graph_len(b);
  while (n >= L) {
    if (b->graphs_ok && !b->gexec[b->parity] && build_graph(b, b->parity) != LB_OK) b->graphs_ok = 0;
    if (b->graphs_ok && b->gexec[b->parity]) {
      BCUDA(b, cudaGraphLaunch(b->gexec[b->parity], b->stream));
    } else {
      BCUDA(b, enqueue(b, b->parity, L, b->stream));
    }
    n -= L;
    b->step += L;  // L is even: the parity is unchanged
  }
  if (n > 0) {
    BCUDA(b, enqueue(b, b->parity, n, b->stream));
    b->parity = (b->parity + n) & 1;
    b->step += n;
  }
  return LB_OK;
}

int check_err_word(lb_batch* b) {
  int v = 0;
  BCUDA(b, cudaMemcpyAsync(&v, b->ws + b->err_off, sizeof v, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  if (v != 0) return bfail(b, LB_ETIMEOUT, "a persistent-kernel wait at the step barrier ran out; the state is invalid");
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_batch_workspace_size(const lb_params* reps, int n, const int* has_mask, size_t* bytes) {
  if (!reps || n < 1 || !bytes) return bfail(nullptr, LB_EINVAL, "reps, n >= 1 and bytes are required");
  for (int r = 0; r < n; ++r) {
    if (const char* why = check_params(&reps[r])) return bfail(nullptr, LB_EINVAL, "replica %d: %s", r, why);
    if (reps[r].precision != reps[0].precision) return bfail(nullptr, LB_EINVAL, "all replicas need one precision");
    if (reps[r].precision == LB_FP32_FP16T || reps[r].precision == LB_DF64)
      return bfail(nullptr, LB_EINVAL, "batched ensembles store LB_FP64 or LB_FP32_SHIFTED");
  }
  size_t a, c, e, f;
  int m;
  *bytes = batch_layout(reps, n, has_mask, nullptr, nullptr, &a, &c, &e, &f, &m);
  return LB_OK;
}

int lb_batch_init(lb_batch** out, const lb_params* reps, int n, const uint8_t* const* masks, const double* const* rho1,
                  const double* const* rho2, const double* const* T0, void* d_workspace, size_t ws_bytes,
                  void* stream) {
  if (!out) return bfail(nullptr, LB_EINVAL, "batch pointer is NULL");
  *out = nullptr;
  if (!reps || n < 1 || !rho1 || !rho2 || !T0) return bfail(nullptr, LB_EINVAL, "reps, n >= 1 and fields are required");
  std::vector<int> has_mask(n, 0);
  for (int r = 0; r < n; ++r) {
    if (const char* why = check_params(&reps[r])) return bfail(nullptr, LB_EINVAL, "replica %d: %s", r, why);
    if (reps[r].precision != reps[0].precision) return bfail(nullptr, LB_EINVAL, "all replicas need one precision");
    if (reps[r].precision == LB_FP32_FP16T || reps[r].precision == LB_DF64)
      return bfail(nullptr, LB_EINVAL, "batched ensembles store LB_FP64 or LB_FP32_SHIFTED");
    has_mask[r] = masks && masks[r] ? 1 : 0;
    if (has_mask[r] && reps[r].periodic_y) return bfail(nullptr, LB_EINVAL, "replica %d: mask needs walls", r);
    if (!rho1[r] || !rho2[r] || !T0[r]) return bfail(nullptr, LB_EINVAL, "replica %d: fields are required", r);
  }
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return bfail(nullptr, LB_EINVAL, "out of host memory");
  b->n = n;
  b->precision = reps[0].precision;
  b->p.assign(reps, reps + n);
  const size_t total = batch_layout(reps, n, has_mask.data(), &b->L, &b->base, &b->reps_off, &b->items_off,
                                    &b->counters_off, &b->err_off, &b->max_items);
  auto bail = [&](int code) {
    std::snprintf(g_batch_err, sizeof g_batch_err, "%s", b->err);
    lb_batch_destroy(b);
    return code;
  };
  if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0)
    return bail(bfail(b, LB_ENOSPACE, "workspace must be a 256-byte aligned device pointer"));
  if (ws_bytes < total) return bail(bfail(b, LB_ENOSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, total));
  b->ws = static_cast<unsigned char*>(d_workspace);
  b->stream = static_cast<cudaStream_t>(stream);
  for (int r = 0; r < n; ++r) {
    char why[256];
    if (const char* bad = prepare_fields(b->p[r], has_mask[r] ? masks[r] : nullptr, rho1[r], rho2[r], T0[r], why,
                                         sizeof why))
      return bail(bfail(b, LB_EINVAL, "replica %d: %s", r, bad));
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(bfail(b, LB_ECUDA, "cudaStreamCreate failed"));
  std::vector<unsigned char> descs((size_t)n * desc_bytes(b->precision));
  cudaError_t e = cudaMemsetAsync(b->ws, 0, total, b->stream);
  for (int r = 0; r < n && e == cudaSuccess; ++r) {
    const Layout& L = b->L[r];
    unsigned char* rb = b->ws + b->base[r];
    uint8_t* d_mask = has_mask[r] ? rb + L.mask_off : nullptr;
    b->cfg.push_back(make_stepcfg(b->p[r], L.pitch, d_mask));
    const size_t N = (size_t)b->p[r].nx * b->p[r].ny;
    double* stage = reinterpret_cast<double*>(rb + L.buf_bytes);
    if (d_mask) e = cudaMemcpyAsync(d_mask, masks[r], N, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage, rho1[r], N * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + N, rho2[r], N * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 2 * N, T0[r], N * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = b->precision == LB_FP64 ? init_f64(b->cfg[r], stage, rb, b->stream) : init_f32(b->cfg[r], stage, rb, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(rb + L.buf_bytes, 0, L.buf_bytes, b->stream);
    if (b->precision == LB_FP64) {
      ReplicaDesc<double> d;
      d.kp = make_kparams<double>(b->cfg[r]);
      d.buf[0] = reinterpret_cast<double*>(rb);
      d.buf[1] = reinterpret_cast<double*>(rb + L.buf_bytes);
      std::memcpy(descs.data() + r * sizeof d, &d, sizeof d);
    } else {
      ReplicaDesc<float> d;
      d.kp = make_kparams<float>(b->cfg[r]);
      d.buf[0] = reinterpret_cast<float*>(rb);
      d.buf[1] = reinterpret_cast<float*>(rb + L.buf_bytes);
      std::memcpy(descs.data() + r * sizeof d, &d, sizeof d);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + b->reps_off, descs.data(), descs.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bail(bfail(b, LB_ECUDA, "lb_batch_init: %s", cudaGetErrorString(e)));
  if (int rc = configure(b, 0, 0, 64)) return bail(rc);
  *out = b;
  return LB_OK;
}

int lb_batch_step(lb_batch* b, int n) {
  if (!b) return bfail(nullptr, LB_EINVAL, "batch is NULL");
  if (n < 0) return bfail(b, LB_EINVAL, "n must be >= 0");
  return do_steps(b, n);
}

int lb_batch_configure(lb_batch* b, int schedule, int tile, int steps_per_launch) {
  if (!b) return bfail(nullptr, LB_EINVAL, "batch is NULL");
  return configure(b, schedule, tile, steps_per_launch);
}

int lb_batch_autotune(lb_batch* b, int trial_steps, int* schedule, int* tile, long long* steps_taken, double* ms,
                      int n_slots) {
  if (!b) return bfail(nullptr, LB_EINVAL, "batch is NULL");
  if (trial_steps < 2 || (trial_steps & 1)) return bfail(b, LB_EINVAL, "trial_steps must be even and >= 2");
  int nc = 0;
  cands(b->precision, &nc);
  if (ms && n_slots < 2 * nc) return bfail(b, LB_EINVAL, "ms needs %d slots", 2 * nc);
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  const long long step0 = b->step;
  double best = -1.0;
  int best_s = 0, best_t = 0, rc = LB_OK;
  for (int sch = 0; sch < 2 && rc == LB_OK; ++sch)
    for (int t = 0; t < nc && rc == LB_OK; ++t) {
      rc = configure(b, sch, t, trial_steps);
      if (rc) break;
      rc = do_steps(b, trial_steps);  // warm-up (builds the graph)
      if (rc) break;
      cudaEventRecord(e0, b->stream);
      rc = do_steps(b, trial_steps);
      cudaEventRecord(e1, b->stream);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = bfail(b, LB_ECUDA, "autotune trial failed");
        break;
      }
      rc = check_err_word(b);
      if (rc) break;
      float t_ms = 0.0f;
      cudaEventElapsedTime(&t_ms, e0, e1);
      const double per = t_ms / trial_steps;
      if (ms) ms[sch * nc + t] = per;
      if (best < 0 || per < best) {
        best = per;
        best_s = sch;
        best_t = t;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (steps_taken) *steps_taken = b->step - step0;
  if (rc) return rc;
  if (int r2 = configure(b, best_s, best_t, 64)) return r2;
  if (schedule) *schedule = best_s;
  if (tile) *tile = best_t;
  return LB_OK;
}

int lb_batch_info(const lb_batch* b, int* n_items, int* grid, int* schedule, int* tile, int* graphs) {
  if (!b) return bfail(nullptr, LB_EINVAL, "batch is NULL");
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid;
  if (schedule) *schedule = b->schedule;
  if (tile) *tile = b->tile;
  if (graphs) *graphs = b->graphs_ok;
  int nc = 0;
  cands(b->precision, &nc);
  return nc;
}

int lb_batch_sync(lb_batch* b) {
  if (!b) return bfail(nullptr, LB_EINVAL, "batch is NULL");
  BCUDA(b, cudaStreamSynchronize(b->stream));
  BCUDA(b, cudaGetLastError());
  return check_err_word(b);
}

int lb_batch_observables(lb_batch* b, int r, lb_obs* out) {
  if (!b || !out || r < 0 || r >= b->n) return bfail(b, LB_EINVAL, "batch, replica and out are required");
  if (int rc = check_err_word(b)) return rc;
  unsigned char* rb = b->ws + b->base[r];
  const Layout& L = b->L[r];
  double* part = reinterpret_cast<double*>(rb + L.part_off);
  double* dobs = reinterpret_cast<double*>(rb + L.obs_off);
  void* cur = rb + (b->parity ? L.buf_bytes : 0);
  BCUDA(b, b->precision == LB_FP64 ? launch_f64(MODE_OBS, b->cfg[r], cur, nullptr, part, b->stream)
                                   : launch_f32(MODE_OBS, b->cfg[r], cur, nullptr, part, b->stream));
  BCUDA(b, obs_finalize(b->cfg[r], part, L.n_blocks, dobs, b->stream));
  double v[kObsOut];
  BCUDA(b, cudaMemcpyAsync(v, dobs, sizeof v, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  out->mass[0] = v[0];
  out->mass[1] = v[1];
  out->mom[0] = v[2];
  out->mom[1] = v[3];
  out->Nu = v[4];
  out->E = v[5];
  out->n_bad = (long long)v[6];
  out->n_fluid = (long long)v[7];
  out->step = b->step;
  out->status = out->n_bad > 0 ? LB_EUNSTABLE : LB_OK;
  out->_pad = 0;
  out->wall_fx[0] = v[10];
  out->wall_fx[1] = v[11];
  return out->status;
}

int lb_batch_get_fields(lb_batch* b, int r, double* rho1, double* rho2, double* T, double* ux, double* uy) {
  if (!b || r < 0 || r >= b->n) return bfail(b, LB_EINVAL, "batch and replica are required");
  if (int rc = check_err_word(b)) return rc;
  unsigned char* rb = b->ws + b->base[r];
  const Layout& L = b->L[r];
  void* cur = rb + (b->parity ? L.buf_bytes : 0);
  double* stage = reinterpret_cast<double*>(rb + (b->parity ? 0 : L.buf_bytes));
  BCUDA(b, b->precision == LB_FP64 ? launch_f64(MODE_FIELDS, b->cfg[r], cur, nullptr, stage, b->stream)
                                   : launch_f32(MODE_FIELDS, b->cfg[r], cur, nullptr, stage, b->stream));
  const size_t N = (size_t)b->p[r].nx * b->p[r].ny;
  double* dst[5] = {rho1, rho2, T, ux, uy};
  for (int k = 0; k < 5; ++k)
    if (dst[k]) BCUDA(b, cudaMemcpyAsync(dst[k], stage + k * N, N * 8, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return LB_OK;
}

int lb_batch_stress(lb_batch* b, int r, double* out4, double* row, double* field) {
  if (!b || r < 0 || r >= b->n) return bfail(b, LB_EINVAL, "batch and replica are required");
  if (!out4 && !row && !field) return bfail(b, LB_EINVAL, "lb_batch_stress: no output requested");
  if (int rc = check_err_word(b)) return rc;
  unsigned char* rb = b->ws + b->base[r];
  const Layout& L = b->L[r];
  void* cur = rb + (b->parity ? L.buf_bytes : 0);
  double* stage = reinterpret_cast<double*>(rb + (b->parity ? 0 : L.buf_bytes));
  double *d_rows = nullptr, *d_tot = nullptr;
  BCUDA(b, stress_run(b->cfg[r], b->precision, cur, stage, b->stream, &d_rows, &d_tot));
  BCUDA(b, stress_fetch(b->p[r].nx, b->p[r].ny, stage, d_rows, d_tot, out4, row, field, b->stream));
  return LB_OK;
}

int lb_batch_get_state(lb_batch* b, int r, double* host, size_t bytes) {
  if (!b || !host || r < 0 || r >= b->n) return bfail(b, LB_EINVAL, "batch, replica and host buffer are required");
  const size_t N = (size_t)b->p[r].nx * b->p[r].ny;
  if (bytes != 27 * N * 8) return bfail(b, LB_EINVAL, "state needs %zu bytes", 27 * N * 8);
  if (int rc = check_err_word(b)) return rc;
  unsigned char* rb = b->ws + b->base[r];
  const Layout& L = b->L[r];
  void* cur = rb + (b->parity ? L.buf_bytes : 0);
  double* stage = reinterpret_cast<double*>(rb + (b->parity ? 0 : L.buf_bytes));
  for (int k = 0; k < 27; ++k) {
    BCUDA(b, b->precision == LB_FP64 ? plane_get_f64(b->cfg[r], k, cur, stage, b->stream)
                                     : plane_get_f32(b->cfg[r], k, cur, stage, b->stream));
    BCUDA(b, cudaMemcpyAsync(host + k * N, stage, N * 8, cudaMemcpyDeviceToHost, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  return LB_OK;
}

int lb_batch_set_wait_budget(lb_batch* b, long long cycles, int withhold_item) {
  if (!b || cycles < 1) return bfail(b, LB_EINVAL, "batch and a positive budget are required");
  b->budget = cycles;
  b->withhold = withhold_item;
  for (auto& g : b->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& g : b->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err : g_batch_err; }

}  // extern "C"
