// Host side of the C ABI declared in include/tlb.h: parameter validation,
// workspace layout, CUDA-graph replay of the fused step, observables,
// fields and state transfer.  Every numerical step runs in the kernels of
// lb_f64.cu / lb_f32.cu; this file only marshals pointers and launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lb_cfg.h"
#include "lb_host.h"
#include "tlb.h"

using namespace tlb;

namespace {

constexpr int kGraphLen = 16;  // steps per captured graph (even: replay keeps the buffer parity)

thread_local char g_err[512] = "no error";

}  // namespace


namespace {

int fail(lb_handle* h, int code, const char* fmt, ...) {
  char* dst = h ? h->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail((h), LB_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

cudaError_t launch(const lb_handle* h, int mode, const void* fin, void* fout, double* aux, cudaStream_t s) {
  const int pr = h->p.precision;
  if (mode == MODE_STEP) {
    switch (pr) {
      case LB_FP64: return launch_step_tile_f64(h->tile, h->cfg, fin, fout, s);
      case LB_FP32_SHIFTED: return launch_step_tile_f32(h->tile, h->cfg, fin, fout, s);
      case LB_FP32_FP16T: return launch_step_tile_f32h(h->tile, h->cfg, fin, fout, s);
      default: return launch_step_tile_df64(h->tile, h->cfg, fin, fout, s);
    }
  }
  return launch_mode(pr, mode, h->cfg, fin, fout, aux, s);
}

int tile_count(const lb_handle* h) {
  switch (h->p.precision) {
    case LB_FP64: return tile_count_f64();
    case LB_FP32_SHIFTED: return tile_count_f32();
    case LB_FP32_FP16T: return tile_count_f32h();
    default: return tile_count_df64();
  }
}

TileChoice tile_info(const lb_handle* h, int k) {
  switch (h->p.precision) {
    case LB_FP64: return tile_info_f64(k);
    case LB_FP32_SHIFTED: return tile_info_f32(k);
    case LB_FP32_FP16T: return tile_info_f32h(k);
    default: return tile_info_df64(k);
  }
}

cudaError_t init_buffer(const lb_handle* h, const double* fields, void* buf) {
  switch (h->p.precision) {
    case LB_FP64: return init_f64(h->cfg, fields, buf, h->stream);
    case LB_FP32_SHIFTED: return init_f32(h->cfg, fields, buf, h->stream);
    case LB_FP32_FP16T: return init_f32h(h->cfg, fields, buf, h->stream);
    default: return init_df64(h->cfg, fields, buf, h->stream);
  }
}

cudaError_t plane_get(const lb_handle* h, int k, const void* buf, double* out) {
  switch (h->p.precision) {
    case LB_FP64: return plane_get_f64(h->cfg, k, buf, out, h->stream);
    case LB_FP32_SHIFTED: return plane_get_f32(h->cfg, k, buf, out, h->stream);
    case LB_FP32_FP16T: return plane_get_f32h(h->cfg, k, buf, out, h->stream);
    default: return plane_get_df64(h->cfg, k, buf, out, h->stream);
  }
}

cudaError_t plane_put(const lb_handle* h, int k, const double* in, void* buf) {
  switch (h->p.precision) {
    case LB_FP64: return plane_put_f64(h->cfg, k, in, buf, h->stream);
    case LB_FP32_SHIFTED: return plane_put_f32(h->cfg, k, in, buf, h->stream);
    case LB_FP32_FP16T: return plane_put_f32h(h->cfg, k, in, buf, h->stream);
    default: return plane_put_df64(h->cfg, k, in, buf, h->stream);
  }
}

void drop_graphs(lb_handle* h) {
  for (auto& g : h->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void fill_cfg(lb_handle* h, const uint8_t* d_mask) {
  h->cfg = make_stepcfg(h->p, h->L.pitch, d_mask);
}

int build_graph(lb_handle* h, int parity) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  int b = parity;
  for (int s = 0; s < kGraphLen; ++s) {
    cudaError_t e = launch(h, MODE_STEP, h->buf[b], h->buf[b ^ 1], nullptr, h->cap);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(h->cap, &g);
      if (g) cudaGraphDestroy(g);
      return fail(h, LB_ECUDA, "step launch during capture: %s", cudaGetErrorString(e));
    }
    b ^= 1;
  }
  CUDA_TRY(h, cudaStreamEndCapture(h->cap, &g));
  cudaError_t e = cudaGraphInstantiate(&h->gexec[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, LB_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_version(void) { return "tlb-gb300 0.1 (sm_103a)"; }

const char* lb_last_error(const lb_handle* h) { return h ? h->err : g_err; }

int lb_workspace_size(const lb_params* p, int has_mask, size_t* bytes) {
  if (const char* why = check_params(p)) return fail(nullptr, LB_EINVAL, "%s", why);
  if (!bytes) return fail(nullptr, LB_EINVAL, "bytes is NULL");
  *bytes = layout_for(p, has_mask).total;
  return LB_OK;
}

int lb_init(lb_handle** out, const lb_params* pin, const uint8_t* mask, const double* rho1, const double* rho2,
            const double* T0, void* d_workspace, size_t ws_bytes, void* stream) {
  if (!out) return fail(nullptr, LB_EINVAL, "handle pointer is NULL");
  *out = nullptr;
  if (const char* why = check_params(pin)) return fail(nullptr, LB_EINVAL, "%s", why);
  if (!rho1 || !rho2 || !T0) return fail(nullptr, LB_EINVAL, "rho1, rho2 and T0 are required");
  if (mask && pin->periodic_y) return fail(nullptr, LB_EINVAL, "an obstacle mask needs walls (periodic_y = 0)");
  lb_params p = *pin;
  const Layout L = layout_for(&p, mask != nullptr);
  if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0)
    return fail(nullptr, LB_ENOSPACE, "workspace must be a 256-byte aligned device pointer");
  if (ws_bytes < L.total) return fail(nullptr, LB_ENOSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, L.total);
  {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return fail(nullptr, LB_ENOSPACE, "workspace is not device memory");
    }
  }
  // initial fields: finite, positive densities at fluid nodes; shifts default to the fluid means
  const size_t N = (size_t)p.nx * p.ny;
  {
    char why[256];
    if (const char* bad = prepare_fields(p, mask, rho1, rho2, T0, why, sizeof why))
      return fail(nullptr, LB_EINVAL, "%s", bad);
  }

  lb_handle* h = new (std::nothrow) lb_handle();
  if (!h) return fail(nullptr, LB_EINVAL, "out of host memory");
  h->p = p;
  h->L = L;
  h->stream = static_cast<cudaStream_t>(stream);
  h->ws = static_cast<unsigned char*>(d_workspace);
  h->buf[0] = h->ws;
  h->buf[1] = h->ws + L.buf_bytes;
  uint8_t* d_mask = mask ? h->ws + L.mask_off : nullptr;
  fill_cfg(h, d_mask);

  auto bail = [&](int code) {
    char msg[512];
    std::snprintf(msg, sizeof msg, "%s", h->err);
    lb_destroy(h);
    return fail(nullptr, code, "%s", msg);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && p.precision == LB_DF64) e = df_exp_tables_init();
  if (e != cudaSuccess) return bail(fail(h, LB_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
  e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);  // buffers, partials and the error word start at zero
  if (e == cudaSuccess && mask) e = cudaMemcpyAsync(d_mask, mask, N, cudaMemcpyHostToDevice, h->stream);
  double* stage = static_cast<double*>(h->buf[1]);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, rho1, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + N, rho2, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 2 * N, T0, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = init_buffer(h, stage, h->buf[0]);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, L.buf_bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bail(fail(h, LB_ECUDA, "lb_init: %s", cudaGetErrorString(e)));
  h->cur = 0;
  h->step = 0;
  *out = h;
  return LB_OK;
}

int lb_step(lb_handle* h, int n) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  if (n < 0) return fail(h, LB_EINVAL, "n must be >= 0");
  while (n >= kGraphLen) {
    if (!h->gexec[h->cur]) {
      int rc = build_graph(h, h->cur);
      if (rc) return rc;
    }
    CUDA_TRY(h, cudaGraphLaunch(h->gexec[h->cur], h->stream));
    n -= kGraphLen;
    h->step += kGraphLen;
  }
  for (; n > 0; --n) {
    CUDA_TRY(h, launch(h, MODE_STEP, h->buf[h->cur], h->buf[h->cur ^ 1], nullptr, h->stream));
    h->cur ^= 1;
    h->step += 1;
  }
  return LB_OK;
}

int lb_observables(lb_handle* h, lb_obs* out) {
  if (!h || !out) return fail(h, LB_EINVAL, "handle and out are required");
  double* part = reinterpret_cast<double*>(h->ws + h->L.part_off);
  double* dobs = reinterpret_cast<double*>(h->ws + h->L.obs_off);
  CUDA_TRY(h, launch(h, MODE_OBS, h->buf[h->cur], nullptr, part, h->stream));
  CUDA_TRY(h, obs_finalize(h->cfg, part, h->L.n_blocks, dobs, h->stream));
  double v[kObsOut];
  CUDA_TRY(h, cudaMemcpyAsync(v, dobs, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  out->mass[0] = v[0];
  out->mass[1] = v[1];
  out->mom[0] = v[2];
  out->mom[1] = v[3];
  out->Nu = v[4];
  out->E = v[5];
  out->n_bad = (long long)v[6];
  out->n_fluid = (long long)v[7];
  out->step = h->step;
  out->status = out->n_bad > 0 ? LB_EUNSTABLE : LB_OK;
  out->_pad = 0;
  out->wall_fx[0] = v[10];
  out->wall_fx[1] = v[11];
  if (out->status != LB_OK) return fail(h, LB_EUNSTABLE, "%lld fluid nodes with non-finite or non-positive density", out->n_bad);
  return LB_OK;
}

int lb_get_fields(lb_handle* h, double* rho1, double* rho2, double* T, double* ux, double* uy) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  const size_t N = (size_t)h->p.nx * h->p.ny;
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);
  CUDA_TRY(h, launch(h, MODE_FIELDS, h->buf[h->cur], nullptr, stage, h->stream));
  double* dst[5] = {rho1, rho2, T, ux, uy};
  for (int k = 0; k < 5; ++k)
    if (dst[k]) CUDA_TRY(h, cudaMemcpyAsync(dst[k], stage + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LB_OK;
}

int lb_get_state(lb_handle* h, double* host, size_t bytes) {
  if (!h || !host) return fail(h, LB_EINVAL, "handle and host buffer are required");
  const size_t N = (size_t)h->p.nx * h->p.ny;
  if (bytes != 27 * N * sizeof(double)) return fail(h, LB_EINVAL, "state needs %zu bytes", 27 * N * sizeof(double));
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);
  for (int k = 0; k < 27; ++k) {
    CUDA_TRY(h, plane_get(h, k, h->buf[h->cur], stage));
    CUDA_TRY(h, cudaMemcpyAsync(host + k * N, stage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LB_OK;
}

int lb_set_state(lb_handle* h, const double* host, size_t bytes) {
  if (!h || !host) return fail(h, LB_EINVAL, "handle and host buffer are required");
  const size_t N = (size_t)h->p.nx * h->p.ny;
  if (bytes != 27 * N * sizeof(double)) return fail(h, LB_EINVAL, "state needs %zu bytes", 27 * N * sizeof(double));
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);
  for (int k = 0; k < 27; ++k) {
    CUDA_TRY(h, cudaMemcpyAsync(stage, host + k * N, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, plane_put(h, k, stage, h->buf[h->cur]));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  h->step = 0;
  return LB_OK;
}

namespace {

// Reads n 16-byte words (an L2 eviction pass: afterwards L2 holds clean lines of this range); one
// word per block goes to sink so that the loads are kept.
__global__ void l2_read_kernel(const uint4* __restrict__ p, size_t n, unsigned* sink) {
  unsigned acc = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldcg(p + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;  // practically never taken; keeps the reads alive
}

// Times one trial of tile candidate h->tile: `launches` launches that read the current state and
// write the inactive buffer.  Without scratch they run back to back (caches warm); with scratch
// every launch is preceded by a write of the first half of the scratch and a read of the second
// half (each larger than L2), which evicts the state and leaves L2 holding clean lines, and only
// the launches themselves are timed.
cudaError_t time_candidate(lb_handle* h, int launches, void* scratch, size_t scratch_bytes, cudaEvent_t e0,
                           cudaEvent_t e1, float* ms_out) {
  cudaError_t e = launch(h, MODE_STEP, h->buf[h->cur], h->buf[h->cur ^ 1], nullptr, h->stream);
  float total = 0.0f;
  if (!scratch) {
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int r = 0; r < launches && e == cudaSuccess; ++r)
      e = launch(h, MODE_STEP, h->buf[h->cur], h->buf[h->cur ^ 1], nullptr, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&total, e0, e1);
  } else {
    const size_t half = scratch_bytes / 2 / 16 * 16;
    unsigned char* second = static_cast<unsigned char*>(scratch) + half;
    for (int r = 0; r < launches && e == cudaSuccess; ++r) {
      e = cudaMemsetAsync(scratch, r & 0xff, half, h->stream);
      if (e == cudaSuccess) {
        l2_read_kernel<<<1024, 256, 0, h->stream>>>(reinterpret_cast<const uint4*>(second), half / 16,
                                                     static_cast<unsigned*>(scratch));
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      if (e == cudaSuccess) e = launch(h, MODE_STEP, h->buf[h->cur], h->buf[h->cur ^ 1], nullptr, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
  }
  *ms_out = total / (float)launches;
  return e;
}

int autotune_impl(lb_handle* h, int launches, void* scratch, size_t scratch_bytes, int* chosen,
                  double* ms_per_candidate, int n_slots) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  if (launches < 1) return fail(h, LB_EINVAL, "launches must be >= 1");
  const int n = tile_count(h);
  if (ms_per_candidate && n_slots < n) return fail(h, LB_EINVAL, "ms_per_candidate needs %d slots", n);
  cudaEvent_t e0, e1;
  CUDA_TRY(h, cudaEventCreate(&e0));
  CUDA_TRY(h, cudaEventCreate(&e1));
  const int saved = h->tile;
  int best = saved;
  float best_ms = 0.0f;
  int rc = LB_OK;
  for (int k = 0; k < n && rc == LB_OK; ++k) {
    h->tile = k;
    float ms = 0.0f;
    const cudaError_t e = time_candidate(h, launches, scratch, scratch_bytes, e0, e1, &ms);
    if (e != cudaSuccess) {
      rc = fail(h, LB_ECUDA, "autotune candidate %d: %s", k, cudaGetErrorString(e));
      break;
    }
    if (ms_per_candidate) ms_per_candidate[k] = ms;
    if (k == 0 || ms < best_ms) {
      best_ms = ms;
      best = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LB_OK) {
    h->tile = saved;
    return rc;
  }
  if (best != saved) drop_graphs(h);
  h->tile = best;
  if (chosen) *chosen = best;
  return LB_OK;
}

}  // namespace

int lb_autotune(lb_handle* h, int launches, int* chosen, double* ms_per_candidate, int n_slots) {
  return autotune_impl(h, launches, nullptr, 0, chosen, ms_per_candidate, n_slots);
}

int lb_autotune_cold(lb_handle* h, int launches, void* d_scratch, size_t scratch_bytes, int* chosen,
                     double* ms_per_candidate, int n_slots) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  if (!d_scratch || scratch_bytes == 0) return fail(h, LB_EINVAL, "cold autotuning needs a scratch buffer");
  return autotune_impl(h, launches, d_scratch, scratch_bytes, chosen, ms_per_candidate, n_slots);
}

int lb_set_tile(lb_handle* h, int candidate) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  if (candidate < 0 || candidate >= tile_count(h)) return fail(h, LB_EINVAL, "tile candidate out of range");
  if (candidate != h->tile) drop_graphs(h);
  h->tile = candidate;
  return LB_OK;
}

int lb_tile_info(const lb_handle* h, int candidate, int* tx, int* ty, int* threads) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  if (candidate < 0) candidate = h->tile;
  if (candidate >= tile_count(h)) return LB_EINVAL;
  const TileChoice t = tile_info(h, candidate);
  if (tx) *tx = t.tx;
  if (ty) *ty = t.ty;
  if (threads) *threads = t.tx * t.by;
  return tile_count(h);
}

int lb_sync(lb_handle* h) {
  if (!h) return fail(nullptr, LB_EINVAL, "handle is NULL");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaGetLastError());
  return LB_OK;
}

void lb_destroy(lb_handle* h) {
  if (!h) return;
  if (h->stream || h->cap) {
    if (h->stream) cudaStreamSynchronize(h->stream);
  }
  drop_graphs(h);
  for (auto& d : h->dgraph)
    if (d.exec) cudaGraphExecDestroy(d.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
