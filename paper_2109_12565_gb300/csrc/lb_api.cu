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
#include "tlb.h"

using namespace tlb;

namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphLen = 16;  // steps per captured graph (even: replay keeps the buffer parity)

thread_local char g_err[512] = "no error";

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  int pitch = 0;
  size_t elem = 0, buf_bytes = 0, mask_off = 0, part_off = 0, obs_off = 0, total = 0;
  int n_blocks = 0;
};

int tile_x(int precision) { return precision == LB_FP64 ? Tile<double>::TX : Tile<float>::TX; }
int tile_y(int precision) { return precision == LB_FP64 ? Tile<double>::TY : Tile<float>::TY; }

const char* check_params(const lb_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1) return "nx and ny must be >= 1";
  if ((long long)p->nx * p->ny > (1LL << 31) - 1) return "nx * ny must fit in 31 bits";
  if (!p->periodic_y && p->ny < 3) return "walls (periodic_y = 0) need ny >= 3";
  if (p->precision != LB_FP64 && p->precision != LB_FP32_SHIFTED) return "precision must be LB_FP64 or LB_FP32_SHIFTED";
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return "tau must be finite and > 1/2";
  if (!(p->tau_g > 0.5) || !std::isfinite(p->tau_g)) return "tau_g must be finite and > 1/2";
  if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return "rho0 must be finite and > 0";
  const double vals[] = {p->G12, p->Ga[0], p->Ga[1], p->Gr[0], p->Gr[1], p->T_down, p->T_up, p->alpha_g, p->body_fx};
  for (double v : vals)
    if (!std::isfinite(v)) return "coupling, temperature and force parameters must be finite";
  if (!(p->rho_wall[0] > 0.0) || !(p->rho_wall[1] > 0.0) || !std::isfinite(p->rho_wall[0]) ||
      !std::isfinite(p->rho_wall[1]))
    return "rho_wall must be finite and > 0";
  return nullptr;
}

Layout layout_for(const lb_params* p, int has_mask) {
  Layout L;
  L.elem = p->precision == LB_FP64 ? 8 : 4;
  const int per_row = (int)(128 / L.elem);
  L.pitch = (p->nx + per_row - 1) / per_row * per_row;
  const size_t plane = (size_t)L.pitch * p->ny;
  L.buf_bytes = round_up(27 * plane * L.elem, kAlign);
  // the inactive buffer doubles as staging for init (3 planes) and fields (5 planes) of doubles
  const size_t staging = (size_t)p->nx * p->ny * 5 * sizeof(double);
  if (staging > L.buf_bytes) L.buf_bytes = round_up(staging, kAlign);
  size_t off = 2 * L.buf_bytes;
  L.mask_off = off;
  if (has_mask) off += round_up((size_t)p->nx * p->ny, kAlign);
  const int tx = tile_x(p->precision), ty = tile_y(p->precision);
  L.n_blocks = ((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty);
  L.part_off = off;
  off += round_up((size_t)L.n_blocks * kObsSlots * sizeof(double), kAlign);
  L.obs_off = off;
  off += round_up(kObsOut * sizeof(double), kAlign);
  L.total = off;
  return L;
}

double psi_exp_host(double rho, double rho0) { return rho0 * (1.0 - std::exp(-rho / rho0)); }

}  // namespace

struct lb_handle {
  lb_params p{};
  Layout L{};
  StepCfg cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  unsigned char* ws = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  long long step = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  char err[512] = "no error";
};

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
  return h->p.precision == LB_FP64 ? launch_f64(mode, h->cfg, fin, fout, aux, s)
                                   : launch_f32(mode, h->cfg, fin, fout, aux, s);
}

void fill_cfg(lb_handle* h, const uint8_t* d_mask) {
  const lb_params& p = h->p;
  StepCfg& c = h->cfg;
  c.nx = p.nx;
  c.ny = p.ny;
  c.pitch = h->L.pitch;
  c.periodic_y = p.periodic_y ? 1 : 0;
  c.plane = (long long)h->L.pitch * p.ny;
  c.mask = d_mask;
  c.tau = p.tau;
  c.inv_tau = 1.0 / p.tau;
  c.inv_tau_g = 1.0 / p.tau_g;
  c.rho0 = p.rho0;
  c.inv_rho0 = 1.0 / p.rho0;
  c.gx = p.G12 / (p.rho0 * p.rho0);
  for (int l = 0; l < 2; ++l) {
    // Fig. 1b weights per shell |c|^2 = 1, 2, 4, 5, 8: w = 1/9, 1/36, 0, 0, 0; p = 4/63, 4/135, 1/180, 2/945, 1/15120
    c.a1[l] = p.Ga[l] / 9.0 + p.Gr[l] * 4.0 / 63.0;
    c.a2[l] = p.Ga[l] / 36.0 + p.Gr[l] * 4.0 / 135.0;
    c.a4x2[l] = 2.0 * p.Gr[l] / 180.0;
    c.a5[l] = p.Gr[l] * 2.0 / 945.0;
    c.a8x2[l] = 2.0 * p.Gr[l] / 15120.0;
    c.rho_w[l] = p.rho_wall[l];
    c.psi_w[l] = psi_exp_host(p.rho_wall[l], p.rho0);
  }
  c.T_down = p.T_down;
  c.T_up = p.T_up;
  c.alpha_g = p.alpha_g;
  c.body_fx = p.body_fx;
  c.rho_bar[0] = c.rho_bar[1] = c.T_bar = 0.0;
  if (p.precision == LB_FP32_SHIFTED) {
    c.rho_bar[0] = p.shift_rho[0];
    c.rho_bar[1] = p.shift_rho[1];
    c.T_bar = p.shift_T;
  }
  c.kappa = (p.tau_g - 0.5) / 3.0;
  c.H = (double)(p.ny - 2);
}

bool is_solid_host(const lb_params& p, const uint8_t* mask, int x, int y) {
  if (!p.periodic_y && (y == 0 || y == p.ny - 1)) return true;
  return mask && mask[(size_t)y * p.nx + x];
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
  double sum1 = 0.0, sum2 = 0.0;
  size_t nf = 0;
  for (int y = 0; y < p.ny; ++y)
    for (int x = 0; x < p.nx; ++x) {
      if (is_solid_host(p, mask, x, y)) continue;
      const size_t n = (size_t)y * p.nx + x;
      if (!(rho1[n] > 0.0) || !(rho2[n] > 0.0) || !std::isfinite(rho1[n]) || !std::isfinite(rho2[n]) ||
          !std::isfinite(T0[n]))
        return fail(nullptr, LB_EINVAL, "initial densities must be finite and > 0 and T0 finite (node %d,%d)", x, y);
      sum1 += rho1[n];
      sum2 += rho2[n];
      ++nf;
    }
  if (nf == 0) return fail(nullptr, LB_EINVAL, "the lattice has no fluid node");
  if (p.precision == LB_FP32_SHIFTED) {
    if (std::isnan(p.shift_rho[0])) p.shift_rho[0] = sum1 / (double)nf;
    if (std::isnan(p.shift_rho[1])) p.shift_rho[1] = sum2 / (double)nf;
    if (std::isnan(p.shift_T)) p.shift_T = 0.5 * (p.T_down + p.T_up);
    if (!std::isfinite(p.shift_rho[0]) || !std::isfinite(p.shift_rho[1]) || !std::isfinite(p.shift_T))
      return fail(nullptr, LB_EINVAL, "shift constants must be finite (or NaN for the defaults)");
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
  if (e != cudaSuccess) return bail(fail(h, LB_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
  e = cudaMemsetAsync(h->ws, 0, 2 * L.buf_bytes, h->stream);
  if (e == cudaSuccess && mask) e = cudaMemcpyAsync(d_mask, mask, N, cudaMemcpyHostToDevice, h->stream);
  double* stage = static_cast<double*>(h->buf[1]);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, rho1, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + N, rho2, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 2 * N, T0, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = p.precision == LB_FP64 ? init_f64(h->cfg, stage, h->buf[0], h->stream)
                                                   : init_f32(h->cfg, stage, h->buf[0], h->stream);
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
    CUDA_TRY(h, h->p.precision == LB_FP64 ? plane_get_f64(h->cfg, k, h->buf[h->cur], stage, h->stream)
                                          : plane_get_f32(h->cfg, k, h->buf[h->cur], stage, h->stream));
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
    CUDA_TRY(h, h->p.precision == LB_FP64 ? plane_put_f64(h->cfg, k, stage, h->buf[h->cur], h->stream)
                                          : plane_put_f32(h->cfg, k, stage, h->buf[h->cur], h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  h->step = 0;
  return LB_OK;
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
  for (auto& g : h->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
