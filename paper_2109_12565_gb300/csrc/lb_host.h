// Host-side helpers shared by the single-lattice and batched C-ABI front ends:
// parameter checks, the per-lattice workspace layout and the FP64 step
// constants derived from lb_params.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdio>

#include "lb_cfg.h"
#include "tlb.h"

namespace tlb {

constexpr size_t kAlign = 256;

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace of one lattice: buffers A and B (27 planes each), optional mask, observable partials,
// final observable vector.  Offsets are relative to the lattice's base address.
struct Layout {
  int pitch = 0;
  size_t elem = 0, buf_bytes = 0, mask_off = 0, part_off = 0, obs_off = 0, total = 0;
  int n_blocks = 0;
};

// 8-byte population storage (FP64, or double-float pairs) versus the FP32 forms.
inline bool wide_storage(int precision) { return precision == LB_FP64 || precision == LB_DF64; }
// Forms that store deviations from the shift equilibria.
inline bool shifted_storage(int precision) { return precision == LB_FP32_SHIFTED || precision == LB_FP32_FP16T; }
inline int obs_tile_x(int precision) { return wide_storage(precision) ? Tile<double>::TX : Tile<float>::TX; }
inline int obs_tile_y(int precision) { return wide_storage(precision) ? Tile<double>::TY : Tile<float>::TY; }

inline const char* check_params(const lb_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1) return "nx and ny must be >= 1";
  if ((long long)p->nx * p->ny > (1LL << 31) - 1) return "nx * ny must fit in 31 bits";
  // the row-wise kernels (init, field read-back, rho_1) launch one block row per lattice row
  if (p->ny > 65535) return "ny must be <= 65535";
  if (!p->periodic_y && p->ny < 3) return "walls (periodic_y = 0) need ny >= 3";
  if (p->precision != LB_FP64 && p->precision != LB_FP32_SHIFTED && p->precision != LB_FP32_FP16T &&
      p->precision != LB_DF64)
    return "precision must be LB_FP64, LB_FP32_SHIFTED, LB_FP32_FP16T or LB_DF64";
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return "tau must be finite and > 1/2";
  if (!(p->tau_g > 0.5) || !std::isfinite(p->tau_g)) return "tau_g must be finite and > 1/2";
  if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return "rho0 must be finite and > 0";
  const double vals[] = {p->G12,    p->Ga[0],  p->Ga[1],   p->Gr[0],      p->Gr[1],      p->T_down,
                         p->T_up,   p->alpha_g, p->body_fx, p->u_wall[0], p->u_wall[1]};
  for (double v : vals)
    if (!std::isfinite(v)) return "coupling, temperature and force parameters must be finite";
  if (!(p->rho_wall[0] > 0.0) || !(p->rho_wall[1] > 0.0) || !std::isfinite(p->rho_wall[0]) ||
      !std::isfinite(p->rho_wall[1]))
    return "rho_wall must be finite and > 0";
  const int per_row = wide_storage(p->precision) ? 16 : 32;
  const double pitch = (double)((p->nx + per_row - 1) / per_row * per_row);
  if (27.0 * pitch * (double)p->ny >= 2147483648.0) return "lattice too large: 27 * pitch * ny must stay below 2^31";
  return nullptr;
}

inline Layout layout_for(const lb_params* p, int has_mask) {
  Layout L;
  L.elem = wide_storage(p->precision) ? 8 : 4;
  const int per_row = (int)(128 / L.elem);
  L.pitch = (p->nx + per_row - 1) / per_row * per_row;
  const size_t plane = (size_t)L.pitch * p->ny;
  // LB_FP32_FP16T: 18 FP32 fluid planes, then 9 FP16 thermal planes of the same pitch
  L.buf_bytes = round_up(p->precision == LB_FP32_FP16T ? (18 * 4 + 9 * 2) * plane : 27 * plane * L.elem, kAlign);
  // the inactive buffer doubles as staging for init (3 planes), fields (5 planes) and the stress pass
  const size_t staging = stress_staging_doubles(p->nx, p->ny) * sizeof(double);
  if (staging > L.buf_bytes) L.buf_bytes = round_up(staging, kAlign);
  size_t off = 2 * L.buf_bytes;
  L.mask_off = off;
  if (has_mask) off += round_up((size_t)p->nx * p->ny, kAlign);
  const int tx = obs_tile_x(p->precision), ty = obs_tile_y(p->precision);
  L.n_blocks = ((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty);
  L.part_off = off;
  off += round_up((size_t)L.n_blocks * kObsSlots * sizeof(double), kAlign);
  L.obs_off = off;
  off += round_up(kObsOut * sizeof(double), kAlign);
  L.total = off;
  return L;
}

inline double psi_exp_host(double rho, double rho0) { return rho0 * (1.0 - std::exp(-rho / rho0)); }

// FP64 step constants of one lattice (storage pitch in elements, device mask or nullptr).  The shift
// constants are used only in the FP32 storage forms.
inline StepCfg make_stepcfg(const lb_params& p, int pitch, const uint8_t* d_mask) {
  StepCfg c{};
  c.nx = p.nx;
  c.ny = p.ny;
  c.pitch = pitch;
  c.periodic_y = p.periodic_y ? 1 : 0;
  c.plane = (long long)pitch * p.ny;
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
  if (shifted_storage(p.precision)) {
    c.rho_bar[0] = p.shift_rho[0];
    c.rho_bar[1] = p.shift_rho[1];
    c.T_bar = p.shift_T;
  }
  c.kappa = (p.tau_g - 0.5) / 3.0;
  c.H = (double)(p.ny - 2);
  c.u_wall[0] = p.periodic_y ? 0.0 : p.u_wall[0];
  c.u_wall[1] = p.periodic_y ? 0.0 : p.u_wall[1];
  return c;
}

inline bool is_solid_host(const lb_params& p, const uint8_t* mask, int x, int y) {
  if (!p.periodic_y && (y == 0 || y == p.ny - 1)) return true;
  return mask && mask[(size_t)y * p.nx + x];
}

// Validate the initial host fields of one lattice and fill the default FP32 shifts (NaN -> mean
// fluid density, (T_down + T_up) / 2).  Returns nullptr or the reason.
inline const char* prepare_fields(lb_params& p, const uint8_t* mask, const double* rho1, const double* rho2,
                                  const double* T0, char* why, size_t why_len) {
  double sum1 = 0.0, sum2 = 0.0;
  size_t nf = 0;
  for (int y = 0; y < p.ny; ++y)
    for (int x = 0; x < p.nx; ++x) {
      if (is_solid_host(p, mask, x, y)) continue;
      const size_t n = (size_t)y * p.nx + x;
      if (!(rho1[n] > 0.0) || !(rho2[n] > 0.0) || !std::isfinite(rho1[n]) || !std::isfinite(rho2[n]) ||
          !std::isfinite(T0[n])) {
        std::snprintf(why, why_len, "initial densities must be finite and > 0 and T0 finite (node %d,%d)", x, y);
        return why;
      }
      sum1 += rho1[n];
      sum2 += rho2[n];
      ++nf;
    }
  if (nf == 0) return "the lattice has no fluid node";
  if (shifted_storage(p.precision)) {
    if (std::isnan(p.shift_rho[0])) p.shift_rho[0] = sum1 / (double)nf;
    if (std::isnan(p.shift_rho[1])) p.shift_rho[1] = sum2 / (double)nf;
    if (std::isnan(p.shift_T)) p.shift_T = 0.5 * (p.T_down + p.T_up);
    if (!std::isfinite(p.shift_rho[0]) || !std::isfinite(p.shift_rho[1]) || !std::isfinite(p.shift_T))
      return "shift constants must be finite (or NaN for the defaults)";
  }
  return nullptr;
}

}  // namespace tlb

// Handle of one lattice (opaque to C callers; shared by the single-lattice and adjoint front ends).
struct lb_handle {
  lb_params p{};
  tlb::Layout L{};
  tlb::StepCfg cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  unsigned char* ws = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  long long step = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // captured droplet analyses (lb_droplets), keyed by what their launches bake in
  struct DropGraph {
    cudaGraphExec_t exec = nullptr;
    const void* ws = nullptr;
    int max_drops = 0, cur = -1;
    double threshold = 0.0;
  } dgraph[4];
  int dgraph_next = 0;
  int tile = 0;  // step-kernel tile candidate (see lb_autotune)
  char err[512] = "no error";
};
