// lb_observables_static: the observables reduction for callers that cannot
// allocate device memory.
//
// Who needs it: code that may not call cudaMalloc or any allocating routine
// - a plug-in running inside a host application that owns every device
// allocation, a real-time loop where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable, or code running between other
// users' CUDA-graph captures.  Such a caller still holds the populations in
// its own device memory and wants the mass, momentum, Nusselt number and
// kinetic energy of that state, with no workspace to hand over.
//
// How: the per-block partial sums and the final vector live in one
// file-scope __device__ array of kStaticScratchDoubles doubles (2 MiB).
// Every GPU that loads this library holds that array until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; that first call should happen
// before any stream capture.  All calls on a device share the array and it
// keeps the last call's contents: every slot a call reads is first written
// by that same call (each block writes its own partial slot, the final
// kernel writes the output slots), so nothing needs clearing, but calls
// that overlap on the GPU (different streams, or different host threads)
// race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "lb_cfg.h"
#include "tlb.h"

using namespace tlb;

namespace {

constexpr int kStaticScratchDoubles = 262144;  // 2 MiB: kObsOut output slots + per-block partials
constexpr int kMaxDevices = 128;

__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};
// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return LB_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LB_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) return LB_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return LB_OK;
}

bool finite_all(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace

// Errors are reported by return code only: LB_EINVAL for arguments (checked before any launch),
// LB_ECUDA for a failed CUDA call; lb_last_error is not updated.
extern "C" int lb_observables_static(const lb_params* p, const double* d_state, const uint8_t* d_mask, lb_obs* out,
                                     void* stream) {
  if (!p || !d_state || !out) return LB_EINVAL;
  if (p->nx < 1 || p->ny < 1 || (!p->periodic_y && p->ny < 3)) return LB_EINVAL;
  if ((long long)p->nx * p->ny > (1LL << 31) - 1) return LB_EINVAL;
  if (d_mask && p->periodic_y) return LB_EINVAL;
  if (!(p->tau > 0.5) || !(p->tau_g > 0.5) || !(p->rho0 > 0.0) || !(p->rho_wall[0] > 0.0) || !(p->rho_wall[1] > 0.0) ||
      !finite_all({p->tau, p->tau_g, p->rho0, p->G12, p->Ga[0], p->Ga[1], p->Gr[0], p->Gr[1], p->rho_wall[0],
                   p->rho_wall[1], p->T_down, p->T_up, p->alpha_g, p->body_fx, p->u_wall[0], p->u_wall[1]}))
    return LB_EINVAL;
  const dim3 grid = grid_for(p->nx, p->ny, Tile<double>::TX, Tile<double>::TY);
  const long long n_blocks = (long long)grid.x * grid.y;
  if (kObsOut + n_blocks * kObsSlots > kStaticScratchDoubles)
    return LB_EINVAL;

  double* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;

  // Same constants as a handle in FP64 storage, read from an unpadded layout (pitch = nx).
  StepCfg c{};
  c.nx = p->nx;
  c.ny = p->ny;
  c.pitch = p->nx;
  c.periodic_y = p->periodic_y ? 1 : 0;
  c.plane = (long long)p->nx * p->ny;
  c.mask = d_mask;
  c.tau = p->tau;
  c.inv_tau = 1.0 / p->tau;
  c.inv_tau_g = 1.0 / p->tau_g;
  c.rho0 = p->rho0;
  c.inv_rho0 = 1.0 / p->rho0;
  c.gx = p->G12 / (p->rho0 * p->rho0);
  for (int l = 0; l < 2; ++l) {
    c.a1[l] = p->Ga[l] / 9.0 + p->Gr[l] * 4.0 / 63.0;
    c.a2[l] = p->Ga[l] / 36.0 + p->Gr[l] * 4.0 / 135.0;
    c.a4x2[l] = 2.0 * p->Gr[l] / 180.0;
    c.a5[l] = p->Gr[l] * 2.0 / 945.0;
    c.a8x2[l] = 2.0 * p->Gr[l] / 15120.0;
    c.rho_w[l] = p->rho_wall[l];
    c.psi_w[l] = p->rho0 * (1.0 - std::exp(-p->rho_wall[l] / p->rho0));
  }
  c.T_down = p->T_down;
  c.T_up = p->T_up;
  c.alpha_g = p->alpha_g;
  c.body_fx = p->body_fx;
  c.kappa = (p->tau_g - 0.5) / 3.0;
  c.H = (double)(p->ny - 2);
  c.u_wall[0] = p->periodic_y ? 0.0 : p->u_wall[0];
  c.u_wall[1] = p->periodic_y ? 0.0 : p->u_wall[1];

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* final_out = scratch;            // kObsOut slots
  double* partials = scratch + kObsOut;   // n_blocks * kObsSlots slots, each written by its block
  cudaError_t e = launch_f64(MODE_OBS, c, d_state, nullptr, partials, s);
  if (e == cudaSuccess) e = obs_finalize(c, partials, (int)n_blocks, final_out, s);
  double v[kObsOut];
  if (e == cudaSuccess) e = cudaMemcpyAsync(v, final_out, sizeof v, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LB_ECUDA;
  out->mass[0] = v[0];
  out->mass[1] = v[1];
  out->mom[0] = v[2];
  out->mom[1] = v[3];
  out->Nu = v[4];
  out->E = v[5];
  out->n_bad = (long long)v[6];
  out->n_fluid = (long long)v[7];
  out->step = 0;
  out->status = out->n_bad > 0 ? LB_EUNSTABLE : LB_OK;
  out->_pad = 0;
  out->wall_fx[0] = v[10];
  out->wall_fx[1] = v[11];
  return out->status;
}
