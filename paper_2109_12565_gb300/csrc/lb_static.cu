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
// exits; with CUDA's lazy module loading the array comes into being on the
// first call on a device, so a caller should make one warm-up call at
// initialisation, before any stream capture.  Host code cannot use the
// array's name as a device address, so every call looks the address up
// with cudaGetSymbolAddress (with the call's device current) and passes it
// to the kernels; nothing is cached, so a device reset between calls does
// no harm.
// All calls on a device share the array and it keeps the last call's
// contents: every slot a call reads is first written by that same call
// (each block writes its own partial slot, the final kernel writes the
// output slots), so nothing needs clearing, but calls that overlap on the
// GPU (different streams, or different host threads) race on the array and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>

#include "lb_cfg.h"
#include "lb_host.h"
#include "tlb.h"

using namespace tlb;

namespace {

constexpr int kStaticScratchDoubles = 262144;  // 2 MiB: kObsOut output slots + per-block partials

__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// Device address of the scratch array on the current device, looked up on every call: a device
// reset, or a context torn down and created again, may move the array, so no address is kept.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) return LB_ECUDA;
  *out = static_cast<double*>(p);
  return LB_OK;
}

}  // namespace

// Errors are reported by return code only: LB_EINVAL for arguments (checked before any launch),
// LB_ECUDA for a failed CUDA call; lb_last_error is not updated.
extern "C" int lb_observables_static(const lb_params* p, const double* d_state, const uint8_t* d_mask, lb_obs* out,
                                     void* stream) {
  if (!p || !d_state || !out) return LB_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_state) % alignof(double)) != 0) return LB_EINVAL;
  // the same checks and constants as a handle in FP64 storage, read from an unpadded layout (pitch = nx)
  lb_params q = *p;
  q.precision = LB_FP64;
  if (check_params(&q) != nullptr) return LB_EINVAL;
  if (d_mask && q.periodic_y) return LB_EINVAL;
  const dim3 grid = grid_for(q.nx, q.ny, Tile<double>::TX, Tile<double>::TY);
  const long long n_blocks = (long long)grid.x * grid.y;
  if (kObsOut + n_blocks * kObsSlots > kStaticScratchDoubles) return LB_EINVAL;
  const StepCfg c = make_stepcfg(q, q.nx, d_mask);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;

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
