// FP64 instantiation of the fused step (populations and arithmetic in FP64)
// and the deterministic final reduction of the observables.
#include "lb_kernels.cuh"
#include "tlb.h"

namespace tlb {

cudaError_t launch_f64(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  return launch_impl<double, false>(mode, c, fin, fout, aux, s);
}

namespace {
using StepFn = cudaError_t (*)(const StepCfg&, const void*, void*, cudaStream_t);
struct Cand {
  TileChoice t;
  StepFn fn;
};
const Cand kCands[] = {
    {{32, 16, 8, 2}, launch_step_shape<double, false, 32, 16, 8, 2>},
    {{64, 16, 4, 2}, launch_step_shape<double, false, 64, 16, 4, 2>},
    {{32, 32, 8, 2}, launch_step_shape<double, false, 32, 32, 8, 2>},
};
}  // namespace

int tile_count_f64() { return (int)(sizeof kCands / sizeof kCands[0]); }
TileChoice tile_info_f64(int k) { return kCands[k].t; }
cudaError_t launch_step_tile_f64(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kCands[k].fn(c, fin, fout, s);
}

// The adjoint's forward step with the u^(H)_y T partial sums: the shape of tile candidate 0.
cudaError_t launch_step_nu_f64(const StepCfg& c, const void* fin, void* fout, double* partials, cudaStream_t s) {
  return launch_tile_kernel<double, MODE_STEP_NU, 32, 16, 8, 2, false>(grid_for(c.nx, c.ny, 32, 16),
                                                                      static_cast<const double*>(fin),
                                                                      static_cast<double*>(fout), make_kparams<double>(c),
                                                                      partials, s);
}

int step_nu_blocks(int precision, int nx, int ny) {  // partials: CTAs x 8 warps (256 threads)
  const dim3 g = precision == LB_FP64 ? grid_for(nx, ny, 32, 16) : grid_for(nx, ny, 32, 8);
  return (int)(g.x * g.y) * 8;
}

cudaError_t init_f64(const StepCfg& c, const double* fields, void* buf, cudaStream_t s) {
  lb_init_kernel<double, false><<<rows_grid(c), 128, 0, s>>>(fields, static_cast<double*>(buf), c);
  return cudaGetLastError();
}

cudaError_t plane_get_f64(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s) {
  lb_plane_get_kernel<double, false><<<rows_grid(c), 128, 0, s>>>(k, static_cast<const double*>(buf), out, c);
  return cudaGetLastError();
}

cudaError_t plane_put_f64(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s) {
  lb_plane_put_kernel<double, false><<<rows_grid(c), 128, 0, s>>>(k, in, static_cast<double*>(buf), c);
  return cudaGetLastError();
}

// One CTA sums the per-block partials in a fixed order (thread t takes blocks t, t+256, ...;
// then a fixed shuffle tree and warp order), so the result does not depend on scheduling.
// out: [0..1] mass, [2..3] momentum, [4] Nu, [5] E, [6] n_bad, [7] n_fluid, [8] <u_y T> sum,
//      [9] dT/dy sum.
__global__ void __launch_bounds__(256) lb_obs_finalize_kernel(const double* __restrict__ part, int n_blocks,
                                                              double* __restrict__ out, const StepCfg cfg) {
  __shared__ double s_red[8][kObsSlots];
  double acc[kObsSlots];
#pragma unroll
  for (int v = 0; v < kObsSlots; ++v) acc[v] = 0.0;
  for (int b = threadIdx.x; b < n_blocks; b += 256) {
#pragma unroll
    for (int v = 0; v < kObsSlots; ++v) acc[v] += part[(long long)b * kObsSlots + v];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < kObsSlots; ++v) {
    const double s = warp_sum(acc[v]);
    if (lane == 0) s_red[warp][v] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[kObsSlots];
    for (int v = 0; v < kObsSlots; ++v) {
      t[v] = 0.0;
      for (int w = 0; w < 8; ++w) t[v] += s_red[w][v];
    }
    const double nf = t[8];
    out[0] = t[0] + nf * cfg.rho_bar[0];
    out[1] = t[1] + nf * cfg.rho_bar[1];
    out[2] = t[2];
    out[3] = t[3];
    const double dT = cfg.T_down - cfg.T_up;
    double Nu = 0.0;
    if (!cfg.periodic_y && dT != 0.0 && nf > 0.0)
      Nu = (t[4] / nf - cfg.kappa * t[5] / nf) / (cfg.kappa * dT / cfg.H);  // Eq. NuTime
    out[4] = Nu;
    out[5] = nf > 0.0 ? t[6] / nf : 0.0;
    out[6] = t[7];
    out[7] = nf;
    out[8] = t[4];
    out[9] = t[5];
    out[10] = t[9];   // x momentum to the bottom wall per step
    out[11] = t[10];  // x momentum to the top wall per step
  }
}

cudaError_t obs_finalize(const StepCfg& c, const double* partials, int n_blocks, double* out, cudaStream_t s) {
  lb_obs_finalize_kernel<<<1, 256, 0, s>>>(partials, n_blocks, out, c);
  return cudaGetLastError();
}

}  // namespace tlb
