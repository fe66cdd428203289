// FP32-shifted instantiation of the fused step: populations stored as FP32
// deviations from the rest equilibria of the shift densities (f - w_i rho_bar_l,
// g - w_i T_bar), FP32 arithmetic; the shift constants stay FP64 on the host
// and in the reductions.
#include "lb_kernels.cuh"

namespace tlb {

cudaError_t launch_f32(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  return launch_impl<float, true>(mode, c, fin, fout, aux, s);
}

namespace {
using StepFn = cudaError_t (*)(const StepCfg&, const void*, void*, cudaStream_t);
struct Cand {
  TileChoice t;
  StepFn fn;
};
const Cand kCands[] = {
    {{64, 16, 4, 3}, launch_step_shape<float, true, 64, 16, 4, 3>},
    {{32, 16, 8, 3}, launch_step_shape<float, true, 32, 16, 8, 3>},
    {{64, 32, 8, 2}, launch_step_shape<float, true, 64, 32, 8, 2>},
    {{128, 16, 2, 3}, launch_step_shape<float, true, 128, 16, 2, 3>},
    {{64, 8, 4, 4}, launch_step_shape<float, true, 64, 8, 4, 4>},
    {{32, 32, 8, 3}, launch_step_shape<float, true, 32, 32, 8, 3>},
    {{64, 16, 4, 4}, launch_step_shape<float, true, 64, 16, 4, 4>},
    {{32, 16, 8, 4}, launch_step_shape<float, true, 32, 16, 8, 4>},
    {{64, 32, 4, 4}, launch_step_shape<float, true, 64, 32, 4, 4>},
    {{32, 32, 8, 4}, launch_step_shape<float, true, 32, 32, 8, 4>},
    // one phase-A pass of node pairs and one phase-B node per thread
    {{32, 8, 8, 4}, launch_step_shape<float, true, 32, 8, 8, 4>},
};
}  // namespace

int tile_count_f32() { return (int)(sizeof kCands / sizeof kCands[0]); }
TileChoice tile_info_f32(int k) { return kCands[k].t; }
cudaError_t launch_step_tile_f32(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kCands[k].fn(c, fin, fout, s);
}

// The adjoint's forward step with the u^(H)_y T partial sums: the 32 x 8 tile (one phase-A pass of node
// pairs, one phase-B node per thread).
cudaError_t launch_step_nu_f32(const StepCfg& c, const void* fin, void* fout, double* partials, cudaStream_t s) {
  return launch_tile_kernel<float, MODE_STEP_NU, 32, 8, 8, 4, true>(grid_for(c.nx, c.ny, 32, 8),
                                                                   static_cast<const float*>(fin),
                                                                   static_cast<float*>(fout), make_kparams<float>(c),
                                                                   partials, s);
}

cudaError_t init_f32(const StepCfg& c, const double* fields, void* buf, cudaStream_t s) {
  lb_init_kernel<float, true><<<rows_grid(c), 128, 0, s>>>(fields, static_cast<float*>(buf), c);
  return cudaGetLastError();
}

cudaError_t plane_get_f32(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s) {
  lb_plane_get_kernel<float, true><<<rows_grid(c), 128, 0, s>>>(k, static_cast<const float*>(buf), out, c);
  return cudaGetLastError();
}

cudaError_t plane_put_f32(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s) {
  lb_plane_put_kernel<float, true><<<rows_grid(c), 128, 0, s>>>(k, in, static_cast<float*>(buf), c);
  return cudaGetLastError();
}

}  // namespace tlb
