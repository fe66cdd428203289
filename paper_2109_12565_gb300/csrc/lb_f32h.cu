// FP32 fluid + FP16 thermal storage form of the fused step: the 18 fluid
// planes stored as FP32 deviations f - w_i rho_bar_l, the 9 thermal planes as
// FP16 deviations g - w_i T_bar (round to nearest on every store), FP32
// arithmetic; the shift constants stay FP64 on the host and in the reductions.
// 180 bytes of population traffic per lattice update instead of 216.
#include "lb_kernels.cuh"

namespace tlb {

cudaError_t launch_f32h(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  return launch_impl<F32H16, true>(mode, c, fin, fout, aux, s);
}

namespace {
using StepFn = cudaError_t (*)(const StepCfg&, const void*, void*, cudaStream_t);
struct Cand {
  TileChoice t;
  StepFn fn;
};
const Cand kCands[] = {
    {{64, 16, 4, 3}, launch_step_shape<F32H16, true, 64, 16, 4, 3>},
    {{64, 8, 4, 4}, launch_step_shape<F32H16, true, 64, 8, 4, 4>},
    {{64, 32, 8, 2}, launch_step_shape<F32H16, true, 64, 32, 8, 2>},
    {{32, 16, 8, 3}, launch_step_shape<F32H16, true, 32, 16, 8, 3>},
    {{32, 8, 8, 4}, launch_step_shape<F32H16, true, 32, 8, 8, 4>},
    // 32 x 9: 1824 tiles at 1024 x 512, exactly three waves of 4 CTAs (56 registers) on 152 SMs
    {{32, 9, 9, 4}, launch_step_shape<F32H16, true, 32, 9, 9, 4>},
};
}  // namespace

int tile_count_f32h() { return (int)(sizeof kCands / sizeof kCands[0]); }
TileChoice tile_info_f32h(int k) { return kCands[k].t; }
cudaError_t launch_step_tile_f32h(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kCands[k].fn(c, fin, fout, s);
}

cudaError_t init_f32h(const StepCfg& c, const double* fields, void* buf, cudaStream_t s) {
  lb_init_kernel<F32H16, true><<<rows_grid(c), 128, 0, s>>>(fields, static_cast<float*>(buf), c);
  return cudaGetLastError();
}

cudaError_t plane_get_f32h(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s) {
  lb_plane_get_kernel<F32H16, true><<<rows_grid(c), 128, 0, s>>>(k, static_cast<const float*>(buf), out, c);
  return cudaGetLastError();
}

cudaError_t plane_put_f32h(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s) {
  lb_plane_put_kernel<F32H16, true><<<rows_grid(c), 128, 0, s>>>(k, in, static_cast<float*>(buf), c);
  return cudaGetLastError();
}

}  // namespace tlb
