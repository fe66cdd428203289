// LB_DF64 instantiation of the fused step: populations stored as double-float (hi, lo) FP32 pairs
// (8 bytes, the footprint of FP64), every operation in double-float arithmetic on the FP32 pipe
// (lb_df.cuh); results stay within the FP64 form's tolerance against the FP64 oracle.
#include <cmath>

#include "lb_df.cuh"

namespace tlb {

namespace {
float2 split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
}  // namespace

// exp(-k / 64) and exp(-j / 4096) as double-float roundings of the FP64 library values, written to the
// current device by every lb_init of an LB_DF64 lattice (2.6 KB, before any stream capture); nothing is
// remembered between calls, so a device reset in between does no harm.
cudaError_t df_exp_tables_init() {
  float2 t1[kDfExpT1], t2[kDfExpT2];
  for (int k = 0; k < kDfExpT1; ++k) t1[k] = split(std::exp(-(double)k / 64.0));
  for (int j = 0; j < kDfExpT2; ++j) t2[j] = split(std::exp(-(double)j / 4096.0));
  cudaError_t e = cudaMemcpyToSymbol(g_df_exp_t1, t1, sizeof t1);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_df_exp_t2, t2, sizeof t2);
  return e;
}

cudaError_t launch_df64(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  return launch_impl<DF, false>(mode, c, fin, fout, aux, s);
}

namespace {
using StepFn = cudaError_t (*)(const StepCfg&, const void*, void*, cudaStream_t);
struct Cand {
  TileChoice t;
  StepFn fn;
};
const Cand kCands[] = {
    {{32, 16, 8, 2}, launch_step_shape<DF, false, 32, 16, 8, 2>},
    {{64, 16, 4, 2}, launch_step_shape<DF, false, 64, 16, 4, 2>},
    {{32, 32, 8, 2}, launch_step_shape<DF, false, 32, 32, 8, 2>},
    {{32, 8, 8, 2}, launch_step_shape<DF, false, 32, 8, 8, 2>},
    // three CTAs per SM: the register bound (85) spills about 230 bytes per thread to L1, and the extra
    // resident warps still win (0.081 against 0.086 ms per step at 1024 x 512)
    {{32, 16, 8, 3}, launch_step_shape<DF, false, 32, 16, 8, 3>},
    {{32, 8, 8, 3}, launch_step_shape<DF, false, 32, 8, 8, 3>},
};
}  // namespace

int tile_count_df64() { return (int)(sizeof kCands / sizeof kCands[0]); }
TileChoice tile_info_df64(int k) { return kCands[k].t; }
cudaError_t launch_step_tile_df64(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kCands[k].fn(c, fin, fout, s);
}

cudaError_t init_df64(const StepCfg& c, const double* fields, void* buf, cudaStream_t s) {
  lb_init_kernel<DF, false><<<rows_grid(c), 128, 0, s>>>(fields, static_cast<float2*>(buf), c);
  return cudaGetLastError();
}

cudaError_t plane_get_df64(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s) {
  lb_plane_get_kernel<DF, false><<<rows_grid(c), 128, 0, s>>>(k, static_cast<const float2*>(buf), out, c);
  return cudaGetLastError();
}

cudaError_t plane_put_df64(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s) {
  lb_plane_put_kernel<DF, false><<<rows_grid(c), 128, 0, s>>>(k, in, static_cast<float2*>(buf), c);
  return cudaGetLastError();
}

}  // namespace tlb
