// TMA-fed, software-pipelined fused step for FP32-shifted storage on sm_103a.
//
// Same arithmetic as lb_step_kernel (phase A and phase B of lb_kernels.cuh);
// only the way the populations reach the SM changes.  For each tile one
// elected thread issues two tensor copies (cp.async.bulk.tensor.3d) into a
// shared-memory stage:
//   - the 18 fluid planes of the (TX + 8) x (TY + 4) box starting at
//     (x0 - 4, y0 - 2): the tile, its 2-node ring and 2 more columns on each
//     side so that the box starts on a 16-byte boundary;
//   - the 9 thermal planes of the TX x TY tile itself.
// Two variants: a persistent grid (one CTA per SM) with two stages and two
// mbarriers (complete_tx), so the copies of tile j + 1 run while tile j is
// computed; and one tile per CTA with one stage, several CTAs per SM.  Columns that wrap around the periodic x
// boundary (and rows that wrap in periodic y) fall outside the box and are
// read from global memory instead.  Every mbarrier wait is bounded by an
// SM-clock budget; a wait that runs out sets the error word, waits (again
// bounded) for the copies still in flight, and the kernel returns; the host
// reports LB_ETIMEOUT.
#include <cuda.h>
#include <cuda_runtime.h>

#include "lb_tma_util.cuh"

namespace tlb {

template <int TX, int TY> struct TmaStage {
  float fluid[18][TY + 4][TX + 8];
  float thermal[9][TY][TX];
};

template <int TX, int TY, int STAGES> struct alignas(128) TmaSmem {
  TmaStage<TX, TY> stage[STAGES];
  TileSmem<float, TX, TY, false> t;
  unsigned long long bar[STAGES];
};

// Phase B source: the tile's own populations from the shared-memory stage.
template <int TX, int TY> struct StagePopSource {
  const TmaStage<TX, TY>* st;
  __device__ __forceinline__ float operator()(int k, int /*idx*/, int tx, int ty) const {
    return k < 18 ? st->fluid[k][ty + 2][tx + 4] : st->thermal[k - 18][ty][tx];
  }
};

// Phase A with the fluid populations taken from the stage (wrapped positions from global memory).
template <int TX, int TY, int NT>
__device__ __forceinline__ bool tma_phase_a(const float* __restrict__ fin, const KParams<float>& kp, int x0, int y0,
                                            const TmaStage<TX, TY>& st, TileSmem<float, TX, TY, false>& sm, int tid) {
  constexpr int RX = TX + 4, RY = TY + 4;
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  const bool small_x = nx < TX + 4, small_y = ny < TY + 4;
  int ring_solid = 0;
  for (int r = tid; r < RX * RY; r += NT) {
    const int ry = r / RX, rx = r - ry * RX;
    const int gxr = x0 + rx - 2, gyr = y0 + ry - 2;
    int gx = small_x ? wrap_any(gxr, nx) : (gxr < 0 ? gxr + nx : (gxr >= nx ? gxr - nx : gxr));
    int gy = gyr;
    bool solid;
    if (kp.periodic_y) {
      gy = small_y ? wrap_any(gyr, ny) : (gyr < 0 ? gyr + ny : (gyr >= ny ? gyr - ny : gyr));
      solid = kp.mask != nullptr && kp.mask[gy * nx + gx] != 0;
    } else {
      solid = (gy <= 0 || gy >= ny - 1) || (kp.mask != nullptr && kp.mask[gy * nx + gx] != 0);
    }
    if (solid && rx >= 1 && rx <= TX + 2 && ry >= 1 && ry <= TY + 2) ring_solid = 1;
    if (solid) {
      sm.rho[ry][rx] = v2<float>(kp.drho_w[0], kp.drho_w[1]);
      sm.psi[ry][rx] = v2<float>(kp.psi_w[0], kp.psi_w[1]);
      sm.solid[ry][rx] = 1;
      continue;
    }
    const bool in_box = gxr >= 0 && gxr < nx && gyr >= 0 && gyr < ny;
    float f[9], h[9];
    if (in_box) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f[i] = st.fluid[i][ry][rx + 2];
        h[i] = st.fluid[9 + i][ry][rx + 2];
      }
    } else {
      const float* src = fin + (gy * pitch + gx);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f[i] = src[i * plane];
        h[i] = src[(9 + i) * plane];
      }
    }
    float d1 = 0.0f, d2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      d1 += f[i];
      d2 += h[i];
    }
    sm.rho[ry][rx] = v2<float>(d1, d2);
    sm.psi[ry][rx] = v2<float>(psi_exp<float>(d1 + kp.rho_bar[0], kp.rho0, kp.inv_rho0),
                               psi_exp<float>(d2 + kp.rho_bar[1], kp.rho0, kp.inv_rho0));
    if (rx >= 2 && rx < TX + 2 && ry >= 2 && ry < TY + 2) {
      sm.jx[ry - 2][rx - 2] = (f[1] - f[3] + f[5] - f[6] - f[7] + f[8]) + (h[1] - h[3] + h[5] - h[6] - h[7] + h[8]);
      sm.jy[ry - 2][rx - 2] = (f[2] - f[4] + f[5] + f[6] - f[7] - f[8]) + (h[2] - h[4] + h[5] + h[6] - h[7] - h[8]);
    }
    sm.solid[ry][rx] = 0;
  }
  const int any = __syncthreads_or(ring_solid);
  const bool no_wrap_x = x0 >= 1 && x0 + TX + 1 <= nx;
  const bool no_wrap_y = !kp.periodic_y || (y0 >= 1 && y0 + TY + 1 <= ny);
  return !any && no_wrap_x && no_wrap_y;
}

// STAGES = 2: persistent grid, two stages, the copies of the next tile overlap this tile's compute.
// STAGES = 1: one tile per CTA (grid = tiles); several CTAs per SM overlap each other's copies.
template <int TX, int TY, int BY, int STAGES>
__global__ void __launch_bounds__(TX * BY, STAGES == 1 ? 2 : 1)
lb_step_tma_kernel(const __grid_constant__ CUtensorMap map_fluid, const __grid_constant__ CUtensorMap map_thermal,
                   const float* __restrict__ fin, float* __restrict__ fout, const KParams<float> kp, int* err,
                   int n_tiles, int tiles_x, long long budget) {
  extern __shared__ __align__(128) unsigned char smem_tma[];
  auto& sm = *reinterpret_cast<TmaSmem<TX, TY, STAGES>*>(smem_tma);
  constexpr int NT = TX * BY;
  constexpr uint32_t kStageBytes = sizeof(TmaStage<TX, TY>);
  const int tid = threadIdx.y * TX + threadIdx.x;
  if ((smem_u32(&sm.stage[0]) & 127u) != 0) {  // tensor copies need 128-byte aligned destinations
    if (tid == 0) atomicExch(err, kErrWaitTimeout);
    return;
  }
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < STAGES; ++q) mbar_init(&sm.bar[q], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int tile, int s) {
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    mbar_expect_tx(&sm.bar[s], kStageBytes);
    tma_load_3d(&sm.stage[s].fluid[0][0][0], &map_fluid, &sm.bar[s], x0 - 4, y0 - 2, 0);
    tma_load_3d(&sm.stage[s].thermal[0][0][0], &map_thermal, &sm.bar[s], x0, y0, 18);
  };
  if (tid == 0) {
    if ((int)blockIdx.x < n_tiles) issue(blockIdx.x, 0);
    if (STAGES == 2 && (int)(blockIdx.x + gridDim.x) < n_tiles) issue(blockIdx.x + gridDim.x, STAGES - 1);
  }
  double acc[kObsSlots];
  int j = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++j) {
    const int s = STAGES == 2 ? (j & 1) : 0;
    const uint32_t parity = (uint32_t)((STAGES == 2 ? (j >> 1) : j) & 1);
    const int timed_out = __syncthreads_or(stage_wait(&sm.bar[s], parity, budget) ? 0 : 1);
    if (timed_out) {
      if (tid == 0) {
        atomicExch(err, kErrWaitTimeout);
        // the other stage may still have a copy in flight: wait for it, again bounded
        if (STAGES == 2 && tile + (int)gridDim.x < n_tiles)
          stage_wait(&sm.bar[STAGES - 1 - s], (uint32_t)(((j + 1) >> 1) & 1), budget);
      }
      return;
    }
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    const bool fast = tma_phase_a<TX, TY, NT>(fin, kp, x0, y0, sm.stage[s], sm.t, tid);
    const StagePopSource<TX, TY> pop{&sm.stage[s]};
    if (fast)
      tile_phase_b<float, float, true, MODE_STEP, true, TX, TY, BY>(pop, fout, kp, x0, y0, sm.t, nullptr, acc);
    else
      tile_phase_b<float, float, true, MODE_STEP, false, TX, TY, BY>(pop, fout, kp, x0, y0, sm.t, nullptr, acc);
    __syncthreads();  // stage s and the tile arrays are free again
    if (tid == 0 && tile + STAGES * (int)gridDim.x < n_tiles) issue(tile + STAGES * gridDim.x, s);
  }
}

}  // namespace tlb

namespace {

using tlb::TileChoice;
using tlb_tma_host::make_map;

template <int TX, int TY, int BY, int STAGES>
cudaError_t launch_tma(const tlb::StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  using namespace tlb;
  static_assert(sizeof(TmaStage<TX, TY>) % 128 == 0, "TMA stages must stay 128-byte aligned");
  static_assert(((TX + 8) * 4) % 16 == 0 && (TX * 4) % 16 == 0, "TMA box rows must be multiples of 16 bytes");
  if (c.err == nullptr || ((uintptr_t)fin % 16) != 0 || (c.pitch * 4) % 16 != 0) return cudaErrorNotSupported;
  CUtensorMap mf, mt;
  if (!make_map(&mf, c, fin, TX + 8, TY + 4, 18) || !make_map(&mt, c, fin, TX, TY, 9)) return cudaErrorNotSupported;
  auto k = lb_step_tma_kernel<TX, TY, BY, STAGES>;
  constexpr size_t bytes = sizeof(TmaSmem<TX, TY, STAGES>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, TX * BY, bytes)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorNotSupported;
  const int tiles_x = (c.nx + TX - 1) / TX, tiles_y = (c.ny + TY - 1) / TY, n_tiles = tiles_x * tiles_y;
  const int grid = STAGES == 1 ? n_tiles : (n_tiles < sms * occ ? n_tiles : sms * occ);
  const long long budget = 4000000000LL;  // SM clock cycles (about 2 s)
  k<<<grid, dim3(TX, BY, 1), bytes, s>>>(mf, mt, static_cast<const float*>(fin), static_cast<float*>(fout),
                                         make_kparams<float>(c), c.err, n_tiles, tiles_x, budget);
  return cudaGetLastError();
}

struct TmaCand {
  TileChoice t;
  cudaError_t (*fn)(const tlb::StepCfg&, const void*, void*, cudaStream_t);
};
// {tx, ty, threads / tx, stages}
const TmaCand kTma[] = {
    {{64, 8, 8, 2}, launch_tma<64, 8, 8, 2>},
    {{32, 16, 8, 2}, launch_tma<32, 16, 8, 2>},
    {{64, 8, 8, 1}, launch_tma<64, 8, 8, 1>},
    {{64, 8, 4, 1}, launch_tma<64, 8, 4, 1>},
    {{32, 16, 8, 1}, launch_tma<32, 16, 8, 1>},
};

}  // namespace

namespace tlb {

int tma_count_f32() { return (int)(sizeof kTma / sizeof kTma[0]); }
TileChoice tma_info_f32(int k) { return kTma[k].t; }
cudaError_t launch_step_tma_f32(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kTma[k].fn(c, fin, fout, s);
}

}  // namespace tlb
