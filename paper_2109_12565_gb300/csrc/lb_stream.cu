// Strip-marching, TMA-fed fused step for FP32-shifted storage on sm_103a.
//
// Same arithmetic as lb_step_kernel (phase A and phase B of lb_kernels.cuh,
// the same device functions); only the order in which nodes are visited and
// the way the populations reach the SM change.  A CTA owns a strip of 64
// columns and a segment of rows and walks it upwards in groups of 4 rows:
//
//   iteration q:  wait for the tensor copy of row group q (18 fluid planes,
//                 72 x 4 box at (x0 - 4, ya - 2 + 4q), 16-byte aligned start);
//                 phase A of group q: rho deviations, psi and momentum of the
//                 4 rows x 68 columns into a row window in shared memory;
//                 issue the copy of group q + NS into the stage just read;
//                 phase B of the 64 x 4 nodes of group q - 1 (forces from the
//                 window rows of groups q - 1 and q, collision, push stores);
//                 load the thermal populations of group q into registers.
//
// Phase A rows run 2 ahead of phase B rows, which is exactly the reach of
// the force stencil (Eqs. FAB, FintAttrattive, FintRepulsive), so each row's
// rho and psi are computed once per segment: only the 2 rows below and
// above a segment are recomputed by its neighbours, against a 2-node ring
// on all four sides of a tile in the tile kernel.  NS stages keep up to NS
// row groups in flight while the SM computes, so the copies of a CTA overlap
// its own compute instead of only other CTAs' compute.
//
// The window holds two row groups; the even group is also written 8 rows
// further down, so the 8 rows a phase B group reads are always contiguous
// and the force helper indexes them like a tile.  Columns that wrap around
// the periodic x boundary are read from global memory.  Lattices periodic in
// y are not handled here (the autotuner then runs the tile kernel).  Every
// mbarrier wait is bounded by an SM-clock budget; a wait that runs out sets
// the error word, waits (bounded) for the copies still in flight and returns.
#include "lb_tma_util.cuh"

namespace tlb {

constexpr int kSW = 64;          // strip width (nodes)
constexpr int kSR = 4;           // rows per group
constexpr int kSBX = kSW + 8;    // copied columns: x0 - 4 .. x0 + 67
constexpr int kSRX = kSW + 4;    // window columns: x0 - 2 .. x0 + 65
constexpr int kSWR = 3 * kSR;    // window rows: groups of parity 0, 1, then parity 0 again
constexpr int kSNT = kSW * kSR;  // threads per CTA: one node of a group each

struct StreamWin {
  float2 rho[kSWR][kSRX];  // density deviations rho_l - rho_bar_l, components interleaved
  float2 psi[kSWR][kSRX];
  float jx[kSWR][kSW], jy[kSWR][kSW];
  unsigned char solid[kSWR][kSRX];
};

template <int NS> struct alignas(128) StreamSmem {
  float stage[NS][18][kSR][kSBX];
  StreamWin w;
  unsigned long long bar[NS];
};

// Phase B of one node of a group (MODE_STEP of tile_phase_b with the window as the tile).
template <bool FAST>
__device__ __forceinline__ void stream_node(const float* __restrict__ fin, float* __restrict__ fout,
                                            const KParams<float>& kp, const StreamWin& w, int cx, int cy, int gx,
                                            int gy, const float g[9]) {
  if (!FAST && w.solid[cy][cx]) return;
  const int idx = gy * kp.pitch + gx, plane = kp.plane;
  float f[9], h[9];
  if (!kp.tau_is_one) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      f[i] = fin[idx + i * plane];
      h[i] = fin[idx + (9 + i) * plane];
    }
  }
  const float dr1 = w.rho[cy][cx].x, dr2 = w.rho[cy][cx].y;
  const float r1 = dr1 + kp.rho_bar[0], r2 = dr2 + kp.rho_bar[1];
  float dT = 0.0f;
#pragma unroll
  for (int i = 0; i < 9; ++i) dT += g[i];
  const float T = dT + kp.T_bar;
  const float jx = w.jx[cy][cx - 2], jy = w.jy[cy][cx - 2];
  float Fx[2], Fy[2];
  node_forces<float>(w, kp, cx, cy, r1, r2, T, Fx, Fy);
  float i1, i2, inv_rho, ux, uy, uHx, uHy;
  three_reciprocals<float>(r1, r2, i1, i2, inv_rho);
  node_velocities<float>(jx, jy, inv_rho, Fx, Fy, ux, uy, uHx, uHy);
  float post[27];
  node_collide<float, true>(kp, f, h, g, r1, r2, dr1, dr2, T, dT, ux, uy, i1, i2, Fx, Fy, uHx, uHy, post);
  push_store<float, float, FAST, kSRX>(fout, kp, idx, gx, gy, post, w.solid, cx, cy, r1, r2);
}

// Grid: (strips, segments).  Segment s covers row groups [s G / S, (s + 1) G / S) of the G = ceil(ny / 4).
template <int NS, int MINB>
__global__ void __launch_bounds__(kSNT, MINB)
lb_step_stream_kernel(const __grid_constant__ CUtensorMap map_fluid, const float* __restrict__ fin,
                      float* __restrict__ fout, const KParams<float> kp, int* err, int groups_total, long long budget) {
  extern __shared__ __align__(128) unsigned char smem_stream[];
  auto& sm = *reinterpret_cast<StreamSmem<NS>*>(smem_stream);
  constexpr uint32_t kStageBytes = 18 * kSR * kSBX * sizeof(float);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kSW + tx;
  if ((smem_u32(&sm.stage[0][0][0][0]) & 127u) != 0) {  // tensor copies need 128-byte aligned destinations
    if (tid == 0) atomicExch(err, kErrWaitTimeout);
    return;
  }
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  const int x0 = blockIdx.x * kSW;
  const int g0 = (int)((long long)blockIdx.y * groups_total / gridDim.y);
  const int g1 = (int)((long long)(blockIdx.y + 1) * groups_total / gridDim.y);
  const int n_b = g1 - g0;  // phase B groups; phase A runs n_b + 1 groups
  if (n_b <= 0) return;
  const int ya = g0 * kSR, yb = min(ny, g1 * kSR);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) mbar_init(&sm.bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int q) {
    const int s = q % NS;
    mbar_expect_tx(&sm.bar[s], kStageBytes);
    tma_load_3d(&sm.stage[s][0][0][0], &map_fluid, &sm.bar[s], x0 - 4, ya - 2 + q * kSR, 0);
  };
  if (tid == 0)
    for (int q = 0; q < NS && q <= n_b; ++q) issue(q);

  const int gx = x0 + tx;
  const bool no_wrap_x = x0 >= 1 && x0 + kSW + 1 <= nx;
  float gpre[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) gpre[i] = 0.0f;
  auto prefetch_thermal = [&](int p) {  // g_i of the node this thread pushes in phase B group p
    const int gy = ya + p * kSR + ty;
    if (gx < nx && gy < yb) {
      const float* src = fin + 18 * (long long)plane + gy * pitch + gx;
#pragma unroll
      for (int i = 0; i < 9; ++i) gpre[i] = src[i * plane];
    }
  };
  prefetch_thermal(0);
  int solid_prev = 0;
  for (int q = 0; q <= n_b; ++q) {
    const int s = q % NS;
    const int timed_out = __syncthreads_or(stage_wait(&sm.bar[s], (uint32_t)((q / NS) & 1), budget) ? 0 : 1);
    if (timed_out) {
      if (tid == 0) {
        atomicExch(err, kErrWaitTimeout);
        for (int r = q + 1; r <= n_b && r < q + NS; ++r)  // copies still in flight
          stage_wait(&sm.bar[r % NS], (uint32_t)((r / NS) & 1), budget);
      }
      return;
    }
    // ---- phase A of row group q: rows ya - 2 + 4q .. ya + 1 + 4q, columns x0 - 2 .. x0 + 65
    const int wbase = (q & 1) * kSR;
    const bool mirror = (q & 1) == 0;
    int ring_solid = 0;
    for (int r = tid; r < kSR * kSRX; r += kSNT) {
      const int ry = r / kSRX, rx = r - ry * kSRX;
      const int gxr = x0 + rx - 2;
      const int gxw = gxr < 0 ? gxr + nx : (gxr >= nx ? gxr - nx : gxr);
      const int gy = ya - 2 + q * kSR + ry;
      const bool solid = (gy <= 0 || gy >= ny - 1) || (kp.mask != nullptr && kp.mask[gy * nx + gxw] != 0);
      if (solid && rx >= 1 && rx <= kSW + 2) ring_solid = 1;
      const int wr = wbase + ry;
      float d1, d2, p1, p2;
      if (solid) {
        d1 = kp.drho_w[0];
        d2 = kp.drho_w[1];
        p1 = kp.psi_w[0];
        p2 = kp.psi_w[1];
      } else {
        float f[9], h[9];
        if (gxr == gxw) {
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            f[i] = sm.stage[s][i][ry][rx + 2];
            h[i] = sm.stage[s][9 + i][ry][rx + 2];
          }
        } else {
          const float* src = fin + (gy * pitch + gxw);
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            f[i] = src[i * plane];
            h[i] = src[(9 + i) * plane];
          }
        }
        d1 = 0.0f;
        d2 = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          d1 += f[i];
          d2 += h[i];
        }
        p1 = psi_exp<float>(d1 + kp.rho_bar[0], kp.rho0, kp.inv_rho0);
        p2 = psi_exp<float>(d2 + kp.rho_bar[1], kp.rho0, kp.inv_rho0);
        if (rx >= 2 && rx < kSW + 2) {
          const float jx = (f[1] - f[3] + f[5] - f[6] - f[7] + f[8]) + (h[1] - h[3] + h[5] - h[6] - h[7] + h[8]);
          const float jy = (f[2] - f[4] + f[5] + f[6] - f[7] - f[8]) + (h[2] - h[4] + h[5] + h[6] - h[7] - h[8]);
          sm.w.jx[wr][rx - 2] = jx;
          sm.w.jy[wr][rx - 2] = jy;
          if (mirror) {
            sm.w.jx[wr + 2 * kSR][rx - 2] = jx;
            sm.w.jy[wr + 2 * kSR][rx - 2] = jy;
          }
        }
      }
      sm.w.rho[wr][rx] = make_float2(d1, d2);
      sm.w.psi[wr][rx] = make_float2(p1, p2);
      sm.w.solid[wr][rx] = solid ? 1 : 0;
      if (mirror) {
        sm.w.rho[wr + 2 * kSR][rx] = make_float2(d1, d2);
        sm.w.psi[wr + 2 * kSR][rx] = make_float2(p1, p2);
        sm.w.solid[wr + 2 * kSR][rx] = solid ? 1 : 0;
      }
    }
    const int solid_cur = __syncthreads_or(ring_solid);  // the window is complete, stage s is free
    if (tid == 0 && q + NS <= n_b) issue(q + NS);
    // ---- phase B of row group q - 1: rows ya + 4(q - 1) .. ya + 4q - 1
    if (q >= 1) {
      const int p = q - 1;
      const int gy = ya + p * kSR + ty;
      const int cy = (p & 1) * kSR + ty + 2, cx = tx + 2;
      if (!(solid_prev | solid_cur) && no_wrap_x)
        stream_node<true>(fin, fout, kp, sm.w, cx, cy, gx, gy, gpre);
      else if (gx < nx && gy < yb)
        stream_node<false>(fin, fout, kp, sm.w, cx, cy, gx, gy, gpre);
      if (q < n_b) prefetch_thermal(q);
    }
    solid_prev = solid_cur;
  }
}

}  // namespace tlb

namespace {

using tlb::TileChoice;
using tlb_tma_host::make_map;

// CTAS_PER_SM > 0: segments so that the grid fills CTAS_PER_SM CTAs on every SM (at most the resident
// count); 0: one segment per strip (each CTA walks a whole column of the lattice).
template <int NS, int MINB, int CTAS_PER_SM>
cudaError_t launch_stream(const tlb::StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  using namespace tlb;
  static_assert((18 * kSR * kSBX * sizeof(float)) % 128 == 0, "TMA stages must stay 128-byte aligned");
  static_assert((kSBX * sizeof(float)) % 16 == 0, "TMA box rows must be multiples of 16 bytes");
  static_assert(kSW % 4 == 0, "strip starts x0 - 4 must be 16-byte aligned");
  if (c.err == nullptr || c.periodic_y || c.nx < 2 * kSW || c.ny < 2 * kSR || ((uintptr_t)fin % 16) != 0 ||
      (c.pitch * 4) % 16 != 0)
    return cudaErrorNotSupported;
  CUtensorMap mf;
  if (!make_map(&mf, c, fin, kSBX, kSR, 18)) return cudaErrorNotSupported;
  auto k = lb_step_stream_kernel<NS, MINB>;
  constexpr size_t bytes = sizeof(StreamSmem<NS>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kSNT, bytes)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorNotSupported;
  const int strips = (c.nx + kSW - 1) / kSW, groups = (c.ny + kSR - 1) / kSR;
  int nseg = 1;
  if (CTAS_PER_SM > 0) {
    const int per_sm = occ < CTAS_PER_SM ? occ : CTAS_PER_SM;
    nseg = (sms * per_sm) / strips;
    if (nseg < 1) nseg = 1;
    if (nseg > groups) nseg = groups;
  }
  const long long budget = 4000000000LL;  // SM clock cycles (about 2 s)
  k<<<dim3((unsigned)strips, (unsigned)nseg, 1), dim3(kSW, kSR, 1), bytes, s>>>(
      mf, static_cast<const float*>(fin), static_cast<float*>(fout), make_kparams<float>(c), c.err, groups, budget);
  return cudaGetLastError();
}

struct StreamCand {
  TileChoice t;
  cudaError_t (*fn)(const tlb::StepCfg&, const void*, void*, cudaStream_t);
};
// {strip width, rows per group, threads / strip width, resident CTAs per SM asked of the compiler}
const StreamCand kStream[] = {
    {{tlb::kSW, tlb::kSR, tlb::kSR, 3}, launch_stream<2, 3, 3>},
    {{tlb::kSW, tlb::kSR, tlb::kSR, 2}, launch_stream<3, 2, 2>},
    {{tlb::kSW, tlb::kSR, tlb::kSR, 3}, launch_stream<2, 3, 2>},
    {{tlb::kSW, tlb::kSR, tlb::kSR, 3}, launch_stream<2, 3, 0>},
};

}  // namespace

namespace tlb {

int stream_count_f32() { return (int)(sizeof kStream / sizeof kStream[0]); }
TileChoice stream_info_f32(int k) { return kStream[k].t; }
cudaError_t launch_step_stream_f32(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return kStream[k].fn(c, fin, fout, s);
}

}  // namespace tlb
