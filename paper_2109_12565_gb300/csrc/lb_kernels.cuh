// Fused single-pass lattice Boltzmann step of the thermal two-component
// emulsion model (TLBfind, arXiv 2109.12565, Sec. 2.1-2.3) for sm_103a.
//
// Storage: structure of arrays, 27 planes (f_{1,0..8}, f_{2,0..8}, g_{0..8})
// of pitch * ny elements, x fastest, rows 128-byte aligned.  A buffer holds
// the PRE-collision populations S_t, so every moment is a local sum and the
// force stencil only needs densities within two nodes.  One CTA owns a
// TX x TY tile:
//   phase A: for the tile plus a 2-node ring, rho_1, rho_2 (local sums of the
//            18 fluid populations) and psi_l = rho0 (1 - exp(-rho_l / rho0))
//            go to shared memory; solid and out-of-domain nodes take the wall
//            densities (Sec. 2.2.1).  One exp per node and component.
//   phase B: per fluid node of the tile: load its 27 populations, momentum
//            and T, the 8-link cross force (Eq. FAB) and the 24-link
//            self force (Eqs. FintAttrattive + FintRepulsive folded into one
//            weighted stencil, evaluated as 12 antisymmetric pair
//            differences), buoyancy (Eq. alphaG), the shifted velocities
//            (Eq. shift, u^(H)), BGK relaxation (Eqs. BGK, LBMg) and the
//            push-store of f*(x) to x + c_i of the other buffer, bouncing back
//            (Sec. 2.2) or anti-bouncing (thermal walls) when x + c_i is solid.
// Writes of direction i from a warp land on one contiguous row shifted by
// c_i; each destination slot has exactly one writer per step.
#pragma once
#include <math.h>
#include <stdint.h>

#include "lb_cfg.h"

namespace tlb {

// D2Q9 links (Fig. 1a): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
__host__ __device__ constexpr int cxq(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cyq(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int oppq(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
// D2Q9 weights w_i (Fig. 1b).
template <class C> __host__ __device__ constexpr C wq(int i) { return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36)); }

__device__ __forceinline__ int wrap_any(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <class C> __device__ __forceinline__ C psi_exp(C rho, C rho0, C inv_rho0);
template <> __device__ __forceinline__ double psi_exp<double>(double rho, double rho0, double inv_rho0) {
  return rho0 * (1.0 - exp(-rho * inv_rho0));
}
template <> __device__ __forceinline__ float psi_exp<float>(float rho, float rho0, float inv_rho0) {
  return -rho0 * expm1f(-rho * inv_rho0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <class S, class C, bool SHIFT, int MODE, int TX, int TY, int BY>
__global__ void __launch_bounds__(TX * BY)
lb_step_kernel(const S* __restrict__ fin, S* __restrict__ fout, const StepCfg cfg, double* __restrict__ aux) {
  constexpr int RX = TX + 4, RY = TY + 4, NT = TX * BY;
  constexpr bool NEED_T = (MODE != MODE_STEP);
  __shared__ C s_rho[2][RY][RX];
  __shared__ C s_psi[2][RY][RX];
  __shared__ C s_T[NEED_T ? RY : 1][NEED_T ? RX : 1];
  __shared__ unsigned char s_solid[RY][RX];

  const int nx = cfg.nx, ny = cfg.ny, pitch = cfg.pitch;
  const long long plane = cfg.plane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const C rho0 = C(cfg.rho0), inv_rho0 = C(cfg.inv_rho0);
  const C rb0 = SHIFT ? C(cfg.rho_bar[0]) : C(0), rb1 = SHIFT ? C(cfg.rho_bar[1]) : C(0);
  const C Tb = SHIFT ? C(cfg.T_bar) : C(0);

  // ---------------- phase A: densities and pseudo-potentials on the tile + 2-node ring
  for (int r = tid; r < RX * RY; r += NT) {
    const int ry = r / RX, rx = r - ry * RX;
    const int gx = wrap_any(x0 + rx - 2, nx);
    int gy = y0 + ry - 2;
    bool solid;
    if (cfg.periodic_y) {
      gy = wrap_any(gy, ny);
      solid = cfg.mask != nullptr && cfg.mask[(long long)gy * nx + gx] != 0;
    } else {
      solid = (gy <= 0 || gy >= ny - 1) || (cfg.mask != nullptr && cfg.mask[(long long)gy * nx + gx] != 0);
    }
    if (solid) {
      s_rho[0][ry][rx] = C(cfg.rho_w[0]);
      s_rho[1][ry][rx] = C(cfg.rho_w[1]);
      s_psi[0][ry][rx] = C(cfg.psi_w[0]);
      s_psi[1][ry][rx] = C(cfg.psi_w[1]);
      if (NEED_T) s_T[NEED_T ? ry : 0][NEED_T ? rx : 0] = C(2 * gy < ny ? cfg.T_down : cfg.T_up);
      s_solid[ry][rx] = 1;
    } else {
      const long long idx = (long long)gy * pitch + gx;
      C r1 = C(0), r2 = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        r1 += C(fin[i * plane + idx]);
        r2 += C(fin[(9 + i) * plane + idx]);
      }
      r1 += rb0;
      r2 += rb1;
      s_rho[0][ry][rx] = r1;
      s_rho[1][ry][rx] = r2;
      s_psi[0][ry][rx] = psi_exp<C>(r1, rho0, inv_rho0);
      s_psi[1][ry][rx] = psi_exp<C>(r2, rho0, inv_rho0);
      if (NEED_T) {
        C t = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) t += C(fin[(18 + i) * plane + idx]);
        s_T[NEED_T ? ry : 0][NEED_T ? rx : 0] = t + Tb;
      }
      s_solid[ry][rx] = 0;
    }
  }
  __syncthreads();

  // ---------------- phase B: one fluid node per (thread, k)
  const C inv_tau = C(cfg.inv_tau), inv_tau_g = C(cfg.inv_tau_g), tau = C(cfg.tau);
  const C gxc = C(cfg.gx), ag = C(cfg.alpha_g), bfx = C(cfg.body_fx);
  double acc[kObsSlots];
  if (MODE == MODE_OBS) {
#pragma unroll
    for (int v = 0; v < kObsSlots; ++v) acc[v] = 0.0;
  }

#pragma unroll 1
  for (int k = 0; k < TY / BY; ++k) {
    const int tx = threadIdx.x, ty = threadIdx.y + k * BY;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= nx || gy >= ny) continue;
    const int cx = tx + 2, cy = ty + 2;
    if (s_solid[cy][cx]) {
      if (MODE == MODE_FIELDS) {
        const long long n = (long long)gy * nx + gx, N = (long long)nx * ny;
        aux[n] = cfg.rho_w[0];
        aux[N + n] = cfg.rho_w[1];
        aux[2 * N + n] = (2 * gy < ny) ? cfg.T_down : cfg.T_up;
        aux[3 * N + n] = 0.0;
        aux[4 * N + n] = 0.0;
      }
      continue;
    }
    const long long idx = (long long)gy * pitch + gx;
    C f[9], h[9], g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      f[i] = C(fin[i * plane + idx]);
      h[i] = C(fin[(9 + i) * plane + idx]);
      g[i] = C(fin[(18 + i) * plane + idx]);
    }
    // moments (Sec. 2.1, 2.3); in shifted storage the sums are deviations from the shift
    const C r1 = s_rho[0][cy][cx], r2 = s_rho[1][cy][cx];
    C dr1 = C(0), dr2 = C(0), dT = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      dr1 += f[i];
      dr2 += h[i];
      dT += g[i];
    }
    const C T = dT + Tb;
    const C jx = (f[1] - f[3] + f[5] - f[6] - f[7] + f[8]) + (h[1] - h[3] + h[5] - h[6] - h[7] + h[8]);
    const C jy = (f[2] - f[4] + f[5] + f[6] - f[7] - f[8]) + (h[2] - h[4] + h[5] + h[6] - h[7] - h[8]);

    // forces, Eqs. FAB, FintAttrattive, FintRepulsive, alphaG
    C Fx[2], Fy[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int m = 1 - l;
      // cross term: -G12/rho0^2 rho_l(x) sum_{NN} w_i rho_m(x + c_i) c_i, as pair differences
      const C e10 = s_rho[m][cy][cx + 1] - s_rho[m][cy][cx - 1];
      const C e01 = s_rho[m][cy + 1][cx] - s_rho[m][cy - 1][cx];
      const C e11 = s_rho[m][cy + 1][cx + 1] - s_rho[m][cy - 1][cx - 1];
      const C em1 = s_rho[m][cy + 1][cx - 1] - s_rho[m][cy - 1][cx + 1];
      const C w1 = C(1) / C(9), w2 = C(1) / C(36);
      const C crx = w1 * e10 + w2 * (e11 - em1);
      const C cry = w1 * e01 + w2 * (e11 + em1);
      const C rl = (l == 0) ? r1 : r2;
      // self term: -psi_l(x) sum_{24 links} (G^a_ll w_i + G^r_ll p_i) psi_l(x + c_i) c_i
      const C d10 = s_psi[l][cy][cx + 1] - s_psi[l][cy][cx - 1];
      const C d01 = s_psi[l][cy + 1][cx] - s_psi[l][cy - 1][cx];
      const C d11 = s_psi[l][cy + 1][cx + 1] - s_psi[l][cy - 1][cx - 1];
      const C dm1 = s_psi[l][cy + 1][cx - 1] - s_psi[l][cy - 1][cx + 1];
      const C d20 = s_psi[l][cy][cx + 2] - s_psi[l][cy][cx - 2];
      const C d02 = s_psi[l][cy + 2][cx] - s_psi[l][cy - 2][cx];
      const C d12 = s_psi[l][cy + 2][cx + 1] - s_psi[l][cy - 2][cx - 1];
      const C dm12 = s_psi[l][cy + 2][cx - 1] - s_psi[l][cy - 2][cx + 1];
      const C d21 = s_psi[l][cy + 1][cx + 2] - s_psi[l][cy - 1][cx - 2];
      const C dm21 = s_psi[l][cy + 1][cx - 2] - s_psi[l][cy - 1][cx + 2];
      const C d22 = s_psi[l][cy + 2][cx + 2] - s_psi[l][cy - 2][cx - 2];
      const C dm22 = s_psi[l][cy + 2][cx - 2] - s_psi[l][cy - 2][cx + 2];
      const C a1 = C(cfg.a1[l]), a2 = C(cfg.a2[l]), a4 = C(cfg.a4x2[l]), a5 = C(cfg.a5[l]), a8 = C(cfg.a8x2[l]);
      const C sx = a1 * d10 + a2 * (d11 - dm1) + a4 * d20 + a5 * (d12 - dm12 + C(2) * (d21 - dm21)) + a8 * (d22 - dm22);
      const C sy = a1 * d01 + a2 * (d11 + dm1) + a4 * d02 + a5 * (C(2) * (d12 + dm12) + d21 + dm21) + a8 * (d22 + dm22);
      const C psl = s_psi[l][cy][cx];
      Fx[l] = -gxc * rl * crx - psl * sx + rl * bfx;
      Fy[l] = -gxc * rl * cry - psl * sy + rl * ag * T;
    }

    // velocities: Eq. velo, Eq. shift, u^(H) = u + F / (2 rho)
    const C rho = r1 + r2;
    const C inv_rho = C(1) / rho;
    const C ux = jx * inv_rho, uy = jy * inv_rho;
    const C uHx = ux + C(0.5) * (Fx[0] + Fx[1]) * inv_rho;
    const C uHy = uy + C(0.5) * (Fy[0] + Fy[1]) * inv_rho;

    if (MODE == MODE_OBS) {
      const C Tc = T;
      const C Tup = s_solid[cy + 1][cx] ? C(2) * s_T[NEED_T ? cy + 1 : 0][NEED_T ? cx : 0] - Tc
                                         : s_T[NEED_T ? cy + 1 : 0][NEED_T ? cx : 0];
      const C Tdn = s_solid[cy - 1][cx] ? C(2) * s_T[NEED_T ? cy - 1 : 0][NEED_T ? cx : 0] - Tc
                                         : s_T[NEED_T ? cy - 1 : 0][NEED_T ? cx : 0];
      acc[0] += (double)dr1;
      acc[1] += (double)dr2;
      acc[2] += (double)(rho * uHx);
      acc[3] += (double)(rho * uHy);
      acc[4] += (double)(uHy * T);
      acc[5] += 0.5 * ((double)Tup - (double)Tdn);
      acc[6] += (double)(uHx * uHx + uHy * uHy);
      const bool bad = !(r1 > C(0)) || !(r2 > C(0)) || !isfinite((double)r1) || !isfinite((double)r2) ||
                       !isfinite((double)T);
      acc[7] += bad ? 1.0 : 0.0;
      acc[8] += 1.0;
      continue;
    }
    if (MODE == MODE_FIELDS) {
      const long long n = (long long)gy * nx + gx, N = (long long)nx * ny;
      aux[n] = (double)r1;
      aux[N + n] = (double)r2;
      aux[2 * N + n] = (double)T;
      aux[3 * N + n] = (double)uHx;
      aux[4 * N + n] = (double)uHy;
      continue;
    }

    // BGK collisions: f* = f + (f^eq(rho_l, u_l) - f) / tau, g* = g + (g^eq(T, u^(H)) - g) / tau_g.
    // Shifted storage relaxes the deviations: f^eq - w_i rho_bar = w_i (drho + rho P_i(u)).
    C post[27];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const C rl = (l == 0) ? r1 : r2;
      const C inv_rl = C(1) / rl;
      const C ulx = ux + tau * Fx[l] * inv_rl, uly = uy + tau * Fy[l] * inv_rl;
      const C usq = C(1.5) * (ulx * ulx + uly * uly);
      const C base = SHIFT ? ((l == 0) ? dr1 : dr2) : rl;
      const C* pop = (l == 0) ? f : h;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C cu = C(cxq(i)) * ulx + C(cyq(i)) * uly;
        const C poly = cu * (C(3) + C(4.5) * cu) - usq;
        const C feq = wq<C>(i) * (base + rl * poly);
        post[9 * l + i] = pop[i] + (feq - pop[i]) * inv_tau;
      }
    }
    {
      const C usq = C(1.5) * (uHx * uHx + uHy * uHy);
      const C base = SHIFT ? dT : T;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C cu = C(cxq(i)) * uHx + C(cyq(i)) * uHy;
        const C poly = cu * (C(3) + C(4.5) * cu) - usq;
        const C geq = wq<C>(i) * (base + T * poly);
        post[18 + i] = g[i] + (geq - g[i]) * inv_tau_g;
      }
    }

    // streaming (push) with half-way bounce-back / thermal anti-bounce-back
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sxl = cx + cxq(i), syl = cy + cyq(i);
      if (!s_solid[syl][sxl]) {
        int dx = gx + cxq(i);
        dx = dx < 0 ? dx + nx : (dx >= nx ? dx - nx : dx);
        int dy = gy + cyq(i);
        if (cfg.periodic_y) dy = dy < 0 ? dy + ny : (dy >= ny ? dy - ny : dy);
        const long long didx = (long long)dy * pitch + dx;
        fout[i * plane + didx] = S(post[i]);
        fout[(9 + i) * plane + didx] = S(post[9 + i]);
        fout[(18 + i) * plane + didx] = S(post[18 + i]);
      } else {
        const int o = oppq(i);
        const int wy = gy + cyq(i);
        const C Tw = C(2 * wy < ny ? cfg.T_down : cfg.T_up) - Tb;
        fout[o * plane + idx] = S(post[i]);
        fout[(9 + o) * plane + idx] = S(post[9 + i]);
        fout[(18 + o) * plane + idx] = S(-post[18 + i] + C(2) * wq<C>(i) * Tw);
      }
    }
  }

  if (MODE == MODE_OBS) {
    __shared__ double s_red[NT / 32][kObsSlots];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int v = 0; v < kObsSlots; ++v) {
      const double s = warp_sum(acc[v]);
      if (lane == 0) s_red[warp][v] = s;
    }
    __syncthreads();
    if (tid < kObsSlots) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += s_red[w][tid];
      aux[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * kObsSlots + tid] = s;
    }
  }
}

// Rest equilibria f = w_i rho, g = w_i T at fluid nodes (stored minus the shift), 0 at solid nodes.
template <class S, bool SHIFT>
__global__ void lb_init_kernel(const double* __restrict__ fields, S* __restrict__ buf, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx, N = (long long)cfg.nx * cfg.ny;
  const long long idx = (long long)gy * cfg.pitch + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  const double r1 = fields[n], r2 = fields[N + n], T = fields[2 * N + n];
  for (int i = 0; i < 9; ++i) {
    const double w = wq<double>(i);
    double a = w * r1, b = w * r2, c = w * T;
    if (SHIFT) {
      a = w * (r1 - cfg.rho_bar[0]);
      b = w * (r2 - cfg.rho_bar[1]);
      c = w * (T - cfg.T_bar);
    }
    buf[i * cfg.plane + idx] = solid ? S(0) : S(a);
    buf[(9 + i) * cfg.plane + idx] = solid ? S(0) : S(b);
    buf[(18 + i) * cfg.plane + idx] = solid ? S(0) : S(c);
  }
}

__device__ __forceinline__ double shift_of(const StepCfg& cfg, int k) {
  const int comp = k / 9, i = k % 9;
  const double s = comp == 0 ? cfg.rho_bar[0] : (comp == 1 ? cfg.rho_bar[1] : cfg.T_bar);
  return wq<double>(i) * s;
}

template <class S, bool SHIFT>
__global__ void lb_plane_get_kernel(int k, const S* __restrict__ buf, double* __restrict__ out, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  const double v = (double)buf[k * cfg.plane + (long long)gy * cfg.pitch + gx];
  out[n] = solid ? 0.0 : (SHIFT ? v + shift_of(cfg, k) : v);
}

template <class S, bool SHIFT>
__global__ void lb_plane_put_kernel(int k, const double* __restrict__ in, S* __restrict__ buf, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  const double v = SHIFT ? in[n] - shift_of(cfg, k) : in[n];
  buf[k * cfg.plane + (long long)gy * cfg.pitch + gx] = solid ? S(0) : S(v);
}

template <class S, bool SHIFT>
cudaError_t launch_impl(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  using T = Tile<S>;
  const dim3 grid = grid_for(c.nx, c.ny, T::TX, T::TY), block(T::TX, T::BY, 1);
  const S* in = static_cast<const S*>(fin);
  S* out = static_cast<S*>(fout);
  switch (mode) {
    case MODE_STEP:
      lb_step_kernel<S, S, SHIFT, MODE_STEP, T::TX, T::TY, T::BY><<<grid, block, 0, s>>>(in, out, c, aux);
      break;
    case MODE_OBS:
      lb_step_kernel<S, S, SHIFT, MODE_OBS, T::TX, T::TY, T::BY><<<grid, block, 0, s>>>(in, out, c, aux);
      break;
    case MODE_FIELDS:
      lb_step_kernel<S, S, SHIFT, MODE_FIELDS, T::TX, T::TY, T::BY><<<grid, block, 0, s>>>(in, out, c, aux);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

inline dim3 rows_grid(const StepCfg& c) { return dim3((unsigned)((c.nx + 127) / 128), (unsigned)c.ny, 1u); }

}  // namespace tlb
