// Discrete adjoint of the fused step and of the time-averaged Nusselt number
//   J = (1/N) sum_{t=1..N} Nu(S_t)          (Nu of Eq. NuTime)
// with respect to the initial temperature field T0 and the bottom-wall
// temperature T_down.  The paper has no adjoint; this is reverse-mode
// differentiation of the forward update of lb_kernels.cuh.
//
// One reverse step lam_t = (dS_{t+1}/dS_t)^T lam_{t+1} + cJ dNu(S_t)/dS_t is
// two tile kernels:
//   adj1  recomputes the forward moments, forces and velocities of S_t
//         (phase A of the forward), pulls lam_{t+1} back along the
//         streaming links (bounce-back and anti-bounce-back transposed),
//         runs the adjoint of the BGK collisions and of the velocity shift,
//         u^(H), u = j / rho and the buoyancy, and the parts of the force
//         adjoint local to the node; it writes lam_t minus the non-local
//         density terms, plus lam_F (the adjoint of the four force
//         components) and the node densities, and accumulates dJ/dT_down
//         per block;
//   adj2  gathers lam_F over the transposed stencils (8 links for the cross
//         force, 24 for the self force) on a 2-node ring, maps the
//         pseudo-potential adjoints back to the densities and adds them to
//         the 18 fluid entries of lam_t.
// The Nu seed needs only d(u_y T)/dS: the mirror-rule temperature gradient
// of Eq. NuTime sums to the wall temperatures (it telescopes column by
// column), so it contributes only to dJ/dT_down.
// lb_adjoint runs the forward pass with Nu after every step and stores a
// checkpoint every `ckpt_every` steps, then walks the segments backwards,
// recomputing each segment's states from its checkpoint.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "lb_host.h"
#include "lb_kernels.cuh"

using namespace tlb;

namespace tlb {

// Tile of the reverse-step kernels and the resident CTAs per SM asked of the compiler: FP32 fits 80
// registers without spills at 3 CTAs per SM; FP64 needs its ~240 registers (a cap spills), two
// 128-thread CTAs per SM.  FP64 is bound by its arithmetic per node, so small tiles cost little ring
// recompute and even out the SMs' shares: at 512 x 256, 128-node tiles leave every SM at most 7 of
// them (896 nodes against a mean of 862), 512-node tiles up to 2 (1024).  In FP32, 16 x 8 tiles
// measured 9% slower than 32 x 8.
template <class S> struct AdjTile;
template <> struct AdjTile<double> { static constexpr int TX = 16, TY = 8, BY = 8, MINB = 2; };
template <> struct AdjTile<float> { static constexpr int TX = 32, TY = 8, BY = 8, MINB = 3; };

// c v for a lattice-velocity component c in {-1, 0, 1} that is a constant once the direction loops are
// unrolled: no product with zero is issued (IEEE arithmetic cannot drop one: 0 v is NaN for infinite
// v and -0 for negative v), and for finite v every sum it enters keeps its value.
template <class C> __device__ __forceinline__ C cmul(int c, C v) { return c == 0 ? C(0) : (c > 0 ? v : -v); }
// c . v of direction i.
template <class C> __device__ __forceinline__ C cdot(int i, C vx, C vy) {
  return cxq(i) == 0 ? cmul(cyq(i), vy) : (cyq(i) == 0 ? cmul(cxq(i), vx) : cmul(cxq(i), vx) + cmul(cyq(i), vy));
}

// RELAX: tau or tau_g differs from 1.  Without it omega = 1, the (1 - omega) lambda terms vanish and
// tau F / rho is F / rho, and those operations are not issued.
template <class S, class C, bool SHIFT, bool RELAX, int TX, int TY, int BY, int MINB>
__global__ void __launch_bounds__(TX * BY, MINB)
lb_adj1_kernel(const S* __restrict__ fin, const S* __restrict__ lam_out, S* __restrict__ lam_in,
               S* __restrict__ lamF, const KParams<C> kp, const C cJ, const C nuc, const double mirror_coef,
               double* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileSmem<C, TX, TY, false>*>(smem_raw);
  constexpr int NT = TX * BY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  tile_phase_a<S, C, SHIFT, false, TX, TY, NT, false>(fin, kp, x0, y0, sm, tid);
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  const C om = RELAX ? kp.inv_tau : C(1), omg = RELAX ? kp.inv_tau_g : C(1), tau = RELAX ? kp.tau : C(1);
  const C Tb = SHIFT ? kp.T_bar : C(0);
  double dtd = 0.0;
#pragma unroll 1
  for (int k = 0; k < TY / BY; ++k) {
    const int tx = threadIdx.x, ty = threadIdx.y + k * BY;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= nx || gy >= ny) continue;
    const int cx = tx + 2, cy = ty + 2;
    const int idx = gy * pitch + gx;
    if (sm.solid[cy][cx]) {
#pragma unroll
      for (int q = 0; q < 27; ++q) lam_in[q * plane + idx] = S(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) lamF[q * plane + idx] = S(0);
      continue;
    }
    // ---- forward quantities of S_t at the node
    C T = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) T += C(fin[(18 + i) * plane + idx]);
    T += Tb;
    const C r1 = sm.rho[cy][cx].x + (SHIFT ? kp.rho_bar[0] : C(0));
    const C r2 = sm.rho[cy][cx].y + (SHIFT ? kp.rho_bar[1] : C(0));
    const C jx = sm.jx[ty][tx], jy = sm.jy[ty][tx];
    lamF[4 * plane + idx] = S(r1);  // the densities, for adj2's transposed stencils
    lamF[5 * plane + idx] = S(r2);
    C Fx[2], Fy[2], crx[2], cry[2], sx[2], sy[2], psl[2];
    node_force_parts<C>(sm, kp, cx, cy, r1, r2, T, Fx, Fy, crx, cry, sx, sy, psl);
    const C rho = r1 + r2;
    C ir[2], irho;
    three_reciprocals<C>(r1, r2, ir[0], ir[1], irho);
    const C rl2[2] = {r1, r2};
    const C ux = jx * irho, uy = jy * irho;
    const C Fxt = Fx[0] + Fx[1], Fyt = Fy[0] + Fy[1];
    const C uHx = ux + C(0.5) * Fxt * irho, uHy = uy + C(0.5) * Fyt * irho;

    // ---- adjoint of the streaming (transposed push, bounce-back and anti-bounce-back)
    C ls[27];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      if (lam_out == nullptr) {
        ls[i] = ls[9 + i] = ls[18 + i] = C(0);
      } else if (!sm.solid[cy + cyq(i)][cx + cxq(i)]) {
        int dx = gx + cxq(i);
        dx = dx < 0 ? dx + nx : (dx >= nx ? dx - nx : dx);
        int dy = gy + cyq(i);
        if (kp.periodic_y) dy = dy < 0 ? dy + ny : (dy >= ny ? dy - ny : dy);
        const int didx = dy * pitch + dx;
        ls[i] = C(lam_out[i * plane + didx]);
        ls[9 + i] = C(lam_out[(9 + i) * plane + didx]);
        ls[18 + i] = C(lam_out[(18 + i) * plane + didx]);
      } else {
        const int o = oppq(i);
        ls[i] = C(lam_out[o * plane + idx]);
        ls[9 + i] = C(lam_out[(9 + o) * plane + idx]);
        const C lg = C(lam_out[(18 + o) * plane + idx]);
        ls[18 + i] = -lg;
        if (2 * (gy + cyq(i)) < ny) dtd += 2.0 * (double)wq<C>(i) * (double)lg;  // d(2 w_i T_w)/dT_down
      }
    }

    // ---- adjoint of the BGK collisions (Eq. BGK with f^eq(rho_l, u_l); Eq. LBMg with g^eq(T, u^(H)))
    C lin[27];
    C lux = C(0), luy = C(0), lrho[2] = {C(0), C(0)}, lFx[2] = {C(0), C(0)}, lFy[2] = {C(0), C(0)}, lT = C(0);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const C ulx = ux + tau * Fx[l] * ir[l], uly = uy + tau * Fy[l] * ir[l];
      const C uu = ulx * ulx + uly * uly;
      C lulx = C(0), luly = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C lsv = ls[9 * l + i];
        lin[9 * l + i] = RELAX ? (C(1) - om) * lsv : C(0);
        const C lfeq = om * lsv * wq<C>(i);
        const C cu = cdot<C>(i, ulx, uly);
        lrho[l] += lfeq * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
        const C g = lfeq * rl2[l];
        lulx += g * (cxq(i) == 0 ? -(C(3) * ulx) : C(3 * cxq(i)) + C(9) * cu * C(cxq(i)) - C(3) * ulx);
        luly += g * (cyq(i) == 0 ? -(C(3) * uly) : C(3 * cyq(i)) + C(9) * cu * C(cyq(i)) - C(3) * uly);
      }
      // u_l = u + tau F_l / rho_l (Eq. shift)
      lux += lulx;
      luy += luly;
      lFx[l] += tau * lulx * ir[l];
      lFy[l] += tau * luly * ir[l];
      lrho[l] -= tau * (Fx[l] * lulx + Fy[l] * luly) * ir[l] * ir[l];
    }
    C luHx = C(0), luHy = C(0);
    {
      const C uu = uHx * uHx + uHy * uHy;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C lsv = ls[18 + i];
        lin[18 + i] = RELAX ? (C(1) - omg) * lsv : C(0);
        const C lgeq = omg * lsv * wq<C>(i);
        const C cu = cdot<C>(i, uHx, uHy);
        lT += lgeq * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
        const C g = lgeq * T;
        luHx += g * (cxq(i) == 0 ? -(C(3) * uHx) : C(3 * cxq(i)) + C(9) * cu * C(cxq(i)) - C(3) * uHx);
        luHy += g * (cyq(i) == 0 ? -(C(3) * uHy) : C(3 * cyq(i)) + C(9) * cu * C(cyq(i)) - C(3) * uHy);
      }
    }
    // ---- Nu seed: cJ d(<u^(H)_y T> / (kappa dT / H))/dS; the mirror-rule gradient term only moves
    //      dJ/dT_down (it telescopes to the wall temperatures)
    if (cJ != C(0)) {
      luHy += cJ * T * nuc;
      lT += cJ * uHy * nuc;
      const int up = (sm.solid[cy + 1][cx] && 2 * (gy + 1) < ny) ? 1 : 0;
      const int dn = (sm.solid[cy - 1][cx] && 2 * (gy - 1) < ny) ? 1 : 0;
      if (up != dn) dtd += (double)cJ * mirror_coef * (double)(up - dn);  // zero away from the walls
    }
    // u^(H) = u + F / (2 rho)
    lux += luHx;
    luy += luHy;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      lFx[l] += C(0.5) * luHx * irho;
      lFy[l] += C(0.5) * luHy * irho;
      lrho[l] -= C(0.5) * (Fxt * luHx + Fyt * luHy) * irho * irho;
    }
    // u = j / rho (Eq. velo)
    const C ljx = lux * irho, ljy = luy * irho;
#pragma unroll
    for (int l = 0; l < 2; ++l) lrho[l] -= (jx * lux + jy * luy) * irho * irho;
    // external force rho_l (body_fx, alpha_g T) (Eq. alphaG)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      lrho[l] += lFx[l] * kp.body_fx + lFy[l] * kp.alpha_g * T;
      lT += lFy[l] * kp.alpha_g * rl2[l];
    }
    // local parts of the force adjoint: the factor rho_l(x) of Eq. FAB and psi_l(x) of the self force
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      lrho[l] -= kp.gx * (crx[l] * lFx[l] + cry[l] * lFy[l]);
      const C lpsi = -(sx[l] * lFx[l] + sy[l] * lFy[l]);
      lrho[l] += lpsi * (C(1) - psl[l] * kp.inv_rho0);  // dpsi/drho = exp(-rho/rho0) = 1 - psi/rho0
    }
    // adjoint of the moments rho_l = sum_i f_{l,i}, j = sum c_i f, T = sum_i g_i
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        C v = RELAX ? lin[9 * l + i] + lrho[l] : lrho[l];
        if (cxq(i) != 0) v = v + cmul(cxq(i), ljx);
        if (cyq(i) != 0) v = v + cmul(cyq(i), ljy);
        lam_in[(9 * l + i) * plane + idx] = S(v);
      }
#pragma unroll
    for (int i = 0; i < 9; ++i) lam_in[(18 + i) * plane + idx] = S(RELAX ? lin[18 + i] + lT : lT);
    lamF[0 * plane + idx] = S(lFx[0]);
    lamF[1 * plane + idx] = S(lFy[0]);
    lamF[2 * plane + idx] = S(lFx[1]);
    lamF[3 * plane + idx] = S(lFy[1]);
  }
  // per-block dJ/dT_down, added to this block's running total (one writer per slot, stream order);
  // only blocks next to a wall have a nonzero share
  if (!__syncthreads_or(dtd != 0.0)) return;
  __shared__ double s_red[NT / 32];
  const double v = warp_sum(dtd);
  if ((tid & 31) == 0) s_red[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += s_red[w];
    acc[blockIdx.y * gridDim.x + blockIdx.x] += t;
  }
}

template <class C, int TX, int TY> struct Adj2Smem {
  static constexpr int RX = TX + 4, RY = TY + 4;
  C vt[2][2][RY][RX];  // rho_l lam_F_l (x, y): the cross force transposed
  C ve[2][2][RY][RX];  // psi_l lam_F_l (x, y): the self force transposed
  C psi[2][TY][TX];    // psi_l at the tile's own nodes
  unsigned char solid[TY][TX];
};

template <class S, class C, bool SHIFT, int TX, int TY, int BY, int MINB>
__global__ void __launch_bounds__(TX * BY, MINB)
lb_adj2_kernel(const S* __restrict__ lamF, S* __restrict__ lam_in, const KParams<C> kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<Adj2Smem<C, TX, TY>*>(smem_raw);
  constexpr int RX = TX + 4, RY = TY + 4, NT = TX * BY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  // Ring positions of this thread: all their loads are issued before any of them is used.
  constexpr int NR = (RX * RY + NT - 1) / NT;
  C val[NR][6];
  bool fluid[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int r = tid + q * NT;
    fluid[q] = false;
    if (r >= RX * RY) continue;
    const int ry = r / RX, rx = r - ry * RX;
    const int gx = wrap_any(x0 + rx - 2, nx);
    int gy = y0 + ry - 2;
    bool solid;
    if (kp.periodic_y) {
      gy = wrap_any(gy, ny);
      solid = kp.mask != nullptr && kp.mask[gy * nx + gx] != 0;
    } else {
      solid = (gy <= 0 || gy >= ny - 1) || (kp.mask != nullptr && kp.mask[gy * nx + gx] != 0);
    }
    if (solid) continue;
    fluid[q] = true;
    const int idx = gy * pitch + gx;
    // lam_F (x, y) of both components, then the densities written by adj1
#pragma unroll
    for (int v = 0; v < 6; ++v) val[q][v] = C(lamF[v * plane + idx]);
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int r = tid + q * NT;
    if (r >= RX * RY) continue;
    const int ry = r / RX, rx = r - ry * RX;
    const bool own = rx >= 2 && rx < TX + 2 && ry >= 2 && ry < TY + 2;
    if (!fluid[q]) {
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int d = 0; d < 2; ++d) sm.vt[l][d][ry][rx] = sm.ve[l][d][ry][rx] = C(0);
      if (own) sm.solid[ry - 2][rx - 2] = 1;
      continue;
    }
    const C rr[2] = {val[q][4], val[q][5]};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const C ps = psi_exp<C>(rr[l], kp.rho0, kp.inv_rho0);
      const C fx = val[q][2 * l], fy = val[q][2 * l + 1];
      sm.vt[l][0][ry][rx] = rr[l] * fx;
      sm.vt[l][1][ry][rx] = rr[l] * fy;
      sm.ve[l][0][ry][rx] = ps * fx;
      sm.ve[l][1][ry][rx] = ps * fy;
      if (own) sm.psi[l][ry - 2][rx - 2] = ps;
    }
    if (own) sm.solid[ry - 2][rx - 2] = 0;
  }
  __syncthreads();
#pragma unroll 1
  for (int k = 0; k < TY / BY; ++k) {
    const int tx = threadIdx.x, ty = threadIdx.y + k * BY;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= nx || gy >= ny || sm.solid[ty][tx]) continue;
    const int cx = tx + 2, cy = ty + 2;
    C lrho[2] = {C(0), C(0)};
    // sum over links k of a_k c_k . v(y - c_k) = sum over half-links h of a_h c_h . (v(y - c_h) - v(y + c_h))
#define TLB_DX(A, l, dx, dy) (sm.A[l][0][cy - (dy)][cx - (dx)] - sm.A[l][0][cy + (dy)][cx + (dx)])
#define TLB_DY(A, l, dx, dy) (sm.A[l][1][cy - (dy)][cx - (dx)] - sm.A[l][1][cy + (dy)][cx + (dx)])
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int l = 1 - m;  // Eq. FAB of component l reads rho_m at the neighbours
      const C w1 = C(1) / C(9), w2 = C(1) / C(36);
      const C G = w1 * (TLB_DX(vt, l, 1, 0) + TLB_DY(vt, l, 0, 1)) +
                  w2 * (TLB_DX(vt, l, 1, 1) + TLB_DY(vt, l, 1, 1) - TLB_DX(vt, l, -1, 1) + TLB_DY(vt, l, -1, 1));
      lrho[m] -= kp.gx * G;
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const C Gs = kp.a1[l] * (TLB_DX(ve, l, 1, 0) + TLB_DY(ve, l, 0, 1)) +
                   kp.a2[l] * (TLB_DX(ve, l, 1, 1) + TLB_DY(ve, l, 1, 1) - TLB_DX(ve, l, -1, 1) + TLB_DY(ve, l, -1, 1)) +
                   kp.a4x2[l] * (TLB_DX(ve, l, 2, 0) + TLB_DY(ve, l, 0, 2)) +
                   kp.a5[l] * (TLB_DX(ve, l, 1, 2) + C(2) * TLB_DY(ve, l, 1, 2) - TLB_DX(ve, l, -1, 2) +
                               C(2) * TLB_DY(ve, l, -1, 2) + C(2) * TLB_DX(ve, l, 2, 1) + TLB_DY(ve, l, 2, 1) -
                               C(2) * TLB_DX(ve, l, -2, 1) + TLB_DY(ve, l, -2, 1)) +
                   kp.a8x2[l] * (TLB_DX(ve, l, 2, 2) + TLB_DY(ve, l, 2, 2) - TLB_DX(ve, l, -2, 2) + TLB_DY(ve, l, -2, 2));
      lrho[l] -= Gs * (C(1) - sm.psi[l][ty][tx] * kp.inv_rho0);
    }
#undef TLB_DX
#undef TLB_DY
    const int idx = gy * pitch + gx;
    // all 18 loads before the stores: through one pointer with a run-time plane stride the compiler
    // cannot tell the entries apart, and a load after a store would wait for it
    C v[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) v[q] = C(lam_in[q * plane + idx]);
#pragma unroll
    for (int q = 0; q < 18; ++q) lam_in[q * plane + idx] = S(v[q] + lrho[q / 9]);
  }
}

// dJ/dT0 = sum_i w_i lam_0[g_i] at fluid nodes (S_0 has g_i = w_i T0), into nx*ny doubles.
template <class S>
__global__ void lb_adj_dT0_kernel(const S* __restrict__ lam, double* __restrict__ out, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  double s = 0.0;
  for (int i = 0; i < 9; ++i) s += wq<double>(i) * (double)lam[(18 + i) * cfg.plane + (long long)gy * cfg.pitch + gx];
  out[n] = solid ? 0.0 : s;
}

// J = mean of Nu over the N post-step observables; dJ/dT_down = sum of the per-block totals
// - J / dT (Nu depends on T_down through the normalisation kappa dT / H).
// Nu(S_t) of Eq. NuTime for the forward steps t = 1 .. n - 1 from the u^(H)_y T partials of the step out
// of S_t (nb per step, summed in CTA order): Nu = nuc (U - kappa D) with D the mirror-rule sum of dT/dy,
// which telescopes to the wall temperatures (the same for every state).  Slot t - 1 of nu, as the
// observables pass would fill it.
__global__ void lb_adj_nu_kernel(const double* __restrict__ part, int nb, int n, double nuc, double mirror_D,
                                 double* __restrict__ nu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (t >= n) return;
  const double* p = part + (long long)t * nb;
  double U = 0.0;
  for (int b = 0; b < nb; ++b) U += p[b];
  nu[(long long)(t - 1) * kObsOut + 4] = nuc * U + mirror_D;
}

__global__ void lb_adj_final_kernel(const double* __restrict__ nu, int n_steps, const double* __restrict__ acc,
                                    int n_blocks, double inv_dT, double* __restrict__ out) {
  __shared__ double s_a[256], s_b[256];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < n_steps; t += 256) a += nu[(long long)t * kObsOut + 4];
  for (int k = threadIdx.x; k < n_blocks; k += 256) b += acc[k];
  s_a[threadIdx.x] = a;
  s_b[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < 256; ++k) {
      ta += s_a[k];
      tb += s_b[k];
    }
    const double J = ta / (double)n_steps;
    out[0] = J;
    out[1] = tb - J * inv_dT;
  }
}

template <class S, bool SHIFT>
cudaError_t adj_step_impl(const StepCfg& c, const void* S_t, const void* lam_out, void* lam_in, void* lamF, double cJ,
                          double nuc, double mirror_coef, double* acc, cudaStream_t s) {
  using T = AdjTile<S>;
  const dim3 grid = grid_for(c.nx, c.ny, T::TX, T::TY), block(T::TX, T::BY, 1);
  const KParams<S> kp = make_kparams<S>(c);
  auto k1r = lb_adj1_kernel<S, S, SHIFT, true, T::TX, T::TY, T::BY, T::MINB>;
  auto k1s = lb_adj1_kernel<S, S, SHIFT, false, T::TX, T::TY, T::BY, T::MINB>;
  auto k1 = (kp.tau_is_one && kp.tau_g_is_one) ? k1s : k1r;
  auto k2 = lb_adj2_kernel<S, S, SHIFT, T::TX, T::TY, T::BY, T::MINB>;
  constexpr size_t b1 = sizeof(TileSmem<S, T::TX, T::TY, false>), b2 = sizeof(Adj2Smem<S, T::TX, T::TY>);
  static std::atomic<unsigned long long> done{0};  // shared-memory opt-in set once per device ordinal (mod 64)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    e = cudaFuncSetAttribute(k1r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit);
  }
  k1<<<grid, block, b1, s>>>(static_cast<const S*>(S_t), static_cast<const S*>(lam_out), static_cast<S*>(lam_in),
                             static_cast<S*>(lamF), kp, S(cJ), S(nuc), mirror_coef, acc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k2<<<grid, block, b2, s>>>(static_cast<const S*>(lamF), static_cast<S*>(lam_in), kp);
  return cudaGetLastError();
}

}  // namespace tlb

namespace {

struct AdjLayout {
  size_t state = 0, lam = 0, lamF = 0, acc = 0, nu = 0, nup = 0, red = 0, dT0 = 0, ckpt = 0, seg = 0, total = 0;
  int n_ckpt = 0, n_blocks = 0, nu_blocks = 0;
};

int adj_blocks(const lb_params& p) {
  return p.precision == LB_FP64 ? (int)(grid_for(p.nx, p.ny, AdjTile<double>::TX, AdjTile<double>::TY).x *
                                        grid_for(p.nx, p.ny, AdjTile<double>::TX, AdjTile<double>::TY).y)
                                : (int)(grid_for(p.nx, p.ny, AdjTile<float>::TX, AdjTile<float>::TY).x *
                                        grid_for(p.nx, p.ny, AdjTile<float>::TX, AdjTile<float>::TY).y);
}

AdjLayout adj_layout(const lb_handle* h, int n_steps, int ckpt_every) {
  AdjLayout A;
  const size_t plane = (size_t)h->L.pitch * h->p.ny;
  const size_t st = round_up(27 * plane * h->L.elem, kAlign);
  A.n_ckpt = (n_steps + ckpt_every - 1) / ckpt_every;
  A.n_blocks = adj_blocks(h->p);
  size_t off = 0;
  A.lam = off;
  off += 2 * st;
  A.lamF = off;
  off += round_up(6 * plane * h->L.elem, kAlign);
  A.acc = off;
  off += round_up((size_t)A.n_blocks * sizeof(double), kAlign);
  A.red = off;
  off += kAlign;
  A.nu = off;
  off += round_up((size_t)(n_steps + 1) * kObsOut * sizeof(double), kAlign);
  A.nu_blocks = step_nu_blocks(h->p.precision, h->p.nx, h->p.ny);
  A.nup = off;  // per forward step: the u^(H)_y T partial sums of its input state, one per CTA
  off += round_up((size_t)n_steps * A.nu_blocks * sizeof(double), kAlign);
  A.dT0 = off;
  off += round_up((size_t)h->p.nx * h->p.ny * sizeof(double), kAlign);
  A.ckpt = off;
  off += (size_t)A.n_ckpt * st;
  A.seg = off;
  off += (size_t)(ckpt_every + 1) * st;
  A.state = st;
  A.total = off;
  return A;
}

// Milliseconds of the phases of the last lb_adjoint call on this thread: forward pass (steps and
// Nu), segment recomputation, reverse sweep (adjoint steps), number of adjoint steps.
thread_local double g_adj_timing[4] = {0.0, 0.0, 0.0, 0.0};

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  double ms() const {
    float v = 0.0f;
    cudaEventElapsedTime(&v, a, b);
    return (double)v;
  }
};

int afail(lb_handle* h, int code, const char* msg, cudaError_t e = cudaSuccess) {
  std::snprintf(h->err, sizeof h->err, "%s%s%s", msg, e != cudaSuccess ? ": " : "",
                e != cudaSuccess ? cudaGetErrorString(e) : "");
  return code;
}

cudaError_t adj_step(const lb_handle* h, const void* S_t, const void* lam_out, void* lam_in, void* lamF, double cJ,
                     double nuc, double mirror_coef, double* acc) {
  return h->p.precision == LB_FP64
             ? adj_step_impl<double, false>(h->cfg, S_t, lam_out, lam_in, lamF, cJ, nuc, mirror_coef, acc, h->stream)
             : adj_step_impl<float, true>(h->cfg, S_t, lam_out, lam_in, lamF, cJ, nuc, mirror_coef, acc, h->stream);
}

cudaError_t fwd_step(const lb_handle* h, const void* in, void* out) {
  return h->p.precision == LB_FP64 ? launch_step_tile_f64(h->tile, h->cfg, in, out, h->stream)
                                   : launch_step_tile_f32(h->tile, h->cfg, in, out, h->stream);
}

cudaError_t fwd_step_nu(const lb_handle* h, const void* in, void* out, double* partials) {
  return h->p.precision == LB_FP64 ? launch_step_nu_f64(h->cfg, in, out, partials, h->stream)
                                   : launch_step_nu_f32(h->cfg, in, out, partials, h->stream);
}

cudaError_t obs_into(const lb_handle* h, const void* state, double* out16) {
  double* part = reinterpret_cast<double*>(h->ws + h->L.part_off);
  cudaError_t e = h->p.precision == LB_FP64 ? launch_f64(MODE_OBS, h->cfg, state, nullptr, part, h->stream)
                                            : launch_f32(MODE_OBS, h->cfg, state, nullptr, part, h->stream);
  if (e != cudaSuccess) return e;
  return obs_finalize(h->cfg, part, h->L.n_blocks, out16, h->stream);
}

// d Nu / d(sum u_y T) = 1 / (N_fluid kappa dT / H), and the coefficient of the mirror count
// (-kappa times that); both 0 when Nu is not defined (periodic y or dT = 0).
int nu_coefs(lb_handle* h, const void* state, double* scratch16, double* nuc, double* mirror, double* dsum = nullptr) {
  cudaError_t e = obs_into(h, state, scratch16);
  double v[kObsOut];
  if (e == cudaSuccess) e = cudaMemcpyAsync(v, scratch16, sizeof v, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return afail(h, LB_ECUDA, "observables for the adjoint", e);
  const double nf = v[7], dT = h->p.T_down - h->p.T_up, kappa = h->cfg.kappa;
  if (dsum) *dsum = v[9];
  if (h->p.periodic_y || dT == 0.0 || nf <= 0.0) {
    *nuc = *mirror = 0.0;
  } else {
    *nuc = 1.0 / (nf * kappa * dT / h->cfg.H);
    *mirror = -kappa * *nuc;
  }
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_state_layout(const lb_handle* h, int* pitch, size_t* plane_elems, int* elem_bytes) {
  if (!h || h->p.precision == LB_FP32_FP16T) return LB_EINVAL;
  if (pitch) *pitch = h->L.pitch;
  if (plane_elems) *plane_elems = (size_t)h->L.pitch * h->p.ny;
  if (elem_bytes) *elem_bytes = (int)h->L.elem;
  return LB_OK;
}

int lb_adjoint_workspace_size(const lb_handle* h, int n_steps, int ckpt_every, size_t* bytes) {
  if (!h || !bytes || n_steps < 1 || ckpt_every < 1 || h->p.precision == LB_FP32_FP16T || h->p.precision == LB_DF64)
    return LB_EINVAL;
  *bytes = adj_layout(h, n_steps, ckpt_every).total;
  return LB_OK;
}

int lb_adjoint_step(lb_handle* h, const void* d_lam_next, void* d_lam, double cJ, void* d_adj_ws, size_t adj_bytes,
                    double* dJ_dTdown) {
  if (!h || !d_lam || !d_adj_ws) return LB_EINVAL;
  if (h->p.precision == LB_FP32_FP16T || h->p.precision == LB_DF64)
    return afail(h, LB_EINVAL, "the adjoint needs LB_FP64 or LB_FP32_SHIFTED");
  if (h->cfg.u_wall[0] != 0.0 || h->cfg.u_wall[1] != 0.0) return afail(h, LB_EINVAL, "the adjoint needs resting walls");
  const AdjLayout A = adj_layout(h, 1, 1);
  if (adj_bytes < A.total || ((uintptr_t)d_adj_ws % kAlign) != 0) return afail(h, LB_ENOSPACE, "adjoint workspace too small");
  unsigned char* ws = static_cast<unsigned char*>(d_adj_ws);
  double* acc = reinterpret_cast<double*>(ws + A.acc);
  double* red = reinterpret_cast<double*>(ws + A.red);
  double nuc = 0.0, mirror = 0.0;
  if (int rc = nu_coefs(h, h->buf[h->cur], red, &nuc, &mirror)) return rc;
  cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)A.n_blocks * sizeof(double), h->stream);
  if (e == cudaSuccess) e = adj_step(h, h->buf[h->cur], d_lam_next, d_lam, ws + A.lamF, cJ, nuc, mirror, acc);
  std::vector<double> a(A.n_blocks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a.data(), acc, a.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return afail(h, LB_ECUDA, "lb_adjoint_step", e);
  if (dJ_dTdown) {
    double s = 0.0;
    for (double v : a) s += v;
    // the Nu normalisation term -cJ Nu / dT
    if (cJ != 0.0 && nuc != 0.0) {
      double v[kObsOut];
      if (cudaMemcpy(v, red, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return afail(h, LB_ECUDA, "copy");
      s -= cJ * v[4] / (h->p.T_down - h->p.T_up);
    }
    *dJ_dTdown = s;
  }
  return LB_OK;
}

int lb_adjoint(lb_handle* h, int n_steps, int ckpt_every, void* d_adj_ws, size_t adj_bytes, double* J, double* dJ_dT0,
               double* dJ_dTdown) {
  if (!h || n_steps < 1 || ckpt_every < 1 || !d_adj_ws || !J) return LB_EINVAL;
  if (h->p.precision == LB_FP32_FP16T || h->p.precision == LB_DF64)
    return afail(h, LB_EINVAL, "the adjoint needs LB_FP64 or LB_FP32_SHIFTED");
  if (h->cfg.u_wall[0] != 0.0 || h->cfg.u_wall[1] != 0.0) return afail(h, LB_EINVAL, "the adjoint needs resting walls");
  const AdjLayout A = adj_layout(h, n_steps, ckpt_every);
  if (adj_bytes < A.total || ((uintptr_t)d_adj_ws % kAlign) != 0) return afail(h, LB_ENOSPACE, "adjoint workspace too small");
  unsigned char* ws = static_cast<unsigned char*>(d_adj_ws);
  double* nu = reinterpret_cast<double*>(ws + A.nu);
  double* acc = reinterpret_cast<double*>(ws + A.acc);
  double* red = reinterpret_cast<double*>(ws + A.red);
  auto ckpt = [&](int k) { return ws + A.ckpt + (size_t)k * A.state; };
  auto seg = [&](int j) { return ws + A.seg + (size_t)j * A.state; };
  const size_t sbytes = (size_t)27 * h->L.pitch * h->p.ny * h->L.elem;
  double nuc = 0.0, mirror = 0.0, dsum = 0.0;
  if (int rc = nu_coefs(h, h->buf[h->cur], red, &nuc, &mirror, &dsum)) return rc;
  cudaStream_t s = h->stream;
  double* nup = reinterpret_cast<double*>(ws + A.nup);
  EventPair t_fwd;
  std::vector<EventPair> t_rec(A.n_ckpt), t_rev(A.n_ckpt);
  // forward pass, a checkpoint every ckpt_every steps: each step also sums u^(H)_y T of its input state,
  // which gives Nu(S_1) .. Nu(S_{n-1}); Nu(S_n) comes from one observables pass at the end
  cudaEventRecord(t_fwd.a, s);
  cudaError_t e = cudaMemcpyAsync(ckpt(0), h->buf[h->cur], sbytes, cudaMemcpyDeviceToDevice, s);
  for (int t = 0; t < n_steps && e == cudaSuccess; ++t) {
    e = fwd_step_nu(h, h->buf[h->cur], h->buf[h->cur ^ 1], nup + (size_t)t * A.nu_blocks);
    h->cur ^= 1;
    h->step += 1;
    if (e == cudaSuccess && (t + 1) % ckpt_every == 0 && t + 1 < n_steps)
      e = cudaMemcpyAsync(ckpt((t + 1) / ckpt_every), h->buf[h->cur], sbytes, cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) e = obs_into(h, h->buf[h->cur], nu + (size_t)(n_steps - 1) * kObsOut);
  if (e == cudaSuccess && n_steps > 1) {
    lb_adj_nu_kernel<<<(n_steps + 127) / 128, 128, 0, s>>>(nup, A.nu_blocks, n_steps, nuc, mirror * dsum, nu);
    e = cudaGetLastError();
  }
  cudaEventRecord(t_fwd.b, s);
  if (e != cudaSuccess) return afail(h, LB_ECUDA, "adjoint forward pass", e);
  const double dT = h->p.T_down - h->p.T_up;
  const double inv_dT = nuc != 0.0 ? 1.0 / dT : 0.0;
  if (!dJ_dT0 && !dJ_dTdown) {
    e = cudaMemsetAsync(acc, 0, sizeof(double), s);
    if (e == cudaSuccess) lb_adj_final_kernel<<<1, 256, 0, s>>>(nu, n_steps, acc, 1, inv_dT, red), e = cudaGetLastError();
    double out[2];
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, red, sizeof out, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return afail(h, LB_ECUDA, "adjoint J", e);
    *J = out[0];
    return LB_OK;
  }
  // reverse sweep over the segments, last first
  unsigned char* lam[2] = {ws + A.lam, ws + A.lam + A.state};
  int cur = 0;
  bool have_lam = false;
  e = cudaMemsetAsync(acc, 0, (size_t)A.n_blocks * sizeof(double), s);
  const double inv_n = 1.0 / (double)n_steps;
  for (int k = A.n_ckpt - 1; k >= 0 && e == cudaSuccess; --k) {
    const int start = k * ckpt_every, end = (start + ckpt_every < n_steps) ? start + ckpt_every : n_steps;
    cudaEventRecord(t_rec[k].a, s);
    e = cudaMemcpyAsync(seg(0), ckpt(k), sbytes, cudaMemcpyDeviceToDevice, s);
    for (int j = 0; j < end - start && e == cudaSuccess; ++j) e = fwd_step(h, seg(j), seg(j + 1));
    cudaEventRecord(t_rec[k].b, s);
    const int t_hi = (k == A.n_ckpt - 1) ? end : end - 1;
    cudaEventRecord(t_rev[k].a, s);
    for (int t = t_hi; t >= start && e == cudaSuccess; --t) {
      const double cJ = t >= 1 ? inv_n : 0.0;
      e = adj_step(h, seg(t - start), have_lam ? lam[cur] : nullptr, lam[cur ^ 1], ws + A.lamF, cJ, nuc, mirror, acc);
      cur ^= 1;
      have_lam = true;
    }
    cudaEventRecord(t_rev[k].b, s);
  }
  if (e != cudaSuccess) return afail(h, LB_ECUDA, "adjoint reverse sweep", e);
  double* dT0 = reinterpret_cast<double*>(ws + A.dT0);
  if (h->p.precision == LB_FP64)
    lb_adj_dT0_kernel<double><<<rows_grid(h->cfg), 128, 0, s>>>(reinterpret_cast<const double*>(lam[cur]), dT0, h->cfg);
  else
    lb_adj_dT0_kernel<float><<<rows_grid(h->cfg), 128, 0, s>>>(reinterpret_cast<const float*>(lam[cur]), dT0, h->cfg);
  lb_adj_final_kernel<<<1, 256, 0, s>>>(nu, n_steps, acc, A.n_blocks, inv_dT, red);
  e = cudaGetLastError();
  double out[2];
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, red, sizeof out, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && dJ_dT0)
    e = cudaMemcpyAsync(dJ_dT0, dT0, (size_t)h->p.nx * h->p.ny * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return afail(h, LB_ECUDA, "adjoint gradient", e);
  *J = out[0];
  if (dJ_dTdown) *dJ_dTdown = out[1];
  g_adj_timing[0] = t_fwd.ms();
  g_adj_timing[1] = g_adj_timing[2] = 0.0;
  for (int k = 0; k < A.n_ckpt; ++k) {
    g_adj_timing[1] += t_rec[k].ms();
    g_adj_timing[2] += t_rev[k].ms();
  }
  g_adj_timing[3] = (double)(n_steps + 1);
  return LB_OK;
}

int lb_adjoint_timing(double* out4) {
  if (!out4) return LB_EINVAL;
  for (int k = 0; k < 4; ++k) out4[k] = g_adj_timing[k];
  return LB_OK;
}

}  // extern "C"
