// Total shear stress of the rheology experiment (TLBfind, arXiv 2109.12565,
// Sec. 2.1 text after Eq. NS, Sec. 3.2.1) on the GPU.
//
// At every fluid node
//   sigma_xy = eta_0 (d_x u^(H)_y + d_y u^(H)_x) - P^int_xy - P^F_xy,   eta_0 = rho (tau - 1/2) / 3
// (Eq. VISCO): the bare viscous stress of u^(H) by central differences (a solid neighbour takes the
// mirror value 2 u_w - u, u_w the x velocity of a flat wall row, 0 otherwise), the virial form of
// the interaction forces of Eqs. FAB, FintAttrattive, FintRepulsive (half of every pair term times
// c_ix c_iy), and the momentum flux the forcing of Eq. shift adds,
//   P^F_xy = tau^2 sum_l F_lx F_ly / rho_l - F_x F_y / (4 rho).
// The space average of sigma_xy over the fluid nodes is the paper's stress Sigma at one time; the
// x-wise average per row is its Pxy_av profile.
//
// Two passes, off the time-step path: the field mode of the step kernel writes rho_1, rho_2, T,
// u^(H) to the inactive buffer; then one CTA per 32 x 8 tile stages rho and psi of the tile and a
// 2-node ring in shared memory, recomputes the forces of both components with the step kernel's own
// stencil code (so the forces are the ones the step applies), adds the virial sums and the viscous
// term, and writes sigma_xy and per-row partial sums.  Row sums and totals follow in fixed order,
// so every result is independent of scheduling.  Everything here is FP64.
#include <cuda_runtime.h>

#include <cstdio>
#include <new>

#include "lb_cfg.h"
#include "lb_host.h"
#include "lb_kernels.cuh"
#include "tlb.h"

namespace tlb {
namespace {

constexpr int kSX = kStressTileX, kSY = 8;  // stress tile: one node per thread
constexpr int kRowVals = kStressRowVals;     // per row: sigma, viscous part, P^int, P^F, fluid count

struct StressSmem {
  double2 rho[kSY + 4][kSX + 4];  // (rho_1, rho_2), full densities (wall values at solid positions)
  double2 psi[kSY + 4][kSX + 4];  // exp pseudo-potentials
  unsigned char solid[kSY + 4][kSX + 4];
};

__device__ __forceinline__ bool solid_at(const StepCfg& c, int x, int y) {
  if (!c.periodic_y && (y <= 0 || y >= c.ny - 1)) return true;
  return c.mask != nullptr && c.mask[(long long)y * c.nx + x] != 0;
}

// x (comp 0) or y (comp 1) component of u^(H) at neighbour (xn, yn) of fluid node (x, y): the mirror
// value at a solid neighbour.
__device__ __forceinline__ double u_nb(const StepCfg& c, const double* __restrict__ u, int comp, double own, int xn,
                                       int yn) {
  xn = xn < 0 ? xn + c.nx : (xn >= c.nx ? xn - c.nx : xn);
  if (c.periodic_y) yn = yn < 0 ? yn + c.ny : (yn >= c.ny ? yn - c.ny : yn);
  if (solid_at(c, xn, yn)) {
    double uw = 0.0;
    if (comp == 0 && !c.periodic_y) uw = yn == 0 ? c.u_wall[0] : (yn == c.ny - 1 ? c.u_wall[1] : 0.0);
    return 2.0 * uw - own;
  }
  return u[(long long)yn * c.nx + xn];
}

// sum_i W_i v(x + c_i) c_ix c_iy over the links with c_ix c_iy != 0 of one component (lane) pair:
// diagonals (weight wd), the (2,1)-type links (w5) and the (2,2) links (w8).
__device__ __forceinline__ double2 virial_sum(const double2 (*v)[kSX + 4], int cx, int cy, double2 wd, double2 w5,
                                              double2 w8) {
  auto at = [&](int dx, int dy) { return v[cy + dy][cx + dx]; };
  auto comb = [](double2 a, double2 b, double2 c, double2 d) {  // a + b - c - d, lane-wise
    return make_double2((a.x + b.x) - (c.x + d.x), (a.y + b.y) - (c.y + d.y));
  };
  const double2 d1 = comb(at(1, 1), at(-1, -1), at(-1, 1), at(1, -1));
  const double2 d5a = comb(at(2, 1), at(-2, -1), at(-2, 1), at(2, -1));
  const double2 d5b = comb(at(1, 2), at(-1, -2), at(-1, 2), at(1, -2));
  const double2 d8 = comb(at(2, 2), at(-2, -2), at(-2, 2), at(2, -2));
  return make_double2(wd.x * d1.x + 2.0 * w5.x * (d5a.x + d5b.x) + 4.0 * w8.x * d8.x,
                      wd.y * d1.y + 2.0 * w5.y * (d5a.y + d5b.y) + 4.0 * w8.y * d8.y);
}

__global__ void __launch_bounds__(kSX * kSY)
lb_stress_kernel(const double* __restrict__ fields, double* __restrict__ sigma, double* __restrict__ part,
                 const StepCfg c, const KParams<double> kp) {
  __shared__ StressSmem sm;
  const int nx = c.nx, ny = c.ny;
  const long long N = (long long)nx * ny;
  const double* rho1 = fields;
  const double* rho2 = fields + N;
  const double* Tf = fields + 2 * N;
  const double* uxf = fields + 3 * N;
  const double* uyf = fields + 4 * N;
  const int x0 = blockIdx.x * kSX, y0 = blockIdx.y * kSY;
  const int tid = threadIdx.y * kSX + threadIdx.x;
  constexpr int RX = kSX + 4, RY = kSY + 4;
  for (int r = tid; r < RX * RY; r += kSX * kSY) {
    const int ry = r / RX, rx = r - ry * RX;
    int gx = x0 + rx - 2, gy = y0 + ry - 2;
    gx = ((gx % nx) + nx) % nx;
    bool s;
    if (c.periodic_y) {
      gy = ((gy % ny) + ny) % ny;
      s = solid_at(c, gx, gy);
    } else {
      s = gy < 0 || gy >= ny || solid_at(c, gx, gy);
    }
    if (s) {
      sm.rho[ry][rx] = make_double2(c.rho_w[0], c.rho_w[1]);
      sm.psi[ry][rx] = make_double2(c.psi_w[0], c.psi_w[1]);
    } else {
      const long long n = (long long)gy * nx + gx;
      const double a = rho1[n], b = rho2[n];
      sm.rho[ry][rx] = make_double2(a, b);
      sm.psi[ry][rx] = make_double2(c.rho0 * (1.0 - exp(-a * c.inv_rho0)), c.rho0 * (1.0 - exp(-b * c.inv_rho0)));
    }
    sm.solid[ry][rx] = s ? 1 : 0;
  }
  __syncthreads();

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx = x0 + tx, gy = y0 + ty;
  double v[kRowVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool in = gx < nx && gy < ny;
  if (in) {
    const long long n = (long long)gy * nx + gx;
    const int cx = tx + 2, cy = ty + 2;
    if (!sm.solid[cy][cx]) {
      const double2 r = sm.rho[cy][cx];
      const double rho = r.x + r.y;
      // forces of both components, as the step computes them (Eqs. FAB, FintAttrattive, FintRepulsive,
      // alphaG, constant x acceleration)
      double2 Fx, Fyp, crx, cry, sx, sy, psl;
      node_force_pair<double>(sm, kp, cx, cy, r, Fx, Fyp, crx, cry, sx, sy, psl);
      const double2 Fy = buoyant_fy<double>(kp, Fyp, r, Tf[n]);
      // P^int_xy: half of every pair term times c_x c_y; the cross force (w_i on the NN diagonals, psi~ =
      // rho / rho0) pairs component l here with the other component there
      const double2 vq = virial_sum(sm.rho, cx, cy, make_double2(1.0 / 36.0, 1.0 / 36.0), make_double2(0.0, 0.0),
                                    make_double2(0.0, 0.0));
      const double2 vs = virial_sum(sm.psi, cx, cy, make_double2(c.a2[0], c.a2[1]), make_double2(c.a5[0], c.a5[1]),
                                    make_double2(0.5 * c.a8x2[0], 0.5 * c.a8x2[1]));
      const double pint = 0.5 * (c.gx * (r.x * vq.y + r.y * vq.x) + (psl.x * vs.x + psl.y * vs.y));
      // P^F_xy: momentum flux of the velocity shift of Eq. shift
      const double t2 = c.tau * c.tau;
      const double FX = Fx.x + Fx.y, FY = Fy.x + Fy.y;
      const double pf = t2 * (Fx.x * Fy.x / r.x + Fx.y * Fy.y / r.y) - FX * FY / (4.0 * rho);
      // bare viscous stress, Eq. VISCO
      const double ux = uxf[n], uy = uyf[n];
      const double dvdx = 0.5 * (u_nb(c, uyf, 1, uy, gx + 1, gy) - u_nb(c, uyf, 1, uy, gx - 1, gy));
      const double dudy = 0.5 * (u_nb(c, uxf, 0, ux, gx, gy + 1) - u_nb(c, uxf, 0, ux, gx, gy - 1));
      const double visc = rho * (c.tau - 0.5) / 3.0 * (dvdx + dudy);
      const double s = visc - pint - pf;
      if (sigma) sigma[n] = s;
      v[0] = s;
      v[1] = visc;
      v[2] = pint;
      v[3] = pf;
      v[4] = 1.0;
    } else if (sigma) {
      sigma[n] = 0.0;
    }
  }
  // one warp = one tile row: a fixed shuffle tree, lane 0 writes the row's partial of this tile column
#pragma unroll
  for (int k = 0; k < kRowVals; ++k) {
    const double t = warp_sum(v[k]);
    if (tx == 0 && gy < ny) part[((long long)blockIdx.x * ny + gy) * kRowVals + k] = t;
  }
}

// Row sums over the tile columns in fixed order: rows[y * kRowVals + k].
__global__ void lb_stress_rows_kernel(const double* __restrict__ part, int ncol, int ny, double* __restrict__ rows) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= ny) return;
  double s[kRowVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < ncol; ++b)
#pragma unroll
    for (int k = 0; k < kRowVals; ++k) s[k] += part[((long long)b * ny + y) * kRowVals + k];
#pragma unroll
  for (int k = 0; k < kRowVals; ++k) rows[(long long)y * kRowVals + k] = s[k];
}

// Totals over the rows in fixed order (one CTA of 256 threads): tot[k].
__global__ void __launch_bounds__(256) lb_stress_total_kernel(const double* __restrict__ rows, int ny,
                                                              double* __restrict__ tot) {
  __shared__ double red[8][kRowVals];
  double s[kRowVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int y = threadIdx.x; y < ny; y += 256)
#pragma unroll
    for (int k = 0; k < kRowVals; ++k) s[k] += rows[(long long)y * kRowVals + k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRowVals; ++k) {
    const double t = warp_sum(s[k]);
    if (lane == 0) red[warp][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < kRowVals) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    tot[threadIdx.x] = t;
  }
}

}  // namespace

cudaError_t stress_run(const StepCfg& cfg_in, int precision, const void* cur, double* stage, cudaStream_t s,
                       double** d_rows, double** d_tot) {
  const int nx = cfg_in.nx, ny = cfg_in.ny;
  const size_t N = (size_t)nx * ny;
  cudaError_t e = launch_mode(precision, MODE_FIELDS, cfg_in, cur, nullptr, stage, s);
  if (e != cudaSuccess) return e;
  // the fields are full values: constants without storage shifts
  StepCfg c = cfg_in;
  c.rho_bar[0] = c.rho_bar[1] = c.T_bar = 0.0;
  const KParams<double> kp = make_kparams<double>(c);
  const int ncol = (nx + kSX - 1) / kSX;
  double* sigma = stage + 5 * N;
  double* part = stage + 6 * N;
  double* rows = part + (size_t)ncol * ny * kRowVals;
  double* tot = rows + (size_t)ny * kRowVals;
  lb_stress_kernel<<<dim3(ncol, (ny + kSY - 1) / kSY), dim3(kSX, kSY), 0, s>>>(stage, sigma, part, c, kp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lb_stress_rows_kernel<<<(ny + 127) / 128, 128, 0, s>>>(part, ncol, ny, rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lb_stress_total_kernel<<<1, 256, 0, s>>>(rows, ny, tot);
  e = cudaGetLastError();
  if (d_rows) *d_rows = rows;
  if (d_tot) *d_tot = tot;
  return e;
}

// Copy results of stress_run to the host: out4 = means, row = per-row means, field = sigma_xy.
cudaError_t stress_fetch(int nx, int ny, const double* stage, const double* d_rows, const double* d_tot, double* out4,
                         double* row, double* field, cudaStream_t s) {
  const size_t N = (size_t)nx * ny;
  double tot[kRowVals];
  cudaError_t e = cudaMemcpyAsync(tot, d_tot, sizeof tot, cudaMemcpyDeviceToHost, s);
  double* rows = nullptr;
  if (e == cudaSuccess && row) {
    rows = new (std::nothrow) double[(size_t)ny * kRowVals];
    if (!rows) return cudaErrorMemoryAllocation;
    e = cudaMemcpyAsync(rows, d_rows, (size_t)ny * kRowVals * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess && field) e = cudaMemcpyAsync(field, stage + 5 * N, N * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    const double nf = tot[4];
    for (int k = 0; k < 4; ++k)
      if (out4) out4[k] = nf > 0.0 ? tot[k] / nf : 0.0;
    if (row)
      for (int y = 0; y < ny; ++y) {
        const double cnt = rows[(size_t)y * kRowVals + 4];
        row[y] = cnt > 0.0 ? rows[(size_t)y * kRowVals] / cnt : 0.0;
      }
  }
  delete[] rows;
  return e;
}

}  // namespace tlb

using namespace tlb;

extern "C" int lb_stress(lb_handle* h, double* out4, double* row, double* field) {
  if (!h) return LB_EINVAL;
  if (!out4 && !row && !field) {
    std::snprintf(h->err, sizeof h->err, "lb_stress: no output requested");
    return LB_EINVAL;
  }
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);
  double *d_rows = nullptr, *d_tot = nullptr;
  cudaError_t e = stress_run(h->cfg, h->p.precision, h->buf[h->cur], stage, h->stream, &d_rows, &d_tot);
  if (e == cudaSuccess) e = stress_fetch(h->p.nx, h->p.ny, stage, d_rows, d_tot, out4, row, field, h->stream);
  if (e != cudaSuccess) {
    std::snprintf(h->err, sizeof h->err, "lb_stress: %s", cudaGetErrorString(e));
    return LB_ECUDA;
  }
  return LB_OK;
}
