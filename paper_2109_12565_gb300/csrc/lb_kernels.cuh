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
// A CTA whose tile and 1-node ring hold no solid node and need no periodic
// wrap takes a fast path: every store is an unconditional constant offset.
// Writes of direction i from a warp land on one contiguous row shifted by
// c_i; each destination slot has exactly one writer per step.
// Shared memory holds the two components of a node in one slot, and the hot
// arithmetic runs on lane pairs (components, opposite directions, or the two
// nodes of a phase-A pair): packed FP32x2 instructions in FP32, one FP64
// instruction per lane in FP64, each rounding once.
#pragma once
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "lb_cfg.h"

namespace tlb {

// D2Q9 links (Fig. 1a): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
__host__ __device__ constexpr int cxq(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cyq(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int oppq(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
// D2Q9 weights w_i (Fig. 1b).
template <class C> __host__ __device__ constexpr C wq(int i) { return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36)); }

// Storage forms.  S = double or float: all 27 planes in S, arithmetic in S.  S = F32H16: the 18
// fluid planes in FP32 and the 9 thermal planes in FP16 (both as deviations from the shift
// equilibria), arithmetic in FP32.  A buffer is the 18 fluid planes followed by the 9 thermal planes,
// each of `plane` elements of its own type.
struct F32H16 {};
// kFastPath: also instantiate the interior fast path of phase B (unconditional stores); a form whose
// arithmetic dominates (double-float) keeps one phase B, halving its code.
template <class S> struct Storage {
  using F = S;  // fluid planes
  using G = S;  // thermal planes
  using C = S;  // arithmetic
  static constexpr bool kFastPath = true;
};
template <> struct Storage<F32H16> {
  using F = float;
  using G = __half;
  using C = float;
  static constexpr bool kFastPath = true;
};
template <class S> using SF = typename Storage<S>::F;
template <class S> using SG = typename Storage<S>::G;
template <class S> using SC = typename Storage<S>::C;

// First thermal plane of a buffer.
template <class S> __host__ __device__ __forceinline__ const SG<S>* thermal_planes(const SF<S>* buf, long long plane) {
  return reinterpret_cast<const SG<S>*>(buf + 18 * plane);
}
template <class S> __host__ __device__ __forceinline__ SG<S>* thermal_planes(SF<S>* buf, long long plane) {
  return reinterpret_cast<SG<S>*>(buf + 18 * plane);
}
// Value conversions between storage and arithmetic (round to nearest into FP16).
template <class C, class T> __device__ __forceinline__ C up(T v) { return C(v); }
template <> __device__ __forceinline__ float up<float, __half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ double up<double, __half>(__half v) { return (double)__half2float(v); }
template <class T, class V> __device__ __forceinline__ T down(V v) { return T(v); }
template <> __device__ __forceinline__ __half down<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __half down<__half, double>(double v) { return __double2half(v); }

// Kernel constants in the compute precision C (rounded once on the host).
template <class C> struct KParams {
  int nx, ny, pitch, periodic_y;
  int plane;  // elements per population plane (27 * plane < 2^31 is checked on the host)
  const uint8_t* mask;
  C tau, inv_tau, inv_tau_g, rho0, inv_rho0, gx;
  C a1[2], a2[2], a4x2[2], a5[2], a8x2[2];
  C rho_w[2], psi_w[2];
  C drho_w[2];  // rho_w - rho_bar (shared memory holds density deviations)
  C T_down, T_up, alpha_g, body_fx;
  C rho_bar[2], T_bar;
  C twoTw_down, twoTw_up;  // 2 (T_w - T_bar) for the anti-bounce-back
  int tau_is_one;          // tau == 1: f* = f^eq exactly, the relaxation is skipped
  int tau_g_is_one;        // tau_g == 1: g* = g^eq
  double rho_w_d[2], T_down_d, T_up_d;  // field output at solid nodes
  C uw6[2];                // 6 u_wall of the bottom / top wall row (moving-wall bounce-back)
};

template <class C> inline KParams<C> make_kparams(const StepCfg& c) {
  KParams<C> k;
  k.nx = c.nx;
  k.ny = c.ny;
  k.pitch = c.pitch;
  k.periodic_y = c.periodic_y;
  k.plane = (int)c.plane;
  k.mask = c.mask;
  k.tau = C(c.tau);
  k.inv_tau = C(c.inv_tau);
  k.inv_tau_g = C(c.inv_tau_g);
  k.rho0 = C(c.rho0);
  k.inv_rho0 = C(c.inv_rho0);
  k.gx = C(c.gx);
  for (int l = 0; l < 2; ++l) {
    k.a1[l] = C(c.a1[l]);
    k.a2[l] = C(c.a2[l]);
    k.a4x2[l] = C(c.a4x2[l]);
    k.a5[l] = C(c.a5[l]);
    k.a8x2[l] = C(c.a8x2[l]);
    k.rho_w[l] = C(c.rho_w[l]);
    k.psi_w[l] = C(c.psi_w[l]);
    k.drho_w[l] = C(c.rho_w[l] - c.rho_bar[l]);
    k.rho_bar[l] = C(c.rho_bar[l]);
    k.rho_w_d[l] = c.rho_w[l];
  }
  k.T_down = C(c.T_down);
  k.T_up = C(c.T_up);
  k.alpha_g = C(c.alpha_g);
  k.body_fx = C(c.body_fx);
  k.T_bar = C(c.T_bar);
  k.twoTw_down = C(2.0 * (c.T_down - c.T_bar));
  k.twoTw_up = C(2.0 * (c.T_up - c.T_bar));
  k.tau_is_one = (c.tau == 1.0) ? 1 : 0;
  k.tau_g_is_one = (c.inv_tau_g == 1.0) ? 1 : 0;
  k.T_down_d = c.T_down;
  k.T_up_d = c.T_up;
  k.uw6[0] = C(6.0 * c.u_wall[0]);
  k.uw6[1] = C(6.0 * c.u_wall[1]);
  return k;
}

// Population load: the read-only path inside one step per launch, L2-coherent loads (ld.global.cg)
// when the same launch rewrites the buffers (persistent multi-step kernels).
template <bool CG, class S> __device__ __forceinline__ S ld_pop(const S* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// Where phase B reads the populations of its own node: straight from the input buffer.
template <class S, bool CG> struct GlobalPopSource {
  const SF<S>* __restrict__ fin;
  int plane;
  __device__ __forceinline__ SC<S> operator()(int k, int idx, int /*tx*/, int /*ty*/) const {
    if (k < 18) return up<SC<S>>(ld_pop<CG>(fin + idx + k * plane));
    return up<SC<S>>(ld_pop<CG>(thermal_planes<S>(fin, plane) + idx + (k - 18) * plane));
  }
};

__device__ __forceinline__ int wrap_any(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <class C> __device__ __forceinline__ C psi_exp(C rho, C rho0, C inv_rho0);
template <> __device__ __forceinline__ double psi_exp<double>(double rho, double rho0, double inv_rho0) {
  return rho0 * (1.0 - exp(-rho * inv_rho0));
}
template <> __device__ __forceinline__ float psi_exp<float>(float rho, float rho0, float inv_rho0) {
  return __fmaf_rn(-rho0, __expf(__fmul_rn(-rho, inv_rho0)), rho0);  // the same roundings as psi_exp2
}

// 1 / x: IEEE in FP64, the fast approximate division in FP32.
template <class C> __device__ __forceinline__ C recip(C x);
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float recip<float>(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// A value per fluid component, interleaved: one 8-byte (FP32) or 16-byte (FP64) shared-memory access
// reads both components of a node.
template <class C> struct V2T;
template <> struct V2T<float> { using type = float2; };
template <> struct V2T<double> { using type = double2; };
template <class C> using V2 = typename V2T<C>::type;
template <class C> __device__ __forceinline__ V2<C> v2(C a, C b) {
  V2<C> r;
  r.x = a;
  r.y = b;
  return r;
}
template <class C> __device__ __forceinline__ V2<C> splat(C a) { return v2<C>(a, a); }
template <class V> __device__ __forceinline__ V swap_lanes(const V& v) {
  V r;
  r.x = v.y;
  r.y = v.x;
  return r;
}

// psi of both components (lanes), one psi_exp per lane.
template <class C> __device__ __forceinline__ V2<C> psi_exp_pair(V2<C> rho, C rho0, C inv_rho0) {
  return v2<C>(psi_exp<C>(rho.x, rho0, inv_rho0), psi_exp<C>(rho.y, rho0, inv_rho0));
}

// Lane-wise arithmetic on pairs: one packed FP32x2 instruction in FP32, one instruction per lane in
// FP64.  Each operation rounds once to nearest, so every lane holds exactly the result of the scalar
// operation (a - b is the fused b * (-1) + a, exact up to its one rounding).
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) {
  return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
template <class V> __device__ __forceinline__ V p_sub(V a, V b) {
  return p_fma(b, splat<decltype(a.x)>(decltype(a.x)(-1)), a);
}
// The add of a running sum (p_sum9 / s_sum9 below).
template <class V> __device__ __forceinline__ V p_acc(V a, V b) { return p_add(a, b); }
// Scalar operations with one rounding each, never fused beyond what is written, so that every caller
// of the functions below computes the same bits.
__device__ __forceinline__ float s_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float s_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float s_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double s_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double s_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double s_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <class C> __device__ __forceinline__ C s_acc(C a, C b) { return s_add(a, b); }
// Sum of the nine populations of a density or of a node's thermal set, in a fixed order: for FP32 and
// FP64 the adds ((u[0] + u[1]) + u[2]) + ... + u[8]; a compound form may specialise it.
template <class V> struct Sum9 {
  __device__ __forceinline__ static V of(const V u[9]) {
    V d = u[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) d = p_acc(d, u[i]);
    return d;
  }
};
template <class V> __device__ __forceinline__ V p_sum9(const V u[9]) { return Sum9<V>::of(u); }
template <class C> struct SSum9 {
  __device__ __forceinline__ static C of(const C u[9]) {
    C d = u[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) d = s_acc(d, u[i]);
    return d;
  }
};
template <class C> __device__ __forceinline__ C s_sum9(const C u[9]) { return SSum9<C>::of(u); }

// The shared-memory form of a lane pair: the pair itself, unless a form keeps it in another order
// (converting on every load and store).
template <class C> struct SmemPairT { using type = V2<C>; };
template <class C> using SmemPair = typename SmemPairT<C>::type;

template <class C, int TX, int TY, bool NEED_T> struct alignas(16) TileSmem {
  static constexpr int RX = TX + 4, RY = TY + 4;
  SmemPair<C> rho[RY][RX];  // density deviations rho_l - rho_bar_l (rho_bar = 0 in FP64), components interleaved
  SmemPair<C> psi[RY][RX];
  C jx[TY][TX], jy[TY][TX];  // bare momentum of the tile's own nodes
  C T[NEED_T ? RY : 1][NEED_T ? RX : 1];
  unsigned char solid[RY][RX];
};

// Two-byte-aligned pair load of populations (8-byte vector load of two FP32 nodes).
template <bool CG> __device__ __forceinline__ float2 ld_pop2(const float2* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <class C, int TX, int TY, bool NEED_T>
__device__ __forceinline__ void phase_a_wall(TileSmem<C, TX, TY, NEED_T>& sm, const KParams<C>& kp, int rx, int ry) {
  sm.rho[ry][rx] = v2<C>(kp.drho_w[0], kp.drho_w[1]);
  sm.psi[ry][rx] = v2<C>(kp.psi_w[0], kp.psi_w[1]);
  sm.solid[ry][rx] = 1;
}

// Sums of one component's 9 populations for phase A: density deviation and the two momentum parts,
// in the order of phase_a_node.
template <class C> struct CompSums {
  C d, jx, jy;
};
template <class C> __device__ __forceinline__ CompSums<C> comp_sums(const C f[9]) {
  CompSums<C> r;
  r.d = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) r.d += f[i];
  r.jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  r.jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  return r;
}

// Lane-wise phase-A sums of one component over two nodes (lanes): density deviation and momentum,
// in the order of comp_sums (bit-identical per lane, up to the sign of an all-zero sum).
__device__ __forceinline__ void comp_sums2(const float2 u[9], float2& d, float2& jx, float2& jy) {
  d = u[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) d = p_add(d, u[i]);
  jx = p_add(p_sub(p_sub(p_add(p_sub(u[1], u[3]), u[5]), u[6]), u[7]), u[8]);
  jy = p_sub(p_sub(p_add(p_add(p_sub(u[2], u[4]), u[5]), u[6]), u[7]), u[8]);
}

// psi_exp<float> of two values (lanes), with the same roundings.
__device__ __forceinline__ float2 psi_exp2(float2 rho, float rho0, float inv_rho0) {
  const float2 x = p_mul(rho, splat<float>(-inv_rho0));
  return p_fma(splat<float>(-rho0), make_float2(__expf(x.x), __expf(x.y)), splat<float>(rho0));
}

// The store part of phase_a_node from the component sums (same values, same rounding).
template <class C, bool SHIFT, int TX, int TY, bool NEED_T>
__device__ __forceinline__ void phase_a_store(TileSmem<C, TX, TY, NEED_T>& sm, const KParams<C>& kp, int rx, int ry,
                                              const CompSums<C>& a, const CompSums<C>& b) {
  const C rb0 = SHIFT ? kp.rho_bar[0] : C(0), rb1 = SHIFT ? kp.rho_bar[1] : C(0);
  sm.rho[ry][rx] = v2<C>(a.d, b.d);
  sm.psi[ry][rx] = v2<C>(psi_exp<C>(a.d + rb0, kp.rho0, kp.inv_rho0), psi_exp<C>(b.d + rb1, kp.rho0, kp.inv_rho0));
  if (rx >= 2 && rx < TX + 2 && ry >= 2 && ry < TY + 2) {
    sm.jx[ry - 2][rx - 2] = a.jx + b.jx;
    sm.jy[ry - 2][rx - 2] = a.jy + b.jy;
  }
  sm.solid[ry][rx] = 0;
}

// Phase A of a step with FP32 fluid storage, two horizontally adjacent region nodes per thread: the
// pair's populations come in as 8-byte loads when both nodes are fluid, contiguous and 8-byte
// aligned (no periodic split between them), else node by node.  Component 1 is loaded and reduced
// before component 2, which keeps 18 values live.  Per node the same arithmetic as the one-node loop,
// so the results are bit-identical.
template <class S, class C, bool SHIFT, int TX, int TY, int NT, bool CG>
__device__ __forceinline__ int tile_phase_a_pairs(const SF<S>* __restrict__ fin, const KParams<C>& kp, int x0, int y0,
                                                  TileSmem<C, TX, TY, false>& sm, int tid) {
  constexpr int RX = TX + 4, RY = TY + 4, PX = RX / 2;
  static_assert(RX % 2 == 0, "pairs need an even region width");
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  const bool small_x = nx < TX + 4, small_y = ny < TY + 4;
  int ring_solid = 0;
  for (int r = tid; r < PX * RY; r += NT) {
    const int ry = r / PX, rx = 2 * (r - ry * PX);
    const int gxr = x0 + rx - 2;
    int gxa, gxb;
    if (small_x) {
      gxa = wrap_any(gxr, nx);
      gxb = wrap_any(gxr + 1, nx);
    } else {
      gxa = gxr < 0 ? gxr + nx : (gxr >= nx ? gxr - nx : gxr);
      const int t = gxr + 1;
      gxb = t < 0 ? t + nx : (t >= nx ? t - nx : t);
    }
    int gy = y0 + ry - 2;
    bool sa, sb;
    if (kp.periodic_y) {
      gy = small_y ? wrap_any(gy, ny) : (gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy));
      sa = kp.mask != nullptr && kp.mask[gy * nx + gxa] != 0;
      sb = kp.mask != nullptr && kp.mask[gy * nx + gxb] != 0;
    } else {
      const bool wall = gy <= 0 || gy >= ny - 1;
      sa = wall || (kp.mask != nullptr && kp.mask[gy * nx + gxa] != 0);
      sb = wall || (kp.mask != nullptr && kp.mask[gy * nx + gxb] != 0);
    }
    const bool ring_row = ry >= 1 && ry <= TY + 2;
    if (ring_row && ((sa && rx >= 1 && rx <= TX + 2) || (sb && rx + 1 >= 1 && rx + 1 <= TX + 2))) ring_solid = 1;
    CompSums<C> a1{}, a2{}, b1{}, b2{};
    if (!sa && !sb && gxb == gxa + 1 && (gxa & 1) == 0) {
      // pitch and plane are even, so the pair starts on an 8-byte boundary; lanes = (node a, node b)
      const float2* src = reinterpret_cast<const float2*>(fin + (gy * pitch + gxa));
      const int pl2 = plane >> 1;
      float2 d[2], jx[2], jy[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float2 u[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) u[i] = ld_pop2<CG>(src + (9 * c + i) * pl2);
        comp_sums2(u, d[c], jx[c], jy[c]);
      }
      const float2 p1 = psi_exp2(p_add(d[0], splat<float>(kp.rho_bar[0])), kp.rho0, kp.inv_rho0);
      const float2 p2 = psi_exp2(p_add(d[1], splat<float>(kp.rho_bar[1])), kp.rho0, kp.inv_rho0);
      // rho[ry][rx .. rx + 1] and psi[ry][rx .. rx + 1] are 16-byte aligned (RX and rx even)
      *reinterpret_cast<float4*>(&sm.rho[ry][rx]) = make_float4(d[0].x, d[1].x, d[0].y, d[1].y);
      *reinterpret_cast<float4*>(&sm.psi[ry][rx]) = make_float4(p1.x, p2.x, p1.y, p2.y);
      sm.solid[ry][rx] = 0;
      sm.solid[ry][rx + 1] = 0;
      if (rx >= 2 && rx < TX + 2 && ry >= 2 && ry < TY + 2) {
        *reinterpret_cast<float2*>(&sm.jx[ry - 2][rx - 2]) = p_add(jx[0], jx[1]);
        *reinterpret_cast<float2*>(&sm.jy[ry - 2][rx - 2]) = p_add(jy[0], jy[1]);
      }
      continue;
    } else {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (k == 0 ? sa : sb) continue;
        const SF<S>* src = fin + (gy * pitch + (k == 0 ? gxa : gxb));
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          C f[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) f[i] = C(ld_pop<CG>(src + (9 * c + i) * plane));
          (k == 0 ? (c == 0 ? a1 : a2) : (c == 0 ? b1 : b2)) = comp_sums<C>(f);
        }
      }
    }
    if (sa) phase_a_wall<C, TX, TY, false>(sm, kp, rx, ry);
    else phase_a_store<C, SHIFT, TX, TY, false>(sm, kp, rx, ry, a1, a2);
    if (sb) phase_a_wall<C, TX, TY, false>(sm, kp, rx + 1, ry);
    else phase_a_store<C, SHIFT, TX, TY, false>(sm, kp, rx + 1, ry, b1, b2);
  }
  return ring_solid;
}

// Phase A on one tile: rho, psi (and T for the observables) on the tile + 2-node ring.
// Returns (CTA-uniform) whether the fast path applies.
template <class S, class C, bool SHIFT, bool NEED_T, int TX, int TY, int NT, bool CG>
__device__ __forceinline__ bool tile_phase_a(const SF<S>* __restrict__ fin, const KParams<C>& kp, int x0, int y0,
                                             TileSmem<C, TX, TY, NEED_T>& sm, int tid) {
  constexpr int RX = TX + 4, RY = TY + 4;
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  const bool small_x = nx < TX + 4, small_y = ny < TY + 4;
  const C rb0 = SHIFT ? kp.rho_bar[0] : C(0), rb1 = SHIFT ? kp.rho_bar[1] : C(0);
  int ring_solid = 0;
  constexpr bool kPairs = !NEED_T && sizeof(SF<S>) == 4 && (RX % 2 == 0);
  if constexpr (kPairs) {
    ring_solid = tile_phase_a_pairs<S, C, SHIFT, TX, TY, NT, CG>(fin, kp, x0, y0, sm, tid);
  } else
  for (int r = tid; r < RX * RY; r += NT) {
    const int ry = r / RX, rx = r - ry * RX;
    int gx = x0 + rx - 2;
    if (small_x) gx = wrap_any(gx, nx);
    else gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    int gy = y0 + ry - 2;
    bool solid;
    if (kp.periodic_y) {
      if (small_y) gy = wrap_any(gy, ny);
      else gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      solid = kp.mask != nullptr && kp.mask[gy * nx + gx] != 0;
    } else {
      solid = (gy <= 0 || gy >= ny - 1) || (kp.mask != nullptr && kp.mask[gy * nx + gx] != 0);
    }
    if (solid && rx >= 1 && rx <= TX + 2 && ry >= 1 && ry <= TY + 2) ring_solid = 1;
    if (solid) {
      sm.rho[ry][rx] = v2<C>(kp.drho_w[0], kp.drho_w[1]);
      sm.psi[ry][rx] = v2<C>(kp.psi_w[0], kp.psi_w[1]);
      if constexpr (NEED_T) sm.T[ry][rx] = (2 * gy < ny) ? kp.T_down : kp.T_up;
      sm.solid[ry][rx] = 1;
    } else {
      const SF<S>* src = fin + (gy * pitch + gx);
      // lanes = the two components: each lane runs the sums of one component in the order written
      V2<C> u[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) u[i] = v2<C>(C(ld_pop<CG>(src + i * plane)), C(ld_pop<CG>(src + (9 + i) * plane)));
      const V2<C> d = p_sum9(u);
      sm.rho[ry][rx] = d;
      sm.psi[ry][rx] = psi_exp_pair<C>(p_add(d, v2<C>(rb0, rb1)), kp.rho0, kp.inv_rho0);
      if (rx >= 2 && rx < TX + 2 && ry >= 2 && ry < TY + 2) {
        const V2<C> jx = p_add(p_sub(p_sub(p_add(p_sub(u[1], u[3]), u[5]), u[6]), u[7]), u[8]);
        const V2<C> jy = p_sub(p_sub(p_add(p_add(p_sub(u[2], u[4]), u[5]), u[6]), u[7]), u[8]);
        sm.jx[ry - 2][rx - 2] = s_add(jx.x, jx.y);
        sm.jy[ry - 2][rx - 2] = s_add(jy.x, jy.y);
      }
      if constexpr (NEED_T) {
        C t = C(0);
        const SG<S>* tsrc = thermal_planes<S>(fin, plane) + (gy * pitch + gx);  // node offset in thermal elements
#pragma unroll
        for (int i = 0; i < 9; ++i) t += up<C>(ld_pop<CG>(tsrc + i * plane));
        sm.T[ry][rx] = t + (SHIFT ? kp.T_bar : C(0));
      }
      sm.solid[ry][rx] = 0;
    }
  }
  const int any = __syncthreads_or(ring_solid);
  const bool no_wrap_x = x0 >= 1 && x0 + TX + 1 <= nx;
  const bool no_wrap_y = !kp.periodic_y || (y0 >= 1 && y0 + TY + 1 <= ny);
  return !any && no_wrap_x && no_wrap_y;
}

// Stencil sums of one node, accumulated row pair by row pair (row 0, rows +-1, rows +-2), which keeps
// only two stencil rows live at a time.  Lane l holds component l (for q,
// the density of component l).  q: Eq. FAB's cross sums sum_NN w_i rho(x + c_i) c_i; s: the self
// sums sum_24 (G^a w_i + G^r p_i) psi_l(x + c_i) c_i of Eqs. FintAttrattive + FintRepulsive, folded
// as pair differences; u5x, v5y: the rows +-1 parts of the (2, 1)-link terms, finished with rows +-2.
template <class C> struct StencilSums {
  V2<C> qx, qy, sx, sy, u5x, v5y;
};

// Row 0: p[k] = psi(x + (k - 2, 0)), rm / rp = rho(x -+ (1, 0)).
template <class C>
__device__ __forceinline__ void sums_row0(StencilSums<C>& a, const KParams<C>& kp, const V2<C> p[5], V2<C> rm,
                                          V2<C> rp) {
  a.qx = p_mul(splat<C>(wq<C>(1)), p_sub(rp, rm));
  a.sx = p_fma(v2<C>(kp.a4x2[0], kp.a4x2[1]), p_sub(p[4], p[0]),
               p_mul(v2<C>(kp.a1[0], kp.a1[1]), p_sub(p[3], p[1])));
}

// Rows +-1: pu[k] = psi(x + (k - 2, 1)), pd[k] = psi(x + (k - 2, -1)), ru[k] = rho(x + (k - 1, 1)),
// rd[k] = rho(x + (k - 1, -1)).
template <class C>
__device__ __forceinline__ void sums_row1(StencilSums<C>& a, const KParams<C>& kp, const V2<C> pu[5],
                                          const V2<C> pd[5], const V2<C> ru[3], const V2<C> rd[3]) {
  using V = V2<C>;
  const V w1 = splat<C>(wq<C>(1)), w2 = splat<C>(wq<C>(5));
  const V e01 = p_sub(ru[1], rd[1]), e11 = p_sub(ru[2], rd[0]), em1 = p_sub(ru[0], rd[2]);
  a.qx = p_fma(w2, p_sub(e11, em1), a.qx);
  a.qy = p_fma(w2, p_add(e11, em1), p_mul(w1, e01));
  const V d01 = p_sub(pu[2], pd[2]), d11 = p_sub(pu[3], pd[1]), dm1 = p_sub(pu[1], pd[3]);
  const V d21 = p_sub(pu[4], pd[0]), dm21 = p_sub(pu[0], pd[4]);
  const V a2 = v2<C>(kp.a2[0], kp.a2[1]);
  a.sx = p_fma(a2, p_sub(d11, dm1), a.sx);
  a.sy = p_fma(a2, p_add(d11, dm1), p_mul(v2<C>(kp.a1[0], kp.a1[1]), d01));
  a.u5x = p_sub(d21, dm21);
  a.v5y = p_add(d21, dm21);
}

// Rows +-2: pu[k] = psi(x + (k - 2, 2)), pd[k] = psi(x + (k - 2, -2)).
template <class C>
__device__ __forceinline__ void sums_row2(StencilSums<C>& a, const KParams<C>& kp, const V2<C> pu[5],
                                          const V2<C> pd[5]) {
  using V = V2<C>;
  const V two = splat<C>(C(2));
  const V a5 = v2<C>(kp.a5[0], kp.a5[1]), a8 = v2<C>(kp.a8x2[0], kp.a8x2[1]);
  const V d02 = p_sub(pu[2], pd[2]), d12 = p_sub(pu[3], pd[1]), dm12 = p_sub(pu[1], pd[3]);
  const V d22 = p_sub(pu[4], pd[0]), dm22 = p_sub(pu[0], pd[4]);
  a.sx = p_fma(a5, p_fma(two, a.u5x, p_sub(d12, dm12)), a.sx);
  a.sx = p_fma(a8, p_sub(d22, dm22), a.sx);
  a.sy = p_fma(v2<C>(kp.a4x2[0], kp.a4x2[1]), d02, a.sy);
  a.sy = p_fma(a5, p_fma(two, p_add(d12, dm12), a.v5y), a.sy);
  a.sy = p_fma(a8, p_add(d22, dm22), a.sy);
}

// Forces from the stencil sums: lane l for component l, the constant x acceleration included, the
// buoyancy of Eq. alphaG left to the caller (buoyant_fy).  crx / cry: the cross sums of the other
// component's density; psl = psi(x); r = (rho_1, rho_2) at the node.
template <class C>
__device__ __forceinline__ void sums_forces(const StencilSums<C>& a, const KParams<C>& kp, V2<C> r, V2<C> psl,
                                            V2<C>& Fx, V2<C>& Fyp, V2<C>& crx, V2<C>& cry) {
  using V = V2<C>;
  crx = swap_lanes(a.qx);  // component l is pushed by the other component's density
  cry = swap_lanes(a.qy);
  const V npsl = p_mul(psl, splat<C>(C(-1)));
  const V gr = p_mul(splat<C>(-kp.gx), r);
  Fx = p_fma(r, splat<C>(kp.body_fx), p_fma(npsl, a.sx, p_mul(gr, crx)));
  Fyp = p_fma(npsl, a.sy, p_mul(gr, cry));
}

// Interaction force on both fluid components at the node whose shared-memory centre is (cx, cy), lane l
// for component l (Eqs. FAB, FintAttrattive, FintRepulsive, with the constant x acceleration; the
// buoyancy is left to the caller), and the parts the adjoint needs: cr, s and psi_l(x) (see
// StencilSums).  SM is any shared-memory view with interleaved pairs rho[rows][cols] and
// psi[rows][cols] (the tile of the fused step, the row window of the strip-marching step).
template <class C, class SM>
__device__ __forceinline__ void node_force_pair(const SM& sm, const KParams<C>& kp, int cx, int cy, V2<C> r,
                                                V2<C>& Fx, V2<C>& Fyp, V2<C>& crx, V2<C>& cry, V2<C>& sx,
                                                V2<C>& sy, V2<C>& psl) {
  using V = V2<C>;
  StencilSums<C> a;
  V pu[5], pd[5], ru[3], rd[3];
#pragma unroll
  for (int k = 0; k < 5; ++k) pu[k] = sm.psi[cy][cx + k - 2];
  sums_row0<C>(a, kp, pu, sm.rho[cy][cx - 1], sm.rho[cy][cx + 1]);
  psl = pu[2];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    pu[k] = sm.psi[cy + 1][cx + k - 2];
    pd[k] = sm.psi[cy - 1][cx + k - 2];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ru[k] = sm.rho[cy + 1][cx + k - 1];
    rd[k] = sm.rho[cy - 1][cx + k - 1];
  }
  sums_row1<C>(a, kp, pu, pd, ru, rd);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    pu[k] = sm.psi[cy + 2][cx + k - 2];
    pd[k] = sm.psi[cy - 2][cx + k - 2];
  }
  sums_row2<C>(a, kp, pu, pd);
  sums_forces<C>(a, kp, r, psl, Fx, Fyp, crx, cry);
  sx = a.sx;
  sy = a.sy;
}

// Fy of both components: the interaction part plus the buoyancy rho_l alpha_g T of Eq. alphaG.
template <class C> __device__ __forceinline__ V2<C> buoyant_fy(const KParams<C>& kp, V2<C> Fyp, V2<C> r, C T) {
  return p_fma(p_mul(r, splat<C>(kp.alpha_g)), splat<C>(T), Fyp);
}

// Forces with their adjoint parts per component (arrays indexed by component).
template <class C, class SM>
__device__ __forceinline__ void node_force_parts(const SM& sm, const KParams<C>& kp, int cx, int cy, C r1, C r2, C T,
                                                 C Fx[2], C Fy[2], C crx[2], C cry[2], C sx[2], C sy[2], C psl[2]) {
  V2<C> fx, fyp, qx, qy, tx, ty, ps;
  const V2<C> r = v2<C>(r1, r2);
  node_force_pair<C, SM>(sm, kp, cx, cy, r, fx, fyp, qx, qy, tx, ty, ps);
  const V2<C> fy = buoyant_fy<C>(kp, fyp, r, T);
  Fx[0] = fx.x, Fx[1] = fx.y, Fy[0] = fy.x, Fy[1] = fy.y;
  crx[0] = qx.x, crx[1] = qx.y, cry[0] = qy.x, cry[1] = qy.y;
  sx[0] = tx.x, sx[1] = tx.y, sy[0] = ty.x, sy[1] = ty.y, psl[0] = ps.x, psl[1] = ps.y;
}

template <class C, class SM>
__device__ __forceinline__ void node_forces(const SM& sm, const KParams<C>& kp, int cx, int cy, C r1, C r2, C T,
                                            C Fx[2], C Fy[2]) {
  V2<C> fx, fyp, qx, qy, tx, ty, ps;
  const V2<C> r = v2<C>(r1, r2);
  node_force_pair<C, SM>(sm, kp, cx, cy, r, fx, fyp, qx, qy, tx, ty, ps);
  const V2<C> fy = buoyant_fy<C>(kp, fyp, r, T);
  Fx[0] = fx.x, Fx[1] = fx.y, Fy[0] = fy.x, Fy[1] = fy.y;
}

// Reciprocals of rho_1, rho_2 and rho_1 + rho_2 from one division.
template <class C> __device__ __forceinline__ void three_reciprocals(C r1, C r2, C& i1, C& i2, C& irho) {
  const C rho = s_add(r1, r2);
  const C p12 = s_mul(r1, r2);
  const C inv = recip<C>(s_mul(p12, rho));
  // i1 = (r2 rho) inv and i2 = (r1 rho) inv as one lane pair (each lane the two scalar products)
  const V2<C> q = p_mul(p_mul(v2<C>(r2, r1), splat<C>(rho)), splat<C>(inv));
  i1 = q.x;
  i2 = q.y;
  irho = s_mul(p12, inv);
}

// Velocities of a node (Eq. velo, u^(H) = u + F / (2 rho)) from its bare momentum and total forces.
template <class C>
__device__ __forceinline__ void node_velocities(C jx, C jy, C inv_rho, const C Fx[2], const C Fy[2], C& ux, C& uy,
                                                C& uHx, C& uHy) {
  // x and y as one lane pair: each lane the scalar operations u = j / rho, u^(H) = (F / 2) / rho + u
  const V2<C> u = p_mul(v2<C>(jx, jy), splat<C>(inv_rho));
  const V2<C> f = p_add(v2<C>(Fx[0], Fy[0]), v2<C>(Fx[1], Fy[1]));
  const V2<C> uh = p_fma(p_mul(splat<C>(C(0.5)), f), splat<C>(inv_rho), u);
  ux = u.x;
  uy = u.y;
  uHx = uh.x;
  uHy = uh.y;
}

// BGK relaxation of the 27 populations of one node (Eqs. BGK, LBMg, Teq); in shifted storage the
// deviations relax: f^eq - w_i rho_bar = w_i (drho + rho P_i(u)) with P_i(u) = 3 c_i.u + 4.5 (c_i.u)^2
// - 1.5 u^2.  With tau = 1 (tau_g = 1) the post-collision population is the equilibrium itself and the
// relaxation arithmetic is skipped.  The fluid components are computed as lane pairs; for the
// direction opposite to c_i, P = c_i.u (4.5 c_i.u - 3) - 1.5 u^2, which is P at -c_i.u exactly.
template <class C, bool SHIFT, bool RELAX>
__device__ __forceinline__ void collide_fluid(const KParams<C>& kp, const C f[9], const C h[9], C r1, C r2, C dr1,
                                              C dr2, C ux, C uy, C irl0, C irl1, const C Fx[2], const C Fy[2],
                                              C post[27]) {
  using V = V2<C>;
  const V r = v2<C>(r1, r2), ir = v2<C>(irl0, irl1);
  const V tau = splat<C>(kp.tau);
  // Eq. shift: u_l = u + tau F_l / rho_l (without relaxation tau is 1 and tau F_l is F_l exactly)
  const V fx = v2<C>(Fx[0], Fx[1]), fy = v2<C>(Fy[0], Fy[1]);
  const V ulx = p_fma(RELAX ? p_mul(tau, fx) : fx, ir, splat<C>(ux));
  const V uly = p_fma(RELAX ? p_mul(tau, fy) : fy, ir, splat<C>(uy));
  const V nusq = p_mul(splat<C>(C(-1.5)), p_fma(ulx, ulx, p_mul(uly, uly)));
  const V base = SHIFT ? v2<C>(dr1, dr2) : r;
  const V k45 = splat<C>(C(4.5)), p3 = splat<C>(C(3)), m3 = splat<C>(C(-3));
  V cu[9];
  cu[1] = ulx, cu[2] = uly, cu[5] = p_add(ulx, uly), cu[6] = p_sub(uly, ulx);
  V feq[9];
  if constexpr (SHIFT) {
    feq[0] = p_mul(splat<C>(wq<C>(0)), p_fma(r, nusq, base));
  } else {
    // without a shift f^eq = w_i rho (1 + P_i) = A + A P_i, A = w_i rho once per weight class
    const V a0 = p_mul(splat<C>(wq<C>(0)), r);
    feq[0] = p_fma(a0, nusq, a0);
  }
  const V a1 = SHIFT ? r : p_mul(splat<C>(wq<C>(1)), r), a5 = SHIFT ? r : p_mul(splat<C>(wq<C>(5)), r);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const bool odd = (i == 3 || i == 4 || i == 7 || i == 8);
    const V c = cu[odd ? oppq(i) : i];
    const V poly = p_fma(c, p_fma(k45, c, odd ? m3 : p3), nusq);
    if constexpr (SHIFT) {
      feq[i] = p_mul(splat<C>(wq<C>(i)), p_fma(r, poly, base));
    } else {
      const V a = i <= 4 ? a1 : a5;
      feq[i] = p_fma(a, poly, a);
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    V q = feq[i];
    if constexpr (RELAX) {
      const V pop = v2<C>(f[i], h[i]);
      q = p_fma(p_sub(q, pop), splat<C>(kp.inv_tau), pop);
    }
    post[i] = q.x;
    post[9 + i] = q.y;
  }
}

// Thermal equilibria (Eq. Teq) with u^(H), the directions paired with their opposites as lanes.
template <class C, bool SHIFT, bool RELAX>
__device__ __forceinline__ void collide_thermal(const KParams<C>& kp, const C g[9], C T, C dT, C uHx, C uHy,
                                                C post[27]) {
  using V = V2<C>;
  const C nusq = s_mul(C(-1.5), s_fma(uHx, uHx, s_mul(uHy, uHy)));
  const C base = SHIFT ? dT : T;
  const V vn = splat<C>(nusq), vT = splat<C>(T), vb = splat<C>(base), k45 = splat<C>(C(4.5));
  const V pm3 = v2<C>(C(3), C(-3));
  // without a shift g^eq = w_i T (1 + P_i) = A + A P_i, A = w_i T once per weight class
  const C g0 = SHIFT ? s_mul(wq<C>(0), s_fma(T, nusq, base)) : s_fma(s_mul(wq<C>(0), T), nusq, s_mul(wq<C>(0), T));
  post[18] = RELAX ? s_fma(s_add(g0, -g[0]), kp.inv_tau_g, g[0]) : g0;
  const C cus[4] = {uHx, uHy, s_add(uHx, uHy), s_add(uHy, -uHx)};
  const int dir[4] = {1, 2, 5, 6};
  const V t1 = splat<C>(SHIFT ? T : s_mul(wq<C>(1), T)), t5 = splat<C>(SHIFT ? T : s_mul(wq<C>(5), T));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = dir[k], o = oppq(i);
    const V c = splat<C>(cus[k]);
    const V poly = p_fma(c, p_fma(k45, c, pm3), vn);
    V q;
    if constexpr (SHIFT) q = p_mul(splat<C>(wq<C>(i)), p_fma(vT, poly, vb));
    else q = p_fma(i <= 4 ? t1 : t5, poly, i <= 4 ? t1 : t5);
    if constexpr (RELAX) {
      const V pop = v2<C>(g[i], g[o]);
      q = p_fma(p_sub(q, pop), splat<C>(kp.inv_tau_g), pop);
    }
    post[18 + i] = q.x;
    post[18 + o] = q.y;
  }
}

template <class C, bool SHIFT>
__device__ __forceinline__ void node_collide(const KParams<C>& kp, const C f[9], const C h[9], const C g[9], C r1, C r2,
                                             C dr1, C dr2, C T, C dT, C ux, C uy, C irl0, C irl1, const C Fx[2],
                                             const C Fy[2], C uHx, C uHy, C post[27]) {
  if (kp.tau_is_one)
    collide_fluid<C, SHIFT, false>(kp, f, h, r1, r2, dr1, dr2, ux, uy, irl0, irl1, Fx, Fy, post);
  else
    collide_fluid<C, SHIFT, true>(kp, f, h, r1, r2, dr1, dr2, ux, uy, irl0, irl1, Fx, Fy, post);
  if (kp.tau_g_is_one)
    collide_thermal<C, SHIFT, false>(kp, g, T, dT, uHx, uHy, post);
  else
    collide_thermal<C, SHIFT, true>(kp, g, T, dT, uHx, uHy, post);
}

// Streaming (push) of the 27 post-collision populations of fluid node (gx, gy) (row-major index idx in
// the padded buffer) with half-way bounce-back of f and thermal anti-bounce-back of g where x + c_i is
// solid (Sec. 2.2).  A link into a moving flat wall row also takes 6 w_i rho_l c_ix u_wall (r1, r2:
// the node's densities).  solid[cy + c_iy][cx + c_ix] is the solid flag of x + c_i in the caller's
// shared-memory view.  FAST: no solid node around and no periodic wrap, every store is a constant offset.
template <class S, class C, bool FAST, int RX>
__device__ __forceinline__ void push_store(SF<S>* __restrict__ fout, const KParams<C>& kp, int idx, int gx, int gy,
                                           const C post[27], const unsigned char (*solid)[RX], int cx, int cy, C r1,
                                           C r2, bool fast_store = false) {
  using F = SF<S>;
  using G = SG<S>;
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
  G* __restrict__ gout = thermal_planes<S>(fout, plane);
  // a form with one phase-B instance takes the constant-offset stores at run time on the tiles that
  // allow them (fast_store: no solid node around the tile and no periodic wrap); the others decide at
  // compile time
  if constexpr (FAST || Storage<S>::kFastPath) fast_store = FAST;
  if (fast_store) {
    F* dst = fout + idx;
    G* gdst = gout + idx;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int off = cxq(i) + cyq(i) * pitch;
      dst[i * plane + off] = down<F>(post[i]);
      dst[(9 + i) * plane + off] = down<F>(post[9 + i]);
      gdst[i * plane + off] = down<G>(post[18 + i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      if (!solid[cy + cyq(i)][cx + cxq(i)]) {
        int dx = gx + cxq(i);
        dx = dx < 0 ? dx + nx : (dx >= nx ? dx - nx : dx);
        int dy = gy + cyq(i);
        if (kp.periodic_y) dy = dy < 0 ? dy + ny : (dy >= ny ? dy - ny : dy);
        const int didx = dy * pitch + dx;
        fout[i * plane + didx] = down<F>(post[i]);
        fout[(9 + i) * plane + didx] = down<F>(post[9 + i]);
        gout[i * plane + didx] = down<G>(post[18 + i]);
      } else {
        const int o = oppq(i);
        const int ys = gy + cyq(i);
        const C twoTw = (2 * ys < ny) ? kp.twoTw_down : kp.twoTw_up;
        C m1 = C(0), m2 = C(0);
        if (cxq(i) != 0 && !kp.periodic_y && (ys == 0 || ys == ny - 1)) {
          const C wc = wq<C>(i) * C(cxq(i)) * (ys == 0 ? kp.uw6[0] : kp.uw6[1]);
          m1 = wc * r1;
          m2 = wc * r2;
        }
        fout[o * plane + idx] = down<F>(post[i] - m1);
        fout[(9 + o) * plane + idx] = down<F>(post[9 + i] - m2);
        gout[o * plane + idx] = down<G>(-post[18 + i] + wq<C>(i) * twoTw);
      }
    }
  }
}

// Moments of a fluid node (Sec. 2.1, 2.3): densities and bare momentum from phase A, T from its thermal
// populations; in shifted storage the sums are deviations from the shift.
template <class C> struct NodeMoments {
  C dr1, dr2, r1, r2, dT, T, jx, jy;
};
template <class C, bool SHIFT, class SMT>
__device__ __forceinline__ NodeMoments<C> node_moments(const SMT& sm, const KParams<C>& kp, int tx, int ty,
                                                       const C g[9]) {
  NodeMoments<C> m;
  const V2<C> dr = sm.rho[ty + 2][tx + 2];
  m.dr1 = dr.x;
  m.dr2 = dr.y;
  m.r1 = SHIFT ? m.dr1 + kp.rho_bar[0] : m.dr1;
  m.r2 = SHIFT ? m.dr2 + kp.rho_bar[1] : m.dr2;
  m.dT = s_sum9(g);
  m.T = m.dT + (SHIFT ? kp.T_bar : C(0));
  m.jx = sm.jx[ty][tx];
  m.jy = sm.jy[ty][tx];
  return m;
}

// The rest of a fluid node's step once its moments and interaction forces (Fx, and Fyp without the
// buoyancy) are known: buoyancy, velocities (Eq. velo, Eq. shift, u^(H) = u + F / (2 rho)), BGK
// collisions and the push store.  Returns u^(H)_y T (the advective part of Eq. NuTime).
template <class S, class C, bool SHIFT, bool FAST, class SMT>
__device__ __forceinline__ C step_finish(SF<S>* __restrict__ fout, const KParams<C>& kp, const SMT& sm,
                                         const C f[9], const C h[9], const C g[9], const NodeMoments<C>& m,
                                         int tx, int ty, int gx, int gy, int idx, V2<C> Fx2, V2<C> Fyp,
                                         bool fast_store = false) {
  const V2<C> Fy2 = buoyant_fy<C>(kp, Fyp, v2<C>(m.r1, m.r2), m.T);
  const C Fx[2] = {Fx2.x, Fx2.y}, Fy[2] = {Fy2.x, Fy2.y};
  C i1, i2, inv_rho, ux, uy, uHx, uHy;
  three_reciprocals<C>(m.r1, m.r2, i1, i2, inv_rho);
  node_velocities<C>(m.jx, m.jy, inv_rho, Fx, Fy, ux, uy, uHx, uHy);
  C post[27];
  node_collide<C, SHIFT>(kp, f, h, g, m.r1, m.r2, m.dr1, m.dr2, m.T, m.dT, ux, uy, i1, i2, Fx, Fy, uHx, uHy, post);
  push_store<S, C, FAST>(fout, kp, idx, gx, gy, post, sm.solid, tx + 2, ty + 2, m.r1, m.r2, fast_store);
  return uHy * m.T;
}

// Phase B on one tile.  MODE_STEP: collide and push-store; MODE_OBS: accumulate the observables
// of the node into acc[]; MODE_FIELDS: write rho1, rho2, T, u^(H) to aux planes.
template <class S, class C, bool SHIFT, int MODE, bool FAST, int TX, int TY, int BY, class Src>
__device__ __forceinline__ void tile_phase_b(const Src& pop, SF<S>* __restrict__ fout, const KParams<C>& kp, int x0, int y0,
                                             const TileSmem<C, TX, TY, mode_needs_T(MODE)>& sm, double* __restrict__ aux,
                                             double acc[kObsSlots], C* nu = nullptr, bool fast_store = false) {
  const int nx = kp.nx, ny = kp.ny, pitch = kp.pitch, plane = kp.plane;
#pragma unroll 1
  for (int k = 0; k < TY / BY; ++k) {
    const int tx = threadIdx.x, ty = threadIdx.y + k * BY;
    const int gx = x0 + tx, gy = y0 + ty;
    if (!FAST && (gx >= nx || gy >= ny)) continue;
    const int cx = tx + 2, cy = ty + 2;
    if (!FAST && sm.solid[cy][cx]) {
      if constexpr (MODE == MODE_FIELDS) {
        const long long n = (long long)gy * nx + gx, N = (long long)nx * ny;
        aux[n] = kp.rho_w_d[0];
        aux[N + n] = kp.rho_w_d[1];
        aux[2 * N + n] = (2 * gy < ny) ? kp.T_down_d : kp.T_up_d;
        aux[3 * N + n] = 0.0;
        aux[4 * N + n] = 0.0;
      }
      continue;
    }
    const int idx = gy * pitch + gx;
    // moments (Sec. 2.1, 2.3): densities and momentum from phase A, T from the thermal populations;
    // in shifted storage the sums are deviations from the shift
    C f[9], h[9], g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = C(pop(18 + i, idx, tx, ty));
    const bool relax = !kp.tau_is_one;
    if (relax) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f[i] = C(pop(i, idx, tx, ty));
        h[i] = C(pop(9 + i, idx, tx, ty));
      }
    }
    const NodeMoments<C> m = node_moments<C, SHIFT>(sm, kp, tx, ty, g);
    const C dr1 = m.dr1, dr2 = m.dr2, r1 = m.r1, r2 = m.r2, dT = m.dT, T = m.T;
    V2<C> fx2, fyp2, q0, q1, q2, q3, q4;
    node_force_pair<C>(sm, kp, cx, cy, v2<C>(r1, r2), fx2, fyp2, q0, q1, q2, q3, q4);
    if constexpr (mode_steps(MODE)) {
      const C uyT = step_finish<S, C, SHIFT, FAST>(fout, kp, sm, f, h, g, m, tx, ty, gx, gy, idx, fx2, fyp2, fast_store);
      if constexpr (MODE == MODE_STEP_NU) *nu = s_add(*nu, uyT);  // in the arithmetic precision
      continue;
    }
    const V2<C> fy2 = buoyant_fy<C>(kp, fyp2, v2<C>(r1, r2), T);
    const C Fx[2] = {fx2.x, fx2.y}, Fy[2] = {fy2.x, fy2.y};
    // velocities: Eq. velo, Eq. shift, u^(H) = u + F / (2 rho)
    C i1, i2, inv_rho, ux, uy, uHx, uHy;
    three_reciprocals<C>(r1, r2, i1, i2, inv_rho);
    node_velocities<C>(m.jx, m.jy, inv_rho, Fx, Fy, ux, uy, uHx, uHy);
    const C rho = r1 + r2;

    if constexpr (MODE == MODE_OBS) {
      const C Tup = sm.solid[cy + 1][cx] ? C(2) * sm.T[cy + 1][cx] - T : sm.T[cy + 1][cx];
      const C Tdn = sm.solid[cy - 1][cx] ? C(2) * sm.T[cy - 1][cx] - T : sm.T[cy - 1][cx];
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
      // x momentum the next step hands to a flat wall row through the bounce-back links of this node
      // (momentum exchange, c_ix (f* + f_bounced) per component).  In shifted storage the
      // 2 w_i rho_bar c_ix terms of the two diagonal links cancel, so deviations suffice.
      if (!kp.periodic_y && (gy == 1 || gy == ny - 2)) {
        C post[27];
        node_collide<C, SHIFT>(kp, f, h, g, r1, r2, dr1, dr2, T, dT, ux, uy, i1, i2, Fx, Fy, uHx, uHy, post);
        double wsum = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int ys = gy + cyq(i);
          if (cxq(i) == 0 || (ys != 0 && ys != ny - 1)) continue;
          const C wc = wq<C>(i) * C(cxq(i)) * (ys == 0 ? kp.uw6[0] : kp.uw6[1]);
          const C b1 = post[i] - wc * r1, b2 = post[9 + i] - wc * r2;
          wsum += (double)cxq(i) * (((double)post[i] + (double)b1) + ((double)post[9 + i] + (double)b2));
        }
        acc[gy == 1 ? 9 : 10] += wsum;
      }
    } else if constexpr (MODE == MODE_FIELDS) {
      const long long n = (long long)gy * nx + gx, N = (long long)nx * ny;
      aux[n] = (double)r1;
      aux[N + n] = (double)r2;
      aux[2 * N + n] = (double)T;
      aux[3 * N + n] = (double)uHx;
      aux[4 * N + n] = (double)uHy;
    }
  }
}

// One tile: phase A, barrier, phase B (fast path when the CTA allows it).
template <class S, class C, bool SHIFT, int MODE, int TX, int TY, int BY, bool CG = false>
__device__ __forceinline__ void tile_step(const SF<S>* __restrict__ fin, SF<S>* __restrict__ fout, const KParams<C>& kp,
                                          int x0, int y0, TileSmem<C, TX, TY, mode_needs_T(MODE)>& sm,
                                          double* __restrict__ aux, double acc[kObsSlots], C* nu = nullptr) {
  constexpr int NT = TX * BY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const bool fast = tile_phase_a<S, C, SHIFT, mode_needs_T(MODE), TX, TY, NT, CG>(fin, kp, x0, y0, sm, tid);
  const GlobalPopSource<S, CG> pop{fin, kp.plane};
  if constexpr (Storage<S>::kFastPath) {
    if (mode_steps(MODE) && fast) {
      tile_phase_b<S, C, SHIFT, MODE, true, TX, TY, BY>(pop, fout, kp, x0, y0, sm, aux, acc, nu);
      return;
    }
  }
  tile_phase_b<S, C, SHIFT, MODE, false, TX, TY, BY>(pop, fout, kp, x0, y0, sm, aux, acc, nu, fast);
}

// Block-wide deterministic sum of the observable accumulators into aux[slot * kObsSlots + v].
template <int NT>
__device__ __forceinline__ void block_obs_store(double acc[kObsSlots], double* __restrict__ aux, long long slot) {
  __shared__ double s_red[NT / 32][kObsSlots];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
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
    aux[slot * kObsSlots + tid] = s;
  }
}

// Warp sum in the arithmetic precision (a fixed shuffle tree).
__device__ __forceinline__ float warp_sum_c(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_c(double v) { return warp_sum(v); }

template <class S, class C, bool SHIFT, int MODE, int TX, int TY, int BY, int MINB>
__global__ void __launch_bounds__(TX * BY, MINB)
lb_step_kernel(const SF<S>* __restrict__ fin, SF<S>* __restrict__ fout, const KParams<C> kp, double* __restrict__ aux) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileSmem<C, TX, TY, mode_needs_T(MODE)>*>(smem_raw);
  double acc[kObsSlots];
#pragma unroll
  for (int v = 0; v < kObsSlots; ++v) acc[v] = 0.0;
  C nu = C(0);
  tile_step<S, C, SHIFT, MODE, TX, TY, BY>(fin, fout, kp, blockIdx.x * TX, blockIdx.y * TY, sm, aux, acc, &nu);
  if constexpr (MODE == MODE_OBS) block_obs_store<TX * BY>(acc, aux, (long long)blockIdx.y * gridDim.x + blockIdx.x);
  if constexpr (MODE == MODE_STEP_NU) {
    // one partial per warp, no CTA barrier: aux[(CTA) * warps + warp]
    const int tid = threadIdx.y * TX + threadIdx.x;
    const C v = warp_sum_c(nu);
    if ((tid & 31) == 0)
      aux[((long long)blockIdx.y * gridDim.x + blockIdx.x) * (TX * BY / 32) + (tid >> 5)] = (double)v;
  }
}

// Rest equilibria f = w_i rho, g = w_i T at fluid nodes (stored minus the shift), 0 at solid nodes.
template <class S, bool SHIFT>
__global__ void lb_init_kernel(const double* __restrict__ fields, SF<S>* __restrict__ buf, const StepCfg cfg) {
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
    buf[i * cfg.plane + idx] = down<SF<S>>(solid ? 0.0 : a);
    buf[(9 + i) * cfg.plane + idx] = down<SF<S>>(solid ? 0.0 : b);
    thermal_planes<S>(buf, cfg.plane)[i * cfg.plane + idx] = down<SG<S>>(solid ? 0.0 : c);
  }
}

__device__ __forceinline__ double shift_of(const StepCfg& cfg, int k) {
  const int comp = k / 9, i = k % 9;
  const double s = comp == 0 ? cfg.rho_bar[0] : (comp == 1 ? cfg.rho_bar[1] : cfg.T_bar);
  return wq<double>(i) * s;
}

template <class S, bool SHIFT>
__global__ void lb_plane_get_kernel(int k, const SF<S>* __restrict__ buf, double* __restrict__ out, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  const long long idx = (long long)gy * cfg.pitch + gx;
  const double v = k < 18 ? up<double>(buf[k * cfg.plane + idx])
                          : up<double>(thermal_planes<S>(buf, cfg.plane)[(k - 18) * cfg.plane + idx]);
  out[n] = solid ? 0.0 : (SHIFT ? v + shift_of(cfg, k) : v);
}

template <class S, bool SHIFT>
__global__ void lb_plane_put_kernel(int k, const double* __restrict__ in, SF<S>* __restrict__ buf, const StepCfg cfg) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= cfg.nx || gy >= cfg.ny) return;
  const long long n = (long long)gy * cfg.nx + gx;
  bool solid = cfg.mask != nullptr && cfg.mask[n] != 0;
  if (!cfg.periodic_y && (gy == 0 || gy == cfg.ny - 1)) solid = true;
  const double v = SHIFT ? in[n] - shift_of(cfg, k) : in[n];
  const long long idx = (long long)gy * cfg.pitch + gx;
  if (k < 18)
    buf[k * cfg.plane + idx] = down<SF<S>>(solid ? 0.0 : v);
  else
    thermal_planes<S>(buf, cfg.plane)[(k - 18) * cfg.plane + idx] = down<SG<S>>(solid ? 0.0 : v);
}

// Launch with the tile's shared memory as dynamic shared memory (the larger tiles need more than
// the 48 KB static limit); the opt-in attribute is set once per kernel instantiation.
template <class S, int MODE, int TX, int TY, int BY, int MB, bool SHIFT>
cudaError_t launch_tile_kernel(const dim3& grid, const SF<S>* in, SF<S>* out, const KParams<SC<S>>& kp, double* aux,
                               cudaStream_t s) {
  constexpr size_t bytes = sizeof(TileSmem<SC<S>, TX, TY, mode_needs_T(MODE)>);
  auto kern = lb_step_kernel<S, SC<S>, SHIFT, MODE, TX, TY, BY, MB>;
  static std::atomic<unsigned long long> done{0};  // one bit per device ordinal (mod 64)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit);
  }
  kern<<<grid, dim3(TX, BY, 1), bytes, s>>>(in, out, kp, aux);
  return cudaGetLastError();
}

inline dim3 rows_grid(const StepCfg& c) { return dim3((unsigned)((c.nx + 127) / 128), (unsigned)c.ny, 1u); }

// rho_1 of every node (nx*ny doubles; rho_w at solid nodes) with the arithmetic of the field mode:
// phase A's packed sum of component 1's nine populations (p_sum9, lane x; lane y carries zeros),
// plus the shift in shifted storage, widened to double.  The same bits as plane 0 of MODE_FIELDS, from 9 of
// the 27 planes.
template <class S, bool SHIFT>
__global__ void lb_rho1_kernel(const SF<S>* __restrict__ buf, double* __restrict__ out, const KParams<SC<S>> kp) {
  using C = SC<S>;
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= kp.nx || gy >= kp.ny) return;
  const int n = gy * kp.nx + gx;
  bool solid = kp.mask != nullptr && kp.mask[n] != 0;
  if (!kp.periodic_y && (gy == 0 || gy == kp.ny - 1)) solid = true;
  if (solid) {
    out[n] = kp.rho_w_d[0];
    return;
  }
  const SF<S>* src = buf + (gy * kp.pitch + gx);
  V2<C> u[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) u[i] = v2<C>(C(ld_pop<false>(src + i * kp.plane)), C(0));
  const V2<C> d = p_sum9(u);
  const C r1 = SHIFT ? d.x + kp.rho_bar[0] : d.x;
  out[n] = (double)r1;
}

template <class S> struct MinBlocks;
template <> struct MinBlocks<double> { static constexpr int value = 2; };
template <> struct MinBlocks<float> { static constexpr int value = 3; };

template <class S, bool SHIFT>
cudaError_t launch_impl(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s) {
  using C = SC<S>;
  using T = Tile<C>;
  constexpr int MB = MinBlocks<C>::value;
  const dim3 grid = grid_for(c.nx, c.ny, T::TX, T::TY);
  const SF<S>* in = static_cast<const SF<S>*>(fin);
  SF<S>* out = static_cast<SF<S>*>(fout);
  const KParams<C> kp = make_kparams<C>(c);
  switch (mode) {
    case MODE_STEP:
      return launch_tile_kernel<S, MODE_STEP, T::TX, T::TY, T::BY, MB, SHIFT>(grid, in, out, kp, aux, s);
    case MODE_OBS:
      return launch_tile_kernel<S, MODE_OBS, T::TX, T::TY, T::BY, 1, SHIFT>(grid, in, out, kp, aux, s);
    case MODE_FIELDS:
      return launch_tile_kernel<S, MODE_FIELDS, T::TX, T::TY, T::BY, 1, SHIFT>(grid, in, out, kp, aux, s);
    case MODE_RHO1:
      lb_rho1_kernel<S, SHIFT><<<rows_grid(c), 128, 0, s>>>(in, aux, kp);
      return cudaGetLastError();
    default:
      return cudaErrorInvalidValue;
  }
}

template <class S, bool SHIFT, int TX, int TY, int BY, int MB>
cudaError_t launch_step_shape(const StepCfg& c, const void* fin, void* fout, cudaStream_t s) {
  return launch_tile_kernel<S, MODE_STEP, TX, TY, BY, MB, SHIFT>(grid_for(c.nx, c.ny, TX, TY),
                                                               static_cast<const SF<S>*>(fin), static_cast<SF<S>*>(fout),
                                                               make_kparams<SC<S>>(c), nullptr, s);
}

}  // namespace tlb
