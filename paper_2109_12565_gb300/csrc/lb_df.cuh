// Double-float ("df") arithmetic for the LB_DF64 storage form: every value is an unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, a 48-bit significand, and every operation runs
// on the FP32 pipe.  On GB300 the FP64 pipe issues 2 operations per clock and SM, the FP32 pipe 128,
// so a fused step in double-float arithmetic outruns the FP64 one although each operation takes
// several FP32 instructions.
//
// The error-free transformations are the classical ones: the sum of two floats as s + e (Knuth's
// two-sum, six operations; Dekker's fast two-sum, three, when |a| >= |b|) and their product as p + e
// with one fused multiply-add (p = a b rounded, e = fma(a, b, -p)).  Every operation is written with
// explicit round-to-nearest intrinsics, so the compiler contracts nothing and every kernel that calls
// these functions computes the same bits.
//
// Storage: a population is a float2 (hi, lo) in memory, 8 bytes, the footprint of an FP64 value; no
// conversion to or from FP64 happens in the step (on GB300 those conversions run at the FP64 rate).
#pragma once
#include <math.h>
#include <stdint.h>

#include "lb_kernels.cuh"

namespace tlb {

struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr df(float v) : hi(v), lo(0.0f) {}
  // round a double to the nearest double-float (exact for the 48 leading significand bits)
  __host__ __device__ constexpr df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit df(float2 v) : hi(v.x), lo(v.y) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// Knuth two-sum: s + e = a + b exactly.
__device__ __forceinline__ float df_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
// Dekker fast two-sum, |a| >= |b| (or a = 0): s + e = a + b exactly.
__device__ __forceinline__ float df_fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}
// p + e = a b exactly.
__device__ __forceinline__ float df_two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

// a + b: the leading parts summed error-free, the low parts in FP32, one renormalisation (11
// operations).  The only rounding beyond the final one is that of a.lo + b.lo, at most
// 2^-24 |a.lo + b.lo| <= 2^-48 (|a| + |b|): the error is bounded relative to the operands rather than
// to the sum, which under cancellation is larger than the summands' own rounding in FP64 by a small
// factor only (the step's quantities are O(1) and the tolerance is absolute).  The variant that also
// sums the low parts error-free costs 20 operations; the whole step measured 13% slower with it and
// 5.4e-14 instead of 7.3e-14 from the FP64 oracle after 1000 steps of the 64 x 64 emulsion.
__device__ __forceinline__ df df_add(df a, df b) {
  float e;
  const float s = df_two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float l;
  const float h = df_fast_two_sum(s, e, l);
  return df(h, l);
}
__device__ __forceinline__ df df_neg(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df df_mul(df a, df b) {
  float e;
  float p = df_two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  p = df_fast_two_sum(p, e, e);
  return df(p, e);
}
// a b + c with one renormalisation: the leading product and sum are error-free, the cross terms
// and the low parts are summed in FP32.
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  float e, e2;
  const float p = df_two_prod(a.hi, b.hi, e);
  float s = df_two_sum(p, c.hi, e2);
  float t = __fmaf_rn(a.hi, b.lo, e);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fadd_rn(t, c.lo);
  t = __fadd_rn(t, e2);
  s = df_fast_two_sum(s, t, t);
  return df(s, t);
}

__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = df_add(a, b); }
__device__ __forceinline__ bool operator>(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df a, df b) { return b > a; }

// Lane pair of double-float values (two components, or a direction and its opposite), 16 bytes.
struct __align__(16) df2 {
  df x, y;
};
template <> struct V2T<df> { using type = df2; };

// The lane-pair operations run the double-float algorithms above on packed FP32x2 instructions (one
// instruction for both lanes, each lane rounding once), so each lane equals the scalar operation.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 f2_two_sum(float2 a, float2 b, float2& e) {
  const float2 s = f2_add(a, b);
  const float2 bb = f2_sub(s, a);
  e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
  return s;
}
__device__ __forceinline__ float2 f2_fast_two_sum(float2 a, float2 b, float2& e) {
  const float2 s = f2_add(a, b);
  e = f2_sub(b, f2_sub(s, a));
  return s;
}
__device__ __forceinline__ float2 hi2(df2 a) { return make_float2(a.x.hi, a.y.hi); }
__device__ __forceinline__ float2 lo2(df2 a) { return make_float2(a.x.lo, a.y.lo); }
__device__ __forceinline__ df2 make_df2(float2 h, float2 l) { return df2{df(h.x, l.x), df(h.y, l.y)}; }

// In shared memory a pair is kept as (high parts of both lanes, low parts of both lanes): one 16-byte
// load then gives the two register pairs the packed instructions take.
struct __align__(16) df2s {
  float2 hi, lo;
  __device__ __forceinline__ operator df2() const { return make_df2(hi, lo); }
  __device__ __forceinline__ df2s& operator=(const df2& v) {
    hi = hi2(v);
    lo = lo2(v);
    return *this;
  }
};
template <> struct SmemPairT<df> { using type = df2s; };

__device__ __forceinline__ df2 p_add(df2 a, df2 b) {  // df_add per lane, packed
  float2 e;
  const float2 s = f2_two_sum(hi2(a), hi2(b), e);
  e = f2_add(e, f2_add(lo2(a), lo2(b)));
  float2 l;
  const float2 h = f2_fast_two_sum(s, e, l);
  return make_df2(h, l);
}
__device__ __forceinline__ df2 p_sub(df2 a, df2 b) {
  const float2 bh = hi2(b), bl = lo2(b);
  return p_add(a, make_df2(make_float2(-bh.x, -bh.y), make_float2(-bl.x, -bl.y)));
}
__device__ __forceinline__ df2 p_mul(df2 a, df2 b) {
  const float2 ah = hi2(a), bh = hi2(b);
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ah, lo2(b), e);
  e = __ffma2_rn(lo2(a), bh, e);
  float2 l;
  const float2 h = f2_fast_two_sum(p, e, l);
  return make_df2(h, l);
}
__device__ __forceinline__ df2 p_fma(df2 a, df2 b, df2 c) {
  const float2 ah = hi2(a), bh = hi2(b);
  const float2 p = __fmul2_rn(ah, bh);
  const float2 e = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
  float2 e2;
  const float2 sh = f2_two_sum(p, hi2(c), e2);
  float2 t = __ffma2_rn(ah, lo2(b), e);
  t = __ffma2_rn(lo2(a), bh, t);
  t = f2_add(t, lo2(c));
  t = f2_add(t, e2);
  float2 l;
  const float2 h = f2_fast_two_sum(sh, t, l);
  return make_df2(h, l);
}
// Nine-term sums: the high parts accumulated by two-sums, the two-sums' errors and the low parts summed
// in FP32, one renormalisation at the end (8 operations a term against the 11 of the add).  Every
// rounding beyond the final one is an FP32 rounding of a partial sum of low-order terms, below
// 2^-24 of it: the error regime of the add.
template <> struct Sum9<df2> {
  __device__ __forceinline__ static df2 of(const df2 u[9]) {
    float2 s = hi2(u[0]), err = make_float2(0.0f, 0.0f), lo = lo2(u[0]);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      float2 e;
      s = f2_two_sum(s, hi2(u[i]), e);
      err = f2_add(err, e);
      lo = f2_add(lo, lo2(u[i]));
    }
    float2 l;
    const float2 h = f2_fast_two_sum(s, f2_add(err, lo), l);
    return make_df2(h, l);
  }
};
template <> struct SSum9<df> {
  __device__ __forceinline__ static df of(const df u[9]) {
    float s = u[0].hi, err = 0.0f, lo = u[0].lo;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      float e;
      s = df_two_sum(s, u[i].hi, e);
      err = __fadd_rn(err, e);
      lo = __fadd_rn(lo, u[i].lo);
    }
    float l;
    const float h = df_fast_two_sum(s, __fadd_rn(err, lo), l);
    return df(h, l);
  }
};

__device__ __forceinline__ df s_add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df s_mul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df s_fma(df a, df b, df c) { return df_fma(a, b, c); }

// Storage form: populations as (hi, lo) float pairs, arithmetic in double-float, no shift.
struct DF {};
template <> struct Storage<DF> {
  using F = float2;
  using G = float2;
  using C = df;
  static constexpr bool kFastPath = false;  // one phase B: the step is bound by arithmetic and code size
};
template <> __device__ __forceinline__ df up<df, float2>(float2 v) { return df(v); }
template <> __device__ __forceinline__ double up<double, float2>(float2 v) { return (double)v.x + (double)v.y; }
template <> __device__ __forceinline__ float2 down<float2, df>(df v) { return make_float2(v.hi, v.lo); }
template <> __device__ __forceinline__ float2 down<float2, double>(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// D2Q9 weights as double-float constants: 4/9, 1/9, 1/36 split into their nearest float and the
// float nearest to the remainder.
template <> __host__ __device__ constexpr df wq<df>(int i) {
  return i == 0 ? df(4.0 / 9.0) : (i <= 4 ? df(1.0 / 9.0) : df(1.0 / 36.0));
}

template <> struct Tile<df> { static constexpr int TX = 32, TY = 16, BY = 8; };
template <> struct MinBlocks<df> { static constexpr int value = 3; };

// 1 / x: an FP32 reciprocal refined by two Newton steps y <- y + y (1 - x y), the residual taken in
// double-float; relative error about 2^-47.
template <> __device__ __forceinline__ df recip<df>(df x) {
  const float y0 = __fdividef(1.0f, x.hi);
  float pe;
  const float p = df_two_prod(x.hi, y0, pe);
  pe = __fmaf_rn(x.lo, y0, pe);
  const float e1 = __fsub_rn(__fsub_rn(1.0f, p), pe);  // 1 - p is exact: p is within a few ulps of 1
  float l1;
  const float h1 = df_fast_two_sum(y0, __fmul_rn(y0, e1), l1);
  const df y1(h1, l1);
  const df q = df_mul(x, y1);
  const float e2 = __fsub_rn(__fsub_rn(1.0f, q.hi), q.lo);
  return df_add(y1, df(__fmul_rn(y1.hi, e2), 0.0f));
}

// ---- exp(-x) for the pseudo-potential psi = rho0 (1 - exp(-rho / rho0)) ----
// Two-level table: x = n / 4096 + r with n = rint(4096 x), |r| <= 2^-13;
// exp(-x) = T1[n >> 6] T2[n & 63] exp(-r), T1[k] = exp(-k / 64) (k = 0..256), T2[j] = exp(-j / 4096)
// (j = 0..63), and exp(-r) = 1 - r + r^2 / 2 - r^3 / 6 + r^4 / 24 (the next term is below 2^-70).
// The tables are double-float roundings of FP64 exp values, written by the host before the first
// step (df_exp_tables_init).  Arguments outside [0, 4) take an FP64 exp instead.  The tables are
// defined here: one translation unit (lb_df64.cu) includes this header.
constexpr int kDfExpT1 = 257, kDfExpT2 = 64;
__device__ float2 g_df_exp_t1[kDfExpT1];
__device__ float2 g_df_exp_t2[kDfExpT2];
cudaError_t df_exp_tables_init();

__device__ __forceinline__ df df_exp_neg(df x) {
  const float t = __fmul_rn(x.hi, 4096.0f);
  if (!(x.hi >= 0.0f) || !(t < 16384.0f)) {
    const double v = exp(-(double)x);
    const float h = __double2float_rn(v);
    return df(h, __double2float_rn(v - (double)h));
  }
  // rint(t) by the 1.5 * 2^23 shift: exact for 0 <= t < 2^22
  const float m = __fadd_rn(t, 12582912.0f);
  const int n = __float_as_int(m) - 0x4B400000;
  const float nf = __fmul_rn(__fsub_rn(m, 12582912.0f), 1.0f / 4096.0f);  // n / 4096, exact
  float rl;
  const float rh = df_two_sum(__fsub_rn(x.hi, nf), x.lo, rl);  // x.hi - n / 4096 is exact (Sterbenz)
  // r^2 / 2 in double-float, r^3 / 6 and r^4 / 24 in FP32
  float r2l;
  const float r2h = df_two_prod(rh, rh, r2l);
  r2l = __fmaf_rn(2.0f * rh, rl, r2l);
  const float small = __fmaf_rn(__fmul_rn(r2h, r2h), 1.0f / 24.0f, -__fmul_rn(__fmul_rn(r2h, rh), 1.0f / 6.0f));
  // 1 - r + r^2 / 2 + small; |r| <= 2^-13, so the leading 1 dominates every other term
  float e;
  const float s = df_two_sum(1.0f, -rh, e);
  e = __fadd_rn(e, -rl);
  e = __fadd_rn(e, __fmul_rn(0.5f, r2h));
  e = __fadd_rn(e, __fadd_rn(__fmul_rn(0.5f, r2l), small));
  float el;
  const float eh = df_fast_two_sum(s, e, el);
  const df er(eh, el);
  const df t1(__ldg(&g_df_exp_t1[n >> 6])), t2(__ldg(&g_df_exp_t2[n & 63]));
  return df_mul(df_mul(t1, t2), er);
}

template <> __device__ __forceinline__ df psi_exp<df>(df rho, df rho0, df inv_rho0) {
  const df e = df_exp_neg(df_mul(rho, inv_rho0));
  return df_add(rho0, df_neg(df_mul(rho0, e)));
}

}  // namespace tlb

namespace tlb {

// psi of both components with the arithmetic of psi_exp<df> on packed FP32x2 instructions (per lane the
// same operations, so the same bits); the table lookups stay per lane, and a lane outside the table
// range is recomputed by the scalar path (FP64 exp).
template <> __device__ __forceinline__ df2 psi_exp_pair<df>(df2 rho, df rho0, df inv_rho0) {
  const df2 x = p_mul(rho, df2{inv_rho0, inv_rho0});
  const float2 xh = hi2(x), xl = lo2(x);
  const float2 t = __fmul2_rn(xh, make_float2(4096.0f, 4096.0f));
  const bool ok0 = xh.x >= 0.0f && t.x < 16384.0f, ok1 = xh.y >= 0.0f && t.y < 16384.0f;
  const float2 tc = make_float2(ok0 ? t.x : 0.0f, ok1 ? t.y : 0.0f);
  const float2 xhc = make_float2(ok0 ? xh.x : 0.0f, ok1 ? xh.y : 0.0f);
  const float2 xlc = make_float2(ok0 ? xl.x : 0.0f, ok1 ? xl.y : 0.0f);
  const float2 shift = make_float2(12582912.0f, 12582912.0f);
  const float2 m = f2_add(tc, shift);
  const int n0 = __float_as_int(m.x) - 0x4B400000, n1 = __float_as_int(m.y) - 0x4B400000;
  const float2 nf = __fmul2_rn(f2_sub(m, shift), make_float2(1.0f / 4096.0f, 1.0f / 4096.0f));
  float2 rl;
  const float2 rh = f2_two_sum(f2_sub(xhc, nf), xlc, rl);
  const float2 r2h = __fmul2_rn(rh, rh);
  float2 r2l = __ffma2_rn(rh, rh, make_float2(-r2h.x, -r2h.y));
  r2l = __ffma2_rn(__fmul2_rn(make_float2(2.0f, 2.0f), rh), rl, r2l);
  const float2 c3 = __fmul2_rn(__fmul2_rn(r2h, rh), make_float2(1.0f / 6.0f, 1.0f / 6.0f));
  const float2 small = __ffma2_rn(__fmul2_rn(r2h, r2h), make_float2(1.0f / 24.0f, 1.0f / 24.0f), make_float2(-c3.x, -c3.y));
  float2 e;
  const float2 s = f2_two_sum(make_float2(1.0f, 1.0f), make_float2(-rh.x, -rh.y), e);
  e = f2_add(e, make_float2(-rl.x, -rl.y));
  e = f2_add(e, __fmul2_rn(make_float2(0.5f, 0.5f), r2h));
  e = f2_add(e, f2_add(__fmul2_rn(make_float2(0.5f, 0.5f), r2l), small));
  float2 el;
  const float2 eh = f2_fast_two_sum(s, e, el);
  const df2 t1{df(__ldg(&g_df_exp_t1[n0 >> 6])), df(__ldg(&g_df_exp_t1[n1 >> 6]))};
  const df2 t2{df(__ldg(&g_df_exp_t2[n0 & 63])), df(__ldg(&g_df_exp_t2[n1 & 63]))};
  const df2 E = p_mul(p_mul(t1, t2), make_df2(eh, el));
  const df2 r0{rho0, rho0};
  df2 psi = p_sub(r0, p_mul(r0, E));
  if (!ok0) psi.x = psi_exp<df>(rho.x, rho0, inv_rho0);
  if (!ok1) psi.y = psi_exp<df>(rho.y, rho0, inv_rho0);
  return psi;
}

}  // namespace tlb
