// Arithmetic types of the per-sample elimination state.
//
//   double / cd   IEEE FP64 (real / complex)
//   float  / cf   IEEE FP32
//   df     / cdf  double-float: an unevaluated sum hi + lo of two FP32 numbers with
//                 |lo| <= ulp(hi)/2, about 48 significant bits (Dekker, "A floating-point
//                 technique for extending the available precision", Numer. Math. 18, 1971;
//                 error-free sum after Knuth, TAOCP vol. 2, 4.2.2).  It runs on the FP32
//                 pipes, which on GB300 are about 60 times faster than the FP64 pipe.
//
// The error-free transforms use the _rn intrinsics so that the compiler never fuses or
// reorders them.
#pragma once

#include "ffs_internal.cuh"

namespace fermi {

struct df {
  float hi, lo;
};
struct cdf {
  df re, im;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// a * b with the exact product of the high parts (FMA) plus the cross terms.
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
// acc - a * b
__device__ __forceinline__ df df_fms(df acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(acc.hi, -p);
  return quick_two_sum(s.hi, __fsub_rn(__fadd_rn(s.lo, acc.lo), e));
}
// a / b: quotient of the high parts corrected by one residual step.
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_fms(a, df{q1, 0.f}, b);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}

// Lazy double-float accumulator: the running sum hi gets each high product through an
// error-free sum; the rounding errors, the exact error of the high product (FMA) and the
// cross terms collect in lo without renormalising after every term.  About 13 FP32
// instructions per multiply-add; lz_get renormalises once at the end.
struct lzf {
  float hi, lo;
};
__device__ __forceinline__ void lz_mac(lzf& a, df x, df y) {  // a += x y
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.hi, -p);
  const float cr = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, __fadd_rn(e, cr)));
}
// a += x for an FP32 x: the error-free sum of the high parts, its error added to lo
// (seven instructions, no renormalising).
__device__ __forceinline__ void lz_add(lzf& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ df lz_get(lzf a) {
  const df s = two_sum(a.hi, a.lo);
  return quick_two_sum(s.hi, s.lo);
}

// The value V = sum_{d=2..8} G_d 2^(-8(d-2)) of the seven group accumulators of an Ozaki
// slice product (G_d = sum of the slice products a_i b_j with i + j = d: integers of at
// most 2^23, exact in FP32), for NV outputs at once; ld(d, r) reads G_d into r.  Smallest
// groups first: G_8, G_7 and G_6 in FP32 (one rounding of at most half a unit of G_6,
// 2^-33 of a unit of G_2), then G_5 .. G_2 by lazy error-free sums (seven instructions
// each instead of the twelve of a renormalised double-float addition).
template <int NV, typename Ld>
__device__ __forceinline__ void oz_group_sum(Ld ld, lzf (&S)[NV]) {
  uint32_t r[NV];
  ld(8, r);
#pragma unroll
  for (int n = 0; n < NV; ++n) S[n].hi = __uint_as_float(r[n]) * 0x1p-16f;
  ld(7, r);
#pragma unroll
  for (int n = 0; n < NV; ++n) S[n].hi = __fmaf_rn(__uint_as_float(r[n]), 0x1p-8f, S[n].hi);
  ld(6, r);
#pragma unroll
  for (int n = 0; n < NV; ++n) S[n] = lzf{__fadd_rn(__uint_as_float(r[n]), S[n].hi) * 0x1p-32f, 0.f};
#pragma unroll 1
  for (int d = 5; d >= 2; --d) {
    ld(d, r);
    const float p2 = ldexpf(1.f, -8 * (d - 2));
#pragma unroll
    for (int n = 0; n < NV; ++n) lz_add(S[n], __uint_as_float(r[n]) * p2);
  }
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Uniform interface over the six state types.
template <typename A> struct Ar;

template <> struct Ar<double> {
  using U = double;  // element type of the FP64 copy of U
  static constexpr bool cplx = false;
  __device__ static double from(U u) { return u; }
  __device__ static double out(double a) { return a; }
  __device__ static double zero() { return 0.0; }
  __device__ static double one() { return 1.0; }
  __device__ static double neg(double a) { return -a; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double fms(double acc, double a, double b) { return fma(-a, b, acc); }
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static double abs2(double a) { return a * a; }
};
template <> struct Ar<float> {
  using U = double;
  static constexpr bool cplx = false;
  __device__ static float from(U u) { return (float)u; }
  __device__ static double out(float a) { return a; }
  __device__ static float zero() { return 0.f; }
  __device__ static float one() { return 1.f; }
  __device__ static float neg(float a) { return -a; }
  __device__ static float add(float a, float b) { return a + b; }
  __device__ static float fms(float acc, float a, float b) { return fmaf(-a, b, acc); }
  __device__ static float div(float a, float b) { return a / b; }
  __device__ static double abs2(float a) { return (double)a * a; }
};
template <> struct Ar<df> {
  using U = double;
  static constexpr bool cplx = false;
  __device__ static df from(U u) { return df_from(u); }
  __device__ static double out(df a) { return df_to(a); }
  __device__ static df zero() { return {0.f, 0.f}; }
  __device__ static df one() { return {1.f, 0.f}; }
  __device__ static df neg(df a) { return df_neg(a); }
  __device__ static df add(df a, df b) { return df_add(a, b); }
  __device__ static df fms(df acc, df a, df b) { return df_fms(acc, a, b); }
  __device__ static df div(df a, df b) { return df_div(a, b); }
  __device__ static double abs2(df a) { const double d = df_to(a); return d * d; }
};
template <> struct Ar<cd> {
  using U = cd;
  static constexpr bool cplx = true;
  __device__ static cd from(U u) { return u; }
  __device__ static cd out(cd a) { return a; }
  __device__ static cd zero() { return {0.0, 0.0}; }
  __device__ static cd one() { return {1.0, 0.0}; }
  __device__ static cd neg(cd a) { return {-a.re, -a.im}; }
  __device__ static cd add(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
  __device__ static cd fms(cd acc, cd a, cd b) { return fermi::fms(acc, a, b); }
  __device__ static cd div(cd a, cd b) { return a / b; }
  __device__ static double abs2(cd a) { return a.re * a.re + a.im * a.im; }
};
template <> struct Ar<cf> {
  using U = cd;
  static constexpr bool cplx = true;
  __device__ static cf from(U u) { return {(float)u.re, (float)u.im}; }
  __device__ static cd out(cf a) { return {a.re, a.im}; }
  __device__ static cf zero() { return {0.f, 0.f}; }
  __device__ static cf one() { return {1.f, 0.f}; }
  __device__ static cf neg(cf a) { return {-a.re, -a.im}; }
  __device__ static cf add(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
  __device__ static cf fms(cf acc, cf a, cf b) { return fermi::fms(acc, a, b); }
  __device__ static cf div(cf a, cf b) { return a / b; }
  __device__ static double abs2(cf a) { return (double)a.re * a.re + (double)a.im * a.im; }
};
template <> struct Ar<cdf> {
  using U = cd;
  static constexpr bool cplx = true;
  __device__ static cdf from(U u) { return {df_from(u.re), df_from(u.im)}; }
  __device__ static cd out(cdf a) { return {df_to(a.re), df_to(a.im)}; }
  __device__ static cdf zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
  __device__ static cdf one() { return {{1.f, 0.f}, {0.f, 0.f}}; }
  __device__ static cdf neg(cdf a) { return {df_neg(a.re), df_neg(a.im)}; }
  __device__ static cdf add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
  // acc - a b = (acc.re - a.re b.re + a.im b.im) + i (acc.im - a.re b.im - a.im b.re)
  __device__ static cdf fms(cdf acc, cdf a, cdf b) {
    const df re = df_fms(df_fms(acc.re, a.re, b.re), df_neg(a.im), b.im);
    const df im = df_fms(df_fms(acc.im, a.re, b.im), a.im, b.re);
    return {re, im};
  }
  // a / b = a conj(b) / |b|^2
  __device__ static cdf div(cdf a, cdf b) {
    const df d = df_fms(df_mul(b.re, b.re), df_neg(b.im), b.im);
    const df nr = df_fms(df_mul(a.re, b.re), df_neg(a.im), b.im);
    const df ni = df_fms(df_mul(a.im, b.re), a.re, b.im);
    return {df_div(nr, d), df_div(ni, d)};
  }
  __device__ static double abs2(cdf a) {
    const double r = df_to(a.re), i = df_to(a.im);
    return r * r + i * i;
  }
};

// Warp shuffles of any state type (moved as 32-bit words).
template <typename A> __device__ __forceinline__ A shfl_xor_any(A v, int o) {
  static_assert(sizeof(A) % 4 == 0, "state types are made of 32-bit words");
  constexpr int W = sizeof(A) / 4;
  uint32_t w[W];
  memcpy(w, &v, sizeof(A));
#pragma unroll
  for (int i = 0; i < W; ++i) w[i] = __shfl_xor_sync(0xffffffffu, w[i], o);
  memcpy(&v, w, sizeof(A));
  return v;
}

}  // namespace fermi
