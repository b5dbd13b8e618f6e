// Arithmetic policies for the partition-method kernels.
//
// Each policy supplies one scalar type T and the handful of operations the
// elimination recurrences need: x*y, x - y*z, -x, 1/x, a pivot check, and
// conversions from and to the storage types of the arrays (double, float,
// float2).  The kernels are written once against this interface.
//
//   ArF64  native IEEE binary64.  On GB300 the fp64 pipe retires about
//          1/72 of the fp32 rate, so this is the plain, ALU-bound solve.
//   ArDF   double-float ("float-float") arithmetic: a value is an unevaluated
//          sum hi + lo of two binary32 numbers, |lo| <= ulp(hi).  The
//          error-free transformations are Knuth's TwoSum, Dekker's
//          Fast2Sum, and the fma-based TwoProd (see Muller et al., Handbook
//          of Floating-Point Arithmetic, 2nd ed., ch. 4 and 14).  It keeps
//          about 2^-46 relative accuracy per operation on the fp32 pipes.
//          fp64 inputs are split into hi + lo with integer operations (the
//          fp64<->fp32 conversion instructions share the slow fp64 pipe).
//          Valid for magnitudes in about [2^-103, 2^127]; smaller nonzero
//          inputs are flushed to zero.
//   ArF32  native IEEE binary32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tps {

// ------------------------------------------------------------------ fp64
struct ArF64 {
  using T = double;
  __device__ __forceinline__ static T zero() { return 0.0; }
  __device__ __forceinline__ static T one() { return 1.0; }
  __device__ __forceinline__ static T mul(T x, T y) { return x * y; }
  __device__ __forceinline__ static T mul_nn(T x, T y) { return x * y; }
  __device__ __forceinline__ static T mul_neg_nn(T x, T y) { return -(x * y); }
  __device__ __forceinline__ static T norm(T x) { return x; }
  // x - y*z, one rounding
  __device__ __forceinline__ static T sub_mul(T x, T y, T z) { return fma(-y, z, x); }
  __device__ __forceinline__ static T sub_mul_dom(T x, T y, T z) { return fma(-y, z, x); }
  __device__ __forceinline__ static T sub_mul_nn(T x, T y, T z) { return fma(-y, z, x); }
  __device__ __forceinline__ static T neg(T x) { return -x; }
  // 1/x by one third-order Newton-Raphson (Halley-type) step from the
  // hardware approximation rcp.approx.ftz.f64: with e = 1 - x r,
  // 1/x = r (1 + e + e^2 + ...), so r + r (e + e^2) leaves O(e^3) -- below
  // 2^-53 for a seed good to 2^-18.  Three fp64 fused multiply-adds.
  __device__ __forceinline__ static T rcp(T x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
  // true when x is zero, subnormal, infinite or NaN; integer test on the
  // exponent field, so it does not occupy the slow fp64 pipe
  __device__ __forceinline__ static bool bad_pivot(T x) {
    const unsigned ex = (unsigned)__double2hiint(x) & 0x7FF00000u;
    return ex == 0u || ex == 0x7FF00000u;
  }
  __device__ __forceinline__ static T from(double v) { return v; }
  __device__ __forceinline__ static T from_pivot(double v) { return v; }
  __device__ __forceinline__ static T from(float v) { return (double)v; }
  __device__ __forceinline__ static void to(double& dst, T v) { dst = v; }
};

// ------------------------------------------------------------------ fp32
struct ArF32 {
  using T = float;
  __device__ __forceinline__ static T zero() { return 0.0f; }
  __device__ __forceinline__ static T one() { return 1.0f; }
  __device__ __forceinline__ static T mul(T x, T y) { return __fmul_rn(x, y); }
  __device__ __forceinline__ static T mul_nn(T x, T y) { return __fmul_rn(x, y); }
  __device__ __forceinline__ static T mul_neg_nn(T x, T y) { return __fmul_rn(-x, y); }
  __device__ __forceinline__ static T norm(T x) { return x; }
  __device__ __forceinline__ static T sub_mul(T x, T y, T z) { return fmaf(-y, z, x); }
  __device__ __forceinline__ static T sub_mul_dom(T x, T y, T z) { return fmaf(-y, z, x); }
  __device__ __forceinline__ static T sub_mul_nn(T x, T y, T z) { return fmaf(-y, z, x); }
  __device__ __forceinline__ static T neg(T x) { return -x; }
  // hardware reciprocal approximation refined by one Newton-Raphson step
  __device__ __forceinline__ static T rcp(T x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
  }
  // zero, subnormal, infinite or NaN
  __device__ __forceinline__ static bool bad_pivot(T x) {
    const float m = fabsf(x);
    return !(m >= 1.17549435e-38f && m <= 3.40282347e38f);
  }
  __device__ __forceinline__ static T from(float v) { return v; }
  __device__ __forceinline__ static void to(float& dst, T v) { dst = v; }
  // fp64 storage (the fp32 elimination of the mixed-precision solve): the
  // value truncated to binary32 and widened back exactly, both with integer
  // operations (the conversion instructions run at the slow fp64 rate)
  __device__ __forceinline__ static T from(double v);
  __device__ __forceinline__ static T from_pivot(float v) { return v; }
  __device__ __forceinline__ static T from_pivot(double v);
  __device__ __forceinline__ static void to(double& dst, T v);
};

// ------------------------------------------------------------------ double-float
struct df64 {
  float hi, lo;
};

// Knuth TwoSum: s + e == a + b exactly (no precondition on magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker Fast2Sum: exact when |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Split an fp64 value into hi + lo with integer operations.  hi keeps the
// sign, the exponent and the leading 24 significand bits (truncated); lo is
// the next 23 of the remaining 29 bits (truncated; relative error of the
// pair < 2^-46), built on a power-of-two "magic" float of hi's scale and
// recovered by one exact fp32 subtraction.  Values below 2^-103 in
// magnitude (zero included) give 0; magnitudes from 2^128 up are outside
// the representable range.
__device__ __forceinline__ df64 df_split(double v) {
  const unsigned wl = (unsigned)__double2loint(v);
  const unsigned wh = (unsigned)__double2hiint(v);
  // biased exponent >= 920 <=> float exponent field >= 24
  const bool ok = (wh & 0x7FF00000u) >= (920u << 20);
  const unsigned hb = (__funnelshift_l(wl, wh, 3) + 0x40000000u) | (wh & 0x80000000u);
  const unsigned mag = (hb & 0xFF800000u) - 0x0B800000u;  // +-2^(e-23) of hi
  const unsigned lob = mag | ((wl >> 6) & 0x007FFFFFu);
  df64 r;
  r.hi = ok ? __uint_as_float(hb) : 0.0f;
  r.lo = ok ? __fsub_rn(__uint_as_float(lob), __uint_as_float(mag)) : 0.0f;
  return r;
}

// The same split for a value that feeds a pivot: magnitudes from 2^128 up,
// infinities and NaN (whose exponent would wrap in df_split) have their
// magnitude clamped to exponent 1151 with an all-ones significand first,
// which gives a NaN high part that the pivot test reports (only finite
// magnitudes in [2^128, 2^128 (1 + 2^-20)) come out infinite).  Two integer
// operations more.
__device__ __forceinline__ df64 df_split_checked(double v) {
  const unsigned wl = (unsigned)__double2loint(v);
  const unsigned wh = (unsigned)__double2hiint(v);
  const bool ok = (wh & 0x7FF00000u) >= (920u << 20);
  const unsigned whc = min(wh & 0x7FFFFFFFu, 0x47FFFFFFu);
  const unsigned hb = (__funnelshift_l(wl, whc, 3) + 0x40000000u) | (wh & 0x80000000u);
  const unsigned mag = (hb & 0xFF800000u) - 0x0B800000u;
  const unsigned lob = mag | ((wl >> 6) & 0x007FFFFFu);
  df64 r;
  r.hi = ok ? __uint_as_float(hb) : 0.0f;
  r.lo = ok ? __fsub_rn(__uint_as_float(lob), __uint_as_float(mag)) : 0.0f;
  return r;
}

// Exact binary32 -> binary64 widening with integer operations (normal
// floats and zero; subnormal floats come out slightly off, as if normal).
__device__ __forceinline__ double f32_widen_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mg = u & 0x7FFFFFFFu;
  const unsigned wh = (mg == 0u ? 0u : ((mg >> 3) + 0x38000000u)) | (u & 0x80000000u);
  const unsigned wl = u << 29;
  return __hiloint2double((int)wh, (int)wl);
}

__device__ __forceinline__ float ArF32::from(double v) { return df_split(v).hi; }
__device__ __forceinline__ float ArF32::from_pivot(double v) { return df_split_checked(v).hi; }
__device__ __forceinline__ void ArF32::to(double& dst, float v) { dst = f32_widen_bits(v); }

struct ArDF {
  using T = df64;
  __device__ __forceinline__ static T zero() { return {0.0f, 0.0f}; }
  __device__ __forceinline__ static T one() { return {1.0f, 0.0f}; }
  __device__ __forceinline__ static T neg(T x) { return {-x.hi, -x.lo}; }
  // x*y: TwoProd of the high parts plus the two cross terms, renormalised.
  __device__ __forceinline__ static T mul(T x, T y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    T r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
  }
  // x*y left as the unevaluated pair (p, e), |e| <= ~2^-22 |p|: for a product
  // that only feeds sub_mul / mul (which accept such pairs); recurrences
  // renormalise through mul or sub_mul every step.
  __device__ __forceinline__ static T mul_nn(T x, T y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return {p, e};
  }
  // -(x*y) as an unevaluated pair; the negation rides on the operands.
  __device__ __forceinline__ static T mul_neg_nn(T x, T y) {
    const float p = __fmul_rn(-x.hi, y.hi);
    float e = fmaf(-x.hi, y.hi, -p);
    e = fmaf(-x.hi, y.lo, e);
    e = fmaf(-x.lo, y.hi, e);
    return {p, e};
  }
  // Renormalise a pair (Fast2Sum) so that |lo| <= ulp(hi) / 2.
  __device__ __forceinline__ static T norm(T x) {
    T r;
    fast_two_sum(x.hi, x.lo, r.hi, r.lo);
    return r;
  }
  // x - y*z without the final renormalisation: the pair (s, se) is exact
  // up to the product's rounding, but |se| may exceed ulp(s) / 2.  Safe for
  // a few steps of an accumulator that is renormalised periodically.
  __device__ __forceinline__ static T sub_mul_nn(T x, T y, T z) {
    const float p = __fmul_rn(y.hi, z.hi);
    float pe = fmaf(y.hi, z.hi, -p);
    pe = fmaf(y.hi, z.lo, pe);
    pe = fmaf(y.lo, z.hi, pe);
    float s, se;
    two_sum(x.hi, -p, s, se);
    return {s, __fadd_rn(se, __fsub_rn(x.lo, pe))};
  }
  // x - y*z: the product is formed as an unevaluated pair (p, pe), then
  // TwoSum of the high parts and a final Fast2Sum.
  __device__ __forceinline__ static T sub_mul(T x, T y, T z) {
    const float p = __fmul_rn(y.hi, z.hi);
    float pe = fmaf(y.hi, z.hi, -p);
    pe = fmaf(y.hi, z.lo, pe);
    pe = fmaf(y.lo, z.hi, pe);
    float s, se;
    two_sum(x.hi, -p, s, se);
    se = __fadd_rn(se, __fsub_rn(x.lo, pe));
    T r;
    fast_two_sum(s, se, r.hi, r.lo);
    return r;
  }
  // x - y*z when |x| >= |y*z| is known (the pivot update of a strictly
  // diagonally dominant matrix): Fast2Sum replaces TwoSum for the high parts.
  __device__ __forceinline__ static T sub_mul_dom(T x, T y, T z) {
    const float p = __fmul_rn(y.hi, z.hi);
    float pe = fmaf(y.hi, z.hi, -p);
    pe = fmaf(y.hi, z.lo, pe);
    pe = fmaf(y.lo, z.hi, pe);
    float s, se;
    fast_two_sum(x.hi, -p, s, se);
    se = __fadd_rn(se, __fsub_rn(x.lo, pe));
    T r;
    fast_two_sum(s, se, r.hi, r.lo);
    return r;
  }
  // 1/x: hardware fp32 reciprocal seed r (relative error e0 <= 2^-23),
  // then one third-order Newton-Raphson (Halley-type) correction carried in
  // double-float: with e = 1 - x*r (formed by fma from both parts of x),
  // 1/x = r (1 + e + e^2 + ...), so r + r*(e + e^2) leaves an O(e^3) error.
  __device__ __forceinline__ static T rcp(T x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
    float e = fmaf(-x.hi, r, 1.0f);
    e = fmaf(-x.lo, r, e);
    T out;
    fast_two_sum(r, __fmul_rn(r, fmaf(e, e, e)), out.hi, out.lo);
    return out;
  }
  // zero, subnormal or NaN high part (one comparison: non-finite inputs on
  // the diagonal arrive here as NaN through df_split_checked)
  __device__ __forceinline__ static bool bad_pivot(T x) { return !(fabsf(x.hi) >= 1.17549435e-38f); }
  __device__ __forceinline__ static T from(double v) { return df_split(v); }
  __device__ __forceinline__ static T from(float2 v) { return {v.x, v.y}; }
  // a diagonal entry: out-of-range inputs reach the pivot test
  __device__ __forceinline__ static T from_pivot(double v) { return df_split_checked(v); }
  __device__ __forceinline__ static T from_pivot(float2 v) { return from(v); }
  __device__ __forceinline__ static void to(double& dst, T v) {
    dst = __dadd_rn(f32_widen_bits(v.hi), f32_widen_bits(v.lo));
  }
  __device__ __forceinline__ static void to(float2& dst, T v) { dst = make_float2(v.hi, v.lo); }
};

}  // namespace tps
