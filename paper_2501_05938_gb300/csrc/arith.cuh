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
//          A pair keeps full precision for magnitudes of about [2^-103,
//          2^127], so every row of fp64 inputs is scaled by the power of
//          two that brings its diagonal entry into [1, 2) (exact: only the
//          exponent fields change, and a row's scale does not change x), and
//          d, hence x, by a further 2^26 that centres the pairs' window on
//          the solution's scale (undone when x is written).  What remains is
//          checked (RowChk): a, c or d above 2^84 |b| and an invalid b (0,
//          subnormal, infinite or NaN) in the row, |d / b| of the whole
//          system below 2^-84, an entry taken as 0 in a row that dominates
//          the system, and x at or above 2^101.
//   ArF32  native IEEE binary32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tps {

struct RowChk;

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

  // a row of inputs (native fp64 needs no scaling), and the output check
  template <bool kChk, class Tin>
  __device__ __forceinline__ static void row(Tin a, Tin b, Tin c, Tin d, T& A, T& B, T& C, T& D,
                                             RowChk&) {
    A = from(a); B = from_pivot(b); C = from(c); D = from(d);
  }
  __device__ __forceinline__ static bool out_bad(double v);
  __device__ __forceinline__ static bool out_bad(float) { return false; }
  // k_stage1 skips the first unknown's decayed chain (a second unrolled
  // chunk body): worth it where the fp64 pipe bounds the kernel (measured:
  // Stage 1 2.64 -> 1.97 ms at n = 2^27); the fp32-pipe policies keep one
  // body (the second one cost more in instruction fetch than it saved)
  static constexpr bool kSkipChain = true;
  // |x| below 2^-60 (a decayed product chain, see k_stage1)
  __device__ __forceinline__ static bool chain_small(T x) { return fabs(x) < 0x1p-60; }
  // |c| <= |beta| to about 2^-20, on the high words (integer pipe)
  __device__ __forceinline__ static bool mag_le(T c, T beta) {
    return ((unsigned)__double2hiint(c) & 0x7FFFFFFFu) <= ((unsigned)__double2hiint(beta) & 0x7FFFFFFFu);
  }
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
  // a row of fp32 inputs as they are; of fp64 inputs (the mixed solve)
  // scaled by its diagonal's power of two like the double-float rows
  template <bool kChk>
  __device__ __forceinline__ static void row(float a, float b, float c, float d, T& A, T& B,
                                             T& C, T& D, RowChk&) {
    A = a; B = b; C = c; D = d;
  }
  template <bool kChk>
  __device__ __forceinline__ static void row(double a, double b, double c, double d, T& A,
                                             T& B, T& C, T& D, RowChk& k);
  __device__ __forceinline__ static bool out_bad(float v) {
    return (__float_as_uint(v) & 0x7F800000u) == 0x7F800000u;
  }
  __device__ __forceinline__ static bool out_bad(double v);
  static constexpr bool kSkipChain = false;
  __device__ __forceinline__ static bool chain_small(T x) { return fabsf(x) < 0x1p-30f; }
  __device__ __forceinline__ static bool mag_le(T c, T beta) { return fabsf(c) <= fabsf(beta); }
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

// ------------------------------------------------------------------ row scaling
// Extra scale of d and x in the double-float rows: x's pairs then hold
// solutions with max |d / b| in [2^-84, 2^84] at full precision (a
// window of 2^(-103 - kDScale + 45) .. 2^(127 - kDScale - 17)), one
// as wide on either side of 1.
constexpr int kDScale = 26;

// Range bookkeeping of the fp64 rows a lane has loaded (see split_row).
// Exponent fields are the biased fp64 exponents in bits 20..30 (one
// binade is 1 << 20).  dcode, ecode, fcode are maxima over rows, per packed
// system, merged across the GPU by atomicMax and judged by range_codes_bad
// once every row is in; the rest is judged per lane.
struct RowChk {
  int ramax = -0x7FFFFFFF; // max over rows of max(E_a, E_c) - E_b
  int rdmax = -0x7FFFFFFF; // max over rows of E_d - E_b (d = 0 counts as E_d = 0)
  unsigned acmax = 0;      // max E_a, E_c (0x7FF00000: infinite or NaN)
  unsigned ebmin = 0x7FF00000u, ebmax = 0;  // E_b range (0 or 0x7FF00000: b
                                            // zero, subnormal, infinite, NaN)
  unsigned ecode = 0;      // max E_d (0: every d was 0; 0x7FF00000: not finite)
  bool flushed = false;    // a nonzero a, c (below 2^-103 |b|) or d (below
                           // 2^-(103 + kDScale) |b|) was taken as 0
  // a, c or d above 2^84 |b| (beyond what the solution's pairs hold, and
  // never part of a strictly diagonally dominant row), or not finite
  __device__ __forceinline__ bool range_bad() const {
    return max(ramax, rdmax) > (84 << 20) || max(acmax, ecode) == 0x7FF00000u;
  }
  __device__ __forceinline__ bool b_bad() const {
    return ebmin == 0u || ebmax == 0x7FF00000u;
  }
  // the codes of range_codes_bad: dcode = 2^31 + max (E_d - E_b), ecode,
  // and fcode = the lane's largest E_b if it took an entry as 0
  __device__ __forceinline__ unsigned dcode() const { return (unsigned)rdmax + 0x80000000u; }
  __device__ __forceinline__ unsigned fcode() const { return flushed ? ebmax : 0u; }
  __device__ __forceinline__ void reset_codes() {
    rdmax = -0x7FFFFFFF;
    ecode = 0u;
    flushed = false;
  }
};

// Code of |d / b| in RowChk::dcode(): 2^31 + ((E_d - E_b) << 20).  A system
// whose largest code is below kDcodeMin (|d / b| < 2^-84 in every row with
// d != 0) has x too small for its pairs' precision: d below 2^-(103 +
// kDScale) |b| is taken as 0, and that must stay below 2^-45 of the largest.
constexpr unsigned kDcodeMin = 0x80000000u - (84u << 20);

// A system's codes out of range: |d / b| too small everywhere, or an a, c or
// d taken as 0 in a block holding a row whose diagonal is so large against the
// system that the dropped term, up to 2^-102 |b| ||x|| (||x|| <= 2^20 max
// |d / b| allowed for), could exceed 2^-41 ||d||: E_b - 102 + (log2
// max|d/b| + 21) > E_d,max - 41, i.e. the exponent sum below exceeds 40.
// ec = 0: d = 0 everywhere, x = 0 exactly.
__host__ __device__ __forceinline__ bool range_codes_bad(unsigned dc, unsigned ec, unsigned fc) {
  if (ec == 0u) return false;
  if (dc < kDcodeMin) return true;
  if (fc == 0u) return false;
  const int rel = (int)(dc >> 20) - 2048;  // log2 max |d / b|, to the binade
  return (int)(fc >> 20) + rel - (int)(ec >> 20) > 40;
}

// df_split of v * 2^(1023 - E_b): `bias` = (127 - E_b) << 23 (mod 2^32)
// replaces the constant fp64-to-fp32 exponent rebias, so the row's scaling
// costs no instruction; `lo` is the smallest biased exponent field kept
// (the row's 2^-103), below which the value gives 0.  ex: v's exponent field.
__device__ __forceinline__ df64 df_split_scaled(double v, unsigned bias, unsigned lo,
                                                unsigned& ex) {
  const unsigned wl = (unsigned)__double2loint(v);
  const unsigned wh = (unsigned)__double2hiint(v);
  ex = wh & 0x7FF00000u;
  const bool ok = ex >= lo;
  const unsigned hb = (__funnelshift_l(wl, wh, 3) + bias) | (wh & 0x80000000u);
  const unsigned mag = (hb & 0xFF800000u) - 0x0B800000u;
  const unsigned lob = mag | ((wl >> 6) & 0x007FFFFFu);
  df64 r;
  r.hi = ok ? __uint_as_float(hb) : 0.0f;
  r.lo = ok ? __fsub_rn(__uint_as_float(lob), __uint_as_float(mag)) : 0.0f;
  return r;
}

// The diagonal entry scaled into [1, 2): sign, exponent 127 and the leading
// 23 fraction bits; the next 23 bits on a magic of 2^-23.
__device__ __forceinline__ df64 df_split_unit(double v) {
  const unsigned wl = (unsigned)__double2loint(v);
  const unsigned wh = (unsigned)__double2hiint(v);
  const unsigned sgn = wh & 0x80000000u;
  const unsigned hb = (__funnelshift_l(wl, wh, 3) & 0x007FFFFFu) | sgn | 0x3F800000u;
  const unsigned mag = sgn | 0x34000000u;
  df64 r;
  r.hi = __uint_as_float(hb);
  r.lo = __fsub_rn(__uint_as_float(mag | ((wl >> 6) & 0x007FFFFFu)), __uint_as_float(mag));
  return r;
}

// One row a x[i-1] + b x[i] + c x[i+1] = d of fp64 inputs as pairs: a, b, c
// multiplied by 2^(1023 - E_b) (b then lies in [1, 2)) and d by
// 2^(1023 - E_b + kDScale); the row's x is unchanged up to the common
// 2^kDScale, and power-of-two scaling is exact.  a and c below 2^-103 |b|
// become 0, which perturbs the row by less than 2^-103 of its diagonal; d
// below 2^-(103 + kDScale) |b| becomes 0.  With kChk the row's range is
// recorded in k (RowChk).
template <bool kChk>
__device__ __forceinline__ void split_row(double a, double b, double c, double d, df64& A,
                                          df64& B, df64& C, df64& D, RowChk& k) {
  const unsigned eb = (unsigned)__double2hiint(b) & 0x7FF00000u;
  const unsigned bias = (127u << 23) - eb * 8u;
  // thresholds of the kept range (at least 1: zero and fp64 subnormals are 0)
  const unsigned lo = (unsigned)max((int)eb - (103 << 20), 1 << 20);
  const unsigned lod = (unsigned)max((int)eb - ((103 + kDScale) << 20), 1 << 20);
  unsigned ea, ec, ed;
  A = df_split_scaled(a, bias, lo, ea);
  B = df_split_unit(b);
  C = df_split_scaled(c, bias, lo, ec);
  D = df_split_scaled(d, bias + ((unsigned)kDScale << 23), lod, ed);
  if constexpr (kChk) {
    const unsigned eac = max(ea, ec);
    k.ramax = max(k.ramax, (int)eac - (int)eb);
    k.rdmax = max(k.rdmax, (int)ed - (int)eb);
    k.acmax = max(k.acmax, eac);
    k.ebmin = min(k.ebmin, eb);
    k.ebmax = max(k.ebmax, eb);
    k.ecode = max(k.ecode, ed);
    // nonzero and below the split's threshold (the split's own comparisons)
    k.flushed |= (ea != 0u && ea < lo) || (ec != 0u && ec < lo) || (ed != 0u && ed < lod);
  }
}

// fp64 value of a pair of x's scale, with the 2^kDScale of split_row
// undone: integer widening of both parts, the exponent rebias lowered by
// kDScale (exact for normal parts and zero; a subnormal part, |x| far
// below the solution's scale, comes out off by at most 2^-(126 + kDScale)).
__device__ __forceinline__ double f32_widen_unscaled(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mg = u & 0x7FFFFFFFu;
  const unsigned wh =
      (mg == 0u ? 0u : ((mg >> 3) + 0x38000000u - ((unsigned)kDScale << 20))) | (u & 0x80000000u);
  return __hiloint2double((int)wh, (int)(u << 29));
}
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  return __dadd_rn(f32_widen_unscaled(hi), f32_widen_unscaled(lo));
}

// A computed fp64 x outside what the arithmetic represents: not finite
// (native fp64), at or above 2^(127 - kDScale) (double-float: the pair's
// high part is near the binary32 limit, or an intermediate overflowed).
__device__ __forceinline__ bool x_out_of_range_f64(double v) {
  return ((unsigned)__double2hiint(v) & 0x7FF00000u) == 0x7FF00000u;
}
__device__ __forceinline__ bool x_out_of_range_df(double v) {
  return ((unsigned)__double2hiint(v) & 0x7FF00000u) >= ((1023u + 127u - kDScale) << 20);
}

__device__ __forceinline__ float ArF32::from(double v) { return df_split(v).hi; }
__device__ __forceinline__ float ArF32::from_pivot(double v) { return df_split_checked(v).hi; }
__device__ __forceinline__ void ArF32::to(double& dst, float v) { dst = f32_widen_unscaled(v); }
template <bool kChk>
__device__ __forceinline__ void ArF32::row(double a, double b, double c, double d, float& A,
                                           float& B, float& C, float& D, RowChk& k) {
  df64 pa, pb, pc, pd;
  split_row<kChk>(a, b, c, d, pa, pb, pc, pd, k);
  A = pa.hi; B = pb.hi; C = pc.hi; D = pd.hi;
}
__device__ __forceinline__ bool ArF32::out_bad(double v) { return x_out_of_range_f64(v); }
__device__ __forceinline__ bool ArF64::out_bad(double v) { return x_out_of_range_f64(v); }

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
  __device__ __forceinline__ static void to(double& dst, T v) { dst = df_to_double(v.hi, v.lo); }
  __device__ __forceinline__ static void to(float2& dst, T v) { dst = make_float2(v.hi, v.lo); }

  // a row of fp64 inputs scaled by its diagonal's power of two (split_row);
  // reduced rows (float2 pairs, already of unit scale) as they are
  template <bool kChk>
  __device__ __forceinline__ static void row(double a, double b, double c, double d, T& A, T& B,
                                             T& C, T& D, RowChk& k) {
    split_row<kChk>(a, b, c, d, A, B, C, D, k);
  }
  template <bool kChk>
  __device__ __forceinline__ static void row(float2 a, float2 b, float2 c, float2 d, T& A,
                                             T& B, T& C, T& D, RowChk&) {
    A = from(a); B = from(b); C = from(c); D = from(d);
  }
  __device__ __forceinline__ static bool out_bad(double v) { return x_out_of_range_df(v); }
  __device__ __forceinline__ static bool out_bad(float2) { return false; }
  static constexpr bool kSkipChain = false;
  __device__ __forceinline__ static bool chain_small(T x) { return fabsf(x.hi) < 0x1p-60f; }
  __device__ __forceinline__ static bool mag_le(T c, T beta) {
    return fabsf(c.hi) <= fabsf(beta.hi);
  }
};

}  // namespace tps
