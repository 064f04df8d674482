// Double-float ("df64") arithmetic: a real number carried as an unevaluated
// sum hi + lo of two floats (about 48 significant bits).  GB300 runs FP32 FMA
// about 54x faster than FP64 FMA, so the FP64-class parts of the solver (outer
// Krylov, its operator, the coarsest solve) use this representation instead
// of the FP64 pipe.
//
// Building blocks are the classical error-free transformations: Knuth's
// TwoSum and Dekker's FastTwoSum for sums, and the FMA-based TwoProduct for
// products (the product error a*b - fl(a*b) is exactly fma(a, b, -fl(a*b))).
// Addition is the "sloppy" double-float add (one TwoSum on the high parts,
// then renormalisation), whose error bound has the same form as an IEEE
// addition with a 48-bit significand.  The __fadd_rn / __fmul_rn intrinsics
// keep the compiler from contracting these steps into FMAs.
//
// Storage: a real df64 is a float2 (x = hi, y = lo); a complex df64 is a
// float4 (x = re.hi, y = re.lo, z = im.hi, w = im.lo), 16 bytes like complex128.
#pragma once
#include <cuda_runtime.h>

namespace ehs {

struct dfr {
  float hi, lo;
};

__device__ __forceinline__ dfr df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return {s, e};
}
__device__ __forceinline__ dfr df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}
__device__ __forceinline__ dfr df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ dfr df_add(dfr a, dfr b) {
  const dfr s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfr df_neg(dfr a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfr df_sub(dfr a, dfr b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfr df_mul(dfr a, dfr b) {
  const dfr p = df_two_prod(a.hi, b.hi);
  return df_fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ dfr df_mulf(dfr a, float b) {
  const dfr p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ dfr df_from_f(float a) { return {a, 0.0f}; }
__device__ __forceinline__ dfr df_from_d(double a) {
  const float hi = __double2float_rn(a);
  return {hi, __double2float_rn(a - (double)hi)};
}
__device__ __forceinline__ double df_to_d(dfr a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfr df_zero() { return {0.0f, 0.0f}; }

// complex df64, stored as a float4 (re.hi, im.hi, re.lo, im.lo): the high parts and the low
// parts of the two components each sit in one aligned register pair after a load, the
// operand form of the paired FP32 instructions (dacc2 below)
struct dfc {
  dfr re, im;
};
__device__ __forceinline__ dfc dfc_ld(const float4* p) {
  const float4 v = __ldg(p);
  return {{v.x, v.z}, {v.y, v.w}};
}
__device__ __forceinline__ dfc dfc_ldv(const float4* p) {   // plain (non-__ldg) load
  const float4 v = *p;
  return {{v.x, v.z}, {v.y, v.w}};
}
__device__ __forceinline__ void dfc_st(float4* p, dfc a) { *p = make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ dfc dfc_zero() { return {df_zero(), df_zero()}; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// a * b with b a single-precision complex
__device__ __forceinline__ dfc dfc_mulf(dfc a, float2 b) {
  return {df_sub(df_mulf(a.re, b.x), df_mulf(a.im, b.y)), df_add(df_mulf(a.re, b.y), df_mulf(a.im, b.x))};
}
// conj(a) * b
__device__ __forceinline__ dfc dfc_cmul(dfc a, dfc b) {
  return {df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dfc dfc_scale(dfc a, dfr s) { return {df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ dfc dfc_scalef(dfc a, float s) { return {df_mulf(a.re, s), df_mulf(a.im, s)}; }
__device__ __forceinline__ dfc dfc_from_f2(float2 z) { return {df_from_f(z.x), df_from_f(z.y)}; }
__device__ __forceinline__ float2 dfc_to_f2(dfc a) {
  return make_float2(__fadd_rn(a.re.hi, a.re.lo), __fadd_rn(a.im.hi, a.im.lo));
}
__device__ __forceinline__ dfc dfc_from_d2(double2 z) { return {df_from_d(z.x), df_from_d(z.y)}; }
__device__ __forceinline__ double2 dfc_to_d2(dfc a) { return make_double2(df_to_d(a.re), df_to_d(a.im)); }

// Compensated sums of products (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, algorithm Dot2): a running FP32 sum s
// whose TwoSum rounding errors, the TwoProduct errors of each product and the
// df64 cross terms hi*lo + lo*hi all go into a second FP32 term c, added back
// once at the end.  The result is as accurate as a sum carried in twice the
// working precision (the same class as df64), with about a third of the
// operations of a renormalised df64 multiply-add per term.
struct dacc {
  float s, c;
};
__device__ __forceinline__ dacc dacc_zero() { return {0.0f, 0.0f}; }
// a += x * y
__device__ __forceinline__ void dacc_fma(dacc& a, dfr x, dfr y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
  const float t = __fadd_rn(a.s, p);
  const float bb = __fadd_rn(t, -a.s);
  const float sg = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(t, -bb)), __fadd_rn(p, -bb));
  a.s = t;
  a.c = __fadd_rn(a.c, __fadd_rn(sg, pe));
}
// a -= x * y
__device__ __forceinline__ void dacc_fms(dacc& a, dfr x, dfr y) { dacc_fma(a, df_neg(x), y); }
__device__ __forceinline__ dfr dacc_val(dacc a) { return df_two_sum(a.s, a.c); }

struct dcacc {
  dacc re, im;
};
__device__ __forceinline__ dcacc dcacc_zero() { return {dacc_zero(), dacc_zero()}; }
// a += conj(x) * y
__device__ __forceinline__ void dcacc_cfma(dcacc& a, dfc x, dfc y) {
  dacc_fma(a.re, x.re, y.re);
  dacc_fma(a.re, x.im, y.im);
  dacc_fma(a.im, x.re, y.im);
  dacc_fms(a.im, x.im, y.re);
}
// a += x * y
__device__ __forceinline__ void dcacc_fma(dcacc& a, dfc x, dfc y) {
  dacc_fma(a.re, x.re, y.re);
  dacc_fms(a.re, x.im, y.im);
  dacc_fma(a.im, x.re, y.im);
  dacc_fma(a.im, x.im, y.re);
}
__device__ __forceinline__ dfc dcacc_val(dcacc a) { return {dacc_val(a.re), dacc_val(a.im)}; }

// The same compensated accumulation for the two components of a complex sum at
// once, lane 0 = real part, lane 1 = imaginary part, on the paired FP32
// instructions (__fmul2_rn, __ffma2_rn, __fadd2_rn: per lane the rounding of
// the scalar operation), so each lane performs dacc_fma's steps.  Operands come
// as (high, low) pairs of lane vectors.
struct dacc2 {
  float2 s, c;
};
__device__ __forceinline__ dacc2 dacc2_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
// a += x * y lane-wise (x = xh + xl, y = yh + yl)
__device__ __forceinline__ void dacc2_fma(dacc2& a, float2 xh, float2 xl, float2 yh, float2 yl) {
  const float2 p = __fmul2_rn(xh, yh);
  const float2 pe = __ffma2_rn(xh, yl, __ffma2_rn(xl, yh, __ffma2_rn(xh, yh, f2neg(p))));
  const float2 t = __fadd2_rn(a.s, p);
  const float2 bb = __fadd2_rn(t, f2neg(a.s));
  const float2 sg = __fadd2_rn(__fadd2_rn(a.s, f2neg(__fadd2_rn(t, f2neg(bb)))), __fadd2_rn(p, f2neg(bb)));
  a.s = t;
  a.c = __fadd2_rn(a.c, __fadd2_rn(sg, pe));
}
__device__ __forceinline__ dfc dacc2_val(dacc2 a) { return {df_two_sum(a.s.x, a.c.x), df_two_sum(a.s.y, a.c.y)}; }
// The lane vectors of one complex df64 value v: (re, im) and (im, re), high and low parts.
struct dfc2 {
  float2 h, l, sh, sl;
};
__device__ __forceinline__ dfc2 dfc2_of(dfc v) {
  return {make_float2(v.re.hi, v.im.hi), make_float2(v.re.lo, v.im.lo), make_float2(v.im.hi, v.re.hi),
          make_float2(v.im.lo, v.re.lo)};
}
// a += conj(x) * w, with wa = (w.re, -w.re) and wb = (w.im, w.im) (high, low parts) formed once
// per element: lane 0 sums x.re w.re + x.im w.im, lane 1 -x.im w.re + x.re w.im
__device__ __forceinline__ void dacc2_cfma(dacc2& a, const dfc2& x, float2 wah, float2 wal, float2 wbh, float2 wbl) {
  dacc2_fma(a, x.h, x.l, wah, wal);
  dacc2_fma(a, x.sh, x.sl, wbh, wbl);
}
// a += x * h, with ha = (h.re, h.re) and hb = (-h.im, h.im) (high, low parts): lane 0 sums
// x.re h.re - x.im h.im, lane 1 x.im h.re + x.re h.im
__device__ __forceinline__ void dacc2_mfma(dacc2& a, const dfc2& x, float2 hah, float2 hal, float2 hbh, float2 hbl) {
  dacc2_fma(a, x.h, x.l, hah, hal);
  dacc2_fma(a, x.sh, x.sl, hbh, hbl);
}

}  // namespace ehs
