// xg_df.cuh -- double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2,
// 48 significant bits (unit roundoff 2^-48 ~ 3.6e-15).  GB300 executes FP32
// FMAs 64x faster than FP64 ones (2 DFMA vs 128 FFMA per clock per SM), so
// FP64-accurate arithmetic built from error-free float transformations is
// several times faster than native FP64 here.  The building blocks are the
// published ones:
//   * TwoSum (Knuth, TAOCP vol. 2): s + e = a + b exactly, 6 flops;
//   * FastTwoSum (Dekker 1971): the same when |a| >= |b|, 3 flops;
//   * TwoProduct with an FMA: p + e = a b exactly, 2 flops;
//   * double-word addition and multiplication as in Dekker (1971) and the
//     "accurate" addition of Hida, Li & Bailey's double-double library;
//   * compensated dot products (Ogita, Rump & Oishi 2005, "Dot2"): the high
//     parts are summed with TwoSum, every rounding error and cross term is
//     gathered in a float correction, so the result is as accurate as if
//     computed in twice the working precision.
// The _rn intrinsics keep the compiler from contracting the error-free
// sequences into FMAs (which would break them).
#pragma once

#include <cuda_runtime.h>

namespace xg {

struct df {
  float h, l;
};

__device__ __forceinline__ df df_of(float h) { return {h, 0.0f}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

// accurate double-word addition
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e, t, f;
  two_sum(a.h, b.h, s, e);
  two_sum(a.l, b.l, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return {s, e};
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// double-word addition without the second TwoSum: accurate when the
// operands do not nearly cancel (e.g. |b| < |a|/2, or equal signs)
__device__ __forceinline__ df df_add_nc(df a, df b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  fast_two_sum(s, e, s, e);
  return {s, e};
}

// double-word + float
__device__ __forceinline__ df df_add_f(df a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  e = __fadd_rn(e, a.l);
  fast_two_sum(s, e, s, e);
  return {s, e};
}

// double-word product (the l*l term is below the working precision)
__device__ __forceinline__ df df_mul(df a, df b) {
  float p, e;
  two_prod(a.h, b.h, p, e);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  fast_two_sum(p, e, p, e);
  return {p, e};
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p, e;
  two_prod(a.h, b, p, e);
  e = __fmaf_rn(a.l, b, e);
  fast_two_sum(p, e, p, e);
  return {p, e};
}

// multiplication by a power of two is exact
__device__ __forceinline__ df df_scale2(df a, float two_k) {
  return {__fmul_rn(a.h, two_k), __fmul_rn(a.l, two_k)};
}

// 1/a for a > 0: float reciprocal r0, residual e = 1 - a r0 (|e| <~ 2^-23,
// formed exactly up to 2^-48 from the exact product), then
// 1/a = r0 (1 + e + e^2 + ...) truncated after e^2 (e^3 < 2^-69).
__device__ __forceinline__ df df_rcp(df a) {
  const float r0 = __frcp_rn(a.h);
  float p, pe;
  two_prod(a.h, r0, p, pe);
  float e = __fsub_rn(1.0f, p);              // exact: p is within 2^-23 of 1
  e = __fsub_rn(e, pe);
  e = __fmaf_rn(-a.l, r0, e);
  const float t = __fmaf_rn(e, e, e);
  float s, c;
  fast_two_sum(r0, __fmul_rn(r0, t), s, c);
  return {s, c};
}

// Compensated dot-product accumulator (Dot2): value = s + c.
struct dacc {
  float s, c;
};

__device__ __forceinline__ dacc dacc_from(df t) { return {t.h, t.l}; }

__device__ __forceinline__ dacc dacc_prod(df d, df f) {
  dacc A;
  two_prod(d.h, f.h, A.s, A.c);
  A.c = __fmaf_rn(d.h, f.l, __fmaf_rn(d.l, f.h, A.c));
  return A;
}

// A += d f
__device__ __forceinline__ void dacc_fma(dacc& A, df d, df f) {
  float p, e, s, q;
  two_prod(d.h, f.h, p, e);
  two_sum(A.s, p, s, q);
  A.s = s;
  A.c = __fadd_rn(A.c, __fadd_rn(q, __fmaf_rn(d.h, f.l, __fmaf_rn(d.l, f.h, e))));
}

// A += t
__device__ __forceinline__ void dacc_add(dacc& A, df t) {
  float s, q;
  two_sum(A.s, t.h, s, q);
  A.s = s;
  A.c = __fadd_rn(A.c, __fadd_rn(q, t.l));
}

__device__ __forceinline__ df dacc_value(dacc A) {
  float s, e;
  two_sum(A.s, A.c, s, e);
  return {s, e};
}

__device__ __forceinline__ bool df_nonfinite(df a) {
  return (__float_as_uint(a.h) & 0x7f800000u) == 0x7f800000u;
}

// conversions (FP64 pipe; used only when data enters or leaves the library)
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

}  // namespace xg
