// df.cuh -- double-float arithmetic on the float32 pipe.
//
// A value is carried as an unevaluated sum h + l of two float32 numbers with
// |l| <= ulp(h) / 2, which holds about 48 significant bits. The building
// blocks are the error-free transformations of floating-point arithmetic:
//   two_sum   (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   fast_sum  (Dekker 1971), the same when |a| >= |b|;
//   two_prod  (with a fused multiply-add): p + e = a * b exactly.
// Every operation is written with the _rn intrinsics, which the compiler
// never fuses or reorders, so the transformations stay exact.
//
// On this GPU the float64 pipe issues two operations per SM and clock
// against 128 on the float32 pipe, so a double-float add (about 11 float32
// operations) or multiply (about 6) costs a small fraction of one float64
// operation's pipe time. Conversions from and to the float64 masters in
// memory take one float64 add each.
#pragma once

#include <cuda_runtime.h>

#include "surfmd.cuh"

namespace surfmd {

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }

// a + b with absolute error about 2^-46 (|a| + |b|) (the low parts are added
// after the high parts' exact sum).
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return df_fast_sum(s.h, s.l);
}

__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

// a + f (f a float32 value)
__device__ __forceinline__ DF df_add_f(DF a, float f) {
  DF s = df_two_sum(a.h, f);
  s.l = __fadd_rn(s.l, a.l);
  return df_fast_sum(s.h, s.l);
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF p = df_two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return df_fast_sum(p.h, p.l);
}

// a * f (f a float32 value)
__device__ __forceinline__ DF df_mul_f(DF a, float f) {
  DF p = df_two_prod(a.h, f);
  p.l = __fmaf_rn(a.l, f, p.l);
  return df_fast_sum(p.h, p.l);
}

// 2^k scaling is exact
__device__ __forceinline__ DF df_scale2(DF a, float two_pow) { return {__fmul_rn(a.h, two_pow), __fmul_rn(a.l, two_pow)}; }

__device__ __forceinline__ DF df_dot3(const DF a[3], const DF b[3]) {
  return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}

// sqrt(a), a > 0: one Newton correction of the float32 root (Karp and
// Markstein's form): h = sqrt(a.h), l = (a - h^2) / (2h).
__device__ __forceinline__ DF df_sqrt(DF a) {
  const float h = __fsqrt_rn(a.h);
  const DF hh = df_two_prod(h, h);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, hh.h), hh.l), a.l);
  return df_fast_sum(h, __fmul_rn(r, __fdividef(0.5f, h)));
}

// a / b, b != 0: the float32 quotient plus one correction from the
// double-float remainder a - q b.
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float rb = __frcp_rn(b.h);
  const float q = __fmul_rn(a.h, rb);
  const DF r = df_sub(a, df_mul_f(b, q));
  return df_fast_sum(q, __fmul_rn(r.h, rb));
}

}  // namespace surfmd
