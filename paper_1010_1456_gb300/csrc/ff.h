// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 retires about two FP64 FMAs per clock per SM but 128 FP32 FMAs, so
// FP64-accurate FFT butterflies run faster as float-float on the FP32 pipes.
// The building blocks are the classical error-free transformations:
//   TwoSum (Knuth):        s = a + b exactly as s + e;
//   FastTwoSum (Dekker):   the same when |a| >= |b|;
//   TwoProduct with FMA:   a * b = p + e, e = fma(a, b, -p).
// Every operation uses the __f*_rn intrinsics so the compiler cannot
// contract or reassociate them (contraction would break the exactness of
// the error terms).  The addition is the "sloppy" variant: its error is
// bounded by about 2^-47 (|a| + |b|), which is the bound an FFT's error
// analysis uses anyway.
#pragma once

#include <cuda_runtime.h>

namespace aim {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff{s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, e);
}

// Addition without the closing renormalisation: hi is the rounded sum of the
// high parts and lo collects that rounding error plus both low parts, so
// hi + lo still carries the sum to about 2^-47 (|a| + |b|) but |lo| may
// exceed ulp(hi)/2 by a few units.  Later TwoSum/TwoProduct steps accept
// such pairs; used inside FFT butterflies, where every value feeds further
// arithmetic.
__device__ __forceinline__ ff ff_add_lazy(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_sub_lazy(ff a, ff b) { return ff_add_lazy(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

// a * b - c * d and a * d + b * c style fused forms: one renormalisation for
// the sum of two products (used by the complex product).
__device__ __forceinline__ ff ff_dot2(ff a, ff b, ff c, ff d) {
  // a*b + c*d
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float p2 = __fmul_rn(c.hi, d.hi);
  const ff s = ff_two_sum(p1, p2);
  float e = __fmaf_rn(a.hi, b.hi, -p1);
  e = __fadd_rn(e, __fmaf_rn(c.hi, d.hi, -p2));
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fmaf_rn(c.hi, d.lo, e);
  e = __fmaf_rn(c.lo, d.hi, e);
  e = __fadd_rn(e, s.lo);
  return ff_fast_two_sum(s.hi, e);
}

// acc + a * b with one closing renormalisation: the product's rounding
// error is recovered with FMA and carried in the low part, so the result is
// good to about 2^-47 (|acc| + |a b|).
__device__ __forceinline__ ff ff_mad(ff a, ff b, ff acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const ff s = ff_two_sum(acc.hi, p);
  const float t = __fadd_rn(__fadd_rn(s.lo, acc.lo), e);
  return ff_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ ff ff_from_double(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  return ff{hi, lo};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Complex float-float, stored as float4 (re.hi, re.lo, im.hi, im.lo).
struct cff {
  ff re, im;
};

}  // namespace aim
