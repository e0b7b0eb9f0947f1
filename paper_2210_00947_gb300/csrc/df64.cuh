// Double-float ("df64") arithmetic on the FP32 pipe: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant
// bits.  Built from error-free transformations: Knuth's TwoSum (The Art of
// Computer Programming vol. 2, 4.2.2), Dekker's FastTwoSum and the FMA form
// of Dekker's TwoProd (Dekker, "A floating-point technique for extending the
// available precision", 1971).  GB300 runs FP64 at 1/58 of the FP32 rate, so
// an FP64-accurate operation costs less as a handful of FP32 operations.
#pragma once

#include <cuda_runtime.h>

namespace mgar {

struct df {
  float hi, lo;
};

// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// s + e == a + b exactly, given |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e == a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_make(float h, float l) {
  df r;
  fast_two_sum(h, l, r.hi, r.lo);
  return r;
}

// a + b (sloppy form: error ~2^-46 of max(|a|, |b|))
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_make(s, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b
__device__ __forceinline__ df df_mul(df a, df b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_make(p, e);
}

// a * b for a float b
__device__ __forceinline__ df df_mulf(df a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = __fmaf_rn(a.lo, b, e);
  return df_make(p, e);
}

// 1 / sqrt(a), a > 0: an FP32 seed and two Newton steps y <- y + y (1 - a y^2) / 2
// with the residual 1 - a y^2 formed in df64 (each step doubles the correct bits)
__device__ __forceinline__ df df_rsqrt(df a) {
  df y{rsqrtf(a.hi), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df e = df_sub(df{1.f, 0.f}, df_mul(df_mul(a, y), y));
    y = df_add(y, df_mulf(y, 0.5f * e.hi));
  }
  return y;
}

// Order of normalised pairs (|lo| <= ulp(hi)/2): by the high words, then the
// low words.
__device__ __forceinline__ bool df_le(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ df df_max(df a, df b) { return df_le(a, b) ? b : a; }
__device__ __forceinline__ df df_min(df a, df b) { return df_le(a, b) ? a : b; }
__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? df_neg(a) : a; }

// conversions (the FP64 side costs one FP64 subtraction per value)
__host__ __device__ __forceinline__ df df_from_double(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace mgar
