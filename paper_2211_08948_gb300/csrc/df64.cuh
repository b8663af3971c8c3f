// Double-float ("df") arithmetic: a value is hi + lo with two float32 parts,
// |lo| <= ulp(hi)/2, giving ~48 significant bits.  GB300 issues float32 FMAs
// about 58x faster than float64 FMAs, so the memory-bound iteration kernels
// keep float64-class accuracy by computing in df.
//
// Error-free transforms (published methods):
//   TwoSum       Knuth, TAOCP vol. 2, 4.2.2 (6 flops, no magnitude condition)
//   FastTwoSum   Dekker 1971 (3 flops, needs |a| >= |b|)
//   TwoProd      exact product error via one fused multiply-add
// Every operation uses the __f*_rn intrinsics, which the compiler never
// contracts or reorders, so the transforms stay exact under -fmad=true.
#pragma once
#include <cuda_runtime.h>

struct df {
  float hi, lo;
};

__host__ __device__ inline df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// Split a double into hi + lo (host or device; device use costs two F2F).
__host__ __device__ inline df df_from_double(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return df_make(hi, lo);
}

__host__ __device__ inline double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

#ifdef __CUDACC__
__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

// a + b: TwoSum of the high parts, low parts added in float32, renormalised.
// Absolute error <= ~2^-47 (|a| + |b|).
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  float t = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b: TwoProd of the high parts plus the cross terms.
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * b + c: the product kept as an unnormalised pair, one renormalisation
// (15 flops instead of 7 + 11)
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// a * b as an unnormalised pair: p + e = a b to ~2^-47 |a b|
__device__ __forceinline__ void df_prod(df a, df b, float& p, float& e) {
  p = __fmul_rn(a.hi, b.hi);
  e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
}

// sum of N products given as unnormalised pairs: TwoSum chain over the high
// parts, all low parts and rounding errors summed in float32, renormalised
// once (absolute error ~2^-47 sum |p_i|, as for a chain of df_add)
template <int N>
__device__ __forceinline__ df df_sum_pairs(const float (&p)[N], const float (&e)[N]) {
  float s = p[0], err = e[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const df t = df_two_sum(s, p[i]);
    s = t.hi;
    err = __fadd_rn(err, __fadd_rn(t.lo, e[i]));
  }
  return df_fast_two_sum(s, err);
}

// multiplication by an exact power of two
__device__ __forceinline__ df df_scale2(df a, float p2) {
  return df_make(__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2));
}

__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
#endif
