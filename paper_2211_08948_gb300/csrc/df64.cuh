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

// Conversions between float64 and double-float by integer operations.  The
// float64 conversions (two roundings to float32 and a float64 subtraction,
// or two widenings and a float64 addition) run on GB300's float64 pipe,
// which makes the vector set-up and output kernels conversion-bound; these
// forms give the same values, bit for bit, from the bit patterns.
//
// df_split_pow2(x, e2) = df_from_double(x * 2^e2): hi = x rounded to float32
// (nearest, ties to even, on the 29 dropped fraction bits: the carry into
// the exponent field is the rounding overflow), lo = the remainder, an
// integer of at most 29 bits times a power of two, rounded to float32 by the
// integer conversion and scaled exactly.  For |x 2^e2| in [2^-60, 2^60); zero
// and every other value take the float64 conversions.
__device__ __forceinline__ df df_split_pow2(double x, int e2) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF) + e2;
  const unsigned int sg = (unsigned int)(u >> 32) & 0x80000000u;
  if (e < 1023 - 60 || e >= 1023 + 60) {
    if ((u << 1) == 0ull) return df_make(__uint_as_float(sg), 0.f);  // signed zero; its remainder +0
    const double y = e2 == 0 ? x : ldexp(x, e2);
    const float hi = __double2float_rn(y);
    return df_make(hi, __double2float_rn(y - (double)hi));
  }
  const unsigned long long f = u & 0xFFFFFFFFFFFFFull;       // 52 fraction bits
  const unsigned int top = (unsigned int)(f >> 29);          // the 23 kept
  const unsigned int low = (unsigned int)f & 0x1FFFFFFFu;    // the 29 dropped
  const unsigned int up = (low > 0x10000000u) | ((low == 0x10000000u) & (top & 1u));
  const unsigned int hb = (((unsigned int)(e - 1023 + 127)) << 23) + top + up;
  const int r = (int)low - (int)(up << 29);                  // x - hi in units of 2^(e - 1075)
  const float lo = __int2float_rn(r) * __uint_as_float((unsigned int)(e - 1075 + 127) << 23);
  return df_make(__uint_as_float(hb | sg), (sg && r != 0) ? -lo : lo);  // an exact remainder is +0
}

// float32 -> float64 times 2^e2 from the bit pattern (normal floats and zero;
// subnormal, infinite and NaN values by the float64 conversion)
__device__ __forceinline__ double f_to_double_pow2(float v, int e2) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int E = (b >> 23) & 0xFFu;
  if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)(b >> 31) << 63));
  const int de = (int)E - 127 + 1023 + e2;  // the float64 exponent field
  if (E == 0u || E == 255u || de < 1 || de > 2046) return ldexp((double)v, e2);
  const unsigned long long d = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)de << 52) |
                               ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// df_to_double(a) * 2^e2: both parts widened exactly, one float64 addition
// (exact: the parts of a normalised pair span at most 48 bits)
__device__ __forceinline__ double df_to_double_pow2(df a, int e2) {
  return f_to_double_pow2(a.hi, e2) + f_to_double_pow2(a.lo, e2);
}

__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
#endif
