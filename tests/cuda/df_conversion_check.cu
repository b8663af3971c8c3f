// The integer conversions of df64.cuh (df_split_pow2, df_to_double_pow2)
// against the float64 conversions they replace, bit for bit, on seeded
// values: random bit patterns over a wide exponent band, ties and near-ties
// of the rounding to float32 (with the carry into the exponent), exact
// float32 values, zeros of both signs, tiny, huge and subnormal values, and
// uniform values, each with a power-of-two scale 2^e2, e2 in [-10, 10].
// Prints the mismatch count; exit status 1 on any mismatch.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "df64.cuh"
__device__ unsigned long long mix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull; z = (z ^ (z >> 27)) * 0x94D049BB133111EBull; return z ^ (z >> 31);
}
__global__ void check(unsigned long long n, unsigned long long seed, unsigned long long* bad, unsigned long long* first) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix(seed * 0x100000001ull + i);
    double x;
    const int kind = (int)(z & 7);
    if (kind < 3) {             // random bit patterns in a wide exponent band
      const unsigned long long ex = 1023 - 80 + ((z >> 8) % 160);
      x = __longlong_as_double((long long)(((z >> 3) & 0x800FFFFFFFFFFFFFull) | (ex << 52)));
    } else if (kind == 3) {     // ties and near-ties of the hi rounding
      const unsigned long long ex = 1023 - 30 + ((z >> 8) % 60);
      unsigned long long f = (z >> 16) & 0xFFFFFFFFFFFFFull;
      f = (f & ~0x1FFFFFFFull) | (((z >> 40) & 3) == 0 ? 0x10000000ull : ((z >> 40) & 3) == 1 ? 0x0FFFFFFFull : 0x10000001ull);
      if ((z >> 45) & 1) f |= 0xFFFFFE0000000ull;  // all kept bits set: the carry case
      x = __longlong_as_double((long long)((((z >> 50) & 1ull) << 63) | (ex << 52) | f));
    } else if (kind == 4) {     // exact float32 values
      x = (double)__uint_as_float((unsigned int)(z & 0x807FFFFFu) | ((unsigned int)(100 + ((z >> 32) % 56)) << 23));
    } else if (kind == 5) {     // zero, tiny, huge, subnormal, special
      const double sp[8] = {0.0, -0.0, 1e-300, -3e-30, 1e30, 4.9e-324, 1e300, 5e-20};
      x = sp[(z >> 8) & 7];
    } else {                    // uniform in [-0.5, 0.5)
      x = ((double)(z >> 11) * 0x1.0p-53) - 0.5;
    }
    const int e2 = (int)((z >> 56) % 21) - 10;
    const double xs = ldexp(x, e2);
    const float hi = __double2float_rn(xs);
    const float lo = __double2float_rn(xs - (double)hi);
    const df a = df_split_pow2(x, e2);
    bool ok = __float_as_uint(a.hi) == __float_as_uint(hi) && __float_as_uint(a.lo) == __float_as_uint(lo);
    // the way back: (hi + lo) 2^-e2
    const double back = ((double)hi + (double)lo) * ldexp(1.0, -e2);
    const double b2 = df_to_double_pow2(df_make(hi, lo), -e2);
    ok = ok && __double_as_longlong(back) == __double_as_longlong(b2);
    if (!ok && atomicAdd(bad, 1ull) == 0ull) *first = i;
  }
}
int main() {
  unsigned long long *bad, *first;
  cudaMallocManaged(&bad, 8); cudaMallocManaged(&first, 8);
  *bad = 0; *first = 0;
  for (unsigned long long seed = 1; seed <= 4; ++seed) check<<<152 * 8, 256>>>(1ull << 25, seed, bad, first);
  cudaDeviceSynchronize();
  printf("checked %llu values, mismatches %llu (first index %llu), %s\n", 4ull << 25, *bad, *first,
         cudaGetErrorString(cudaGetLastError()));
  return *bad != 0;
}
