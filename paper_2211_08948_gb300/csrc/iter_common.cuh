// Device code shared by the iteration kernels (Newton-Leja, power iteration,
// Arnoldi): precision traits, element loads/stores in each storage format,
// the three 5-point stencil Jacobians, and the deterministic last-block
// reduction of per-block partial sums.
#pragma once
#include <type_traits>

#include "phix_internal.h"

namespace phix {

// ---------------------------------------------------------------------------
// Precision traits: storage T (one element), vector pair T2, iteration
// arithmetic C, stencil arithmetic CJ, state storage S, accumulators.
// ---------------------------------------------------------------------------
template <int P>
struct Tr;
template <>
struct Tr<P_FP64> {
  using T = double;
  using T2 = double2;
  using C = double;
  using CJ = double;
  using S = double;
  using S2 = double2;
  using AccN = double;  // Newton norms
  using AccP = double;  // power-iteration norm (sets the interval: full precision)
};
template <>
struct Tr<P_DF64> {
  using T = float2;
  using T2 = float4;
  using C = df;
  using CJ = df;
  using S = float2;
  using S2 = float4;
  using AccN = float;
  using AccP = df;
};
template <>
struct Tr<P_FP32JV> {
  using T = float2;
  using T2 = float4;
  using C = df;
  using CJ = float;
  using S = float;
  using S2 = float2;
  using AccN = float;
  using AccP = df;
};
template <>
struct Tr<P_FP32> {
  using T = float;
  using T2 = float2;
  using C = float;
  using CJ = float;
  using S = float;
  using S2 = float2;
  using AccN = float;
  using AccP = float;
};

// ---- element conversions ----------------------------------------------------
__device__ __forceinline__ double cv(double x) { return x; }
__device__ __forceinline__ df cv(float2 x) { return df_make(x.x, x.y); }
__device__ __forceinline__ float cv(float x) { return x; }

__device__ __forceinline__ void st1(double* p, double x) { *p = x; }
__device__ __forceinline__ void st1(float2* p, df x) { *p = make_float2(x.hi, x.lo); }
__device__ __forceinline__ void st1(float* p, float x) { *p = x; }

__device__ __forceinline__ void st2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void st2(float2* p, df a, df b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}
__device__ __forceinline__ void st2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}

// read-only loads (y_in, state) through the non-coherent path
__device__ __forceinline__ double ldr1(const double* p) { return __ldg(p); }
__device__ __forceinline__ df ldr1(const float2* p) { return cv(__ldg(p)); }
__device__ __forceinline__ float ldr1(const float* p) { return __ldg(p); }
__device__ __forceinline__ void ldr2(const double* p, double& a, double& b) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  a = t.x;
  b = t.y;
}
__device__ __forceinline__ void ldr2(const float2* p, df& a, df& b) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  a = df_make(t.x, t.y);
  b = df_make(t.z, t.w);
}
__device__ __forceinline__ void ldr2(const float* p, float& a, float& b) {
  float2 t = __ldg(reinterpret_cast<const float2*>(p));
  a = t.x;
  b = t.y;
}
// loads of the Newton basis y: through the non-coherent path (COH = 0) when
// every launch is one iteration, through L2 (COH = 1) in a persistent chain,
// where other blocks rewrite the same addresses between iterations
template <int COH>
__device__ __forceinline__ double ldy1(const double* p) {
  if constexpr (COH) return __ldcg(p); else return __ldg(p);
}
template <int COH>
__device__ __forceinline__ df ldy1(const float2* p) {
  if constexpr (COH) return cv(__ldcg(p)); else return cv(__ldg(p));
}
template <int COH>
__device__ __forceinline__ float ldy1(const float* p) {
  if constexpr (COH) return __ldcg(p); else return __ldg(p);
}
template <int COH>
__device__ __forceinline__ void ldy2(const double* p, double& a, double& b) {
  double2 t = COH ? __ldcg(reinterpret_cast<const double2*>(p)) : __ldg(reinterpret_cast<const double2*>(p));
  a = t.x;
  b = t.y;
}
template <int COH>
__device__ __forceinline__ void ldy2(const float2* p, df& a, df& b) {
  float4 t = COH ? __ldcg(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
  a = df_make(t.x, t.y);
  b = df_make(t.z, t.w);
}
template <int COH>
__device__ __forceinline__ void ldy2(const float* p, float& a, float& b) {
  float2 t = COH ? __ldcg(reinterpret_cast<const float2*>(p)) : __ldg(reinterpret_cast<const float2*>(p));
  a = t.x;
  b = t.y;
}

// read-write loads (accumulators)
__device__ __forceinline__ double ldw1(const double* p) { return *p; }
__device__ __forceinline__ df ldw1(const float2* p) { return cv(*p); }
__device__ __forceinline__ float ldw1(const float* p) { return *p; }
__device__ __forceinline__ void ldw2(const double* p, double& a, double& b) {
  double2 t = *reinterpret_cast<const double2*>(p);
  a = t.x;
  b = t.y;
}
__device__ __forceinline__ void ldw2(const float2* p, df& a, df& b) {
  float4 t = *reinterpret_cast<const float4*>(p);
  a = df_make(t.x, t.y);
  b = df_make(t.z, t.w);
}
__device__ __forceinline__ void ldw2(const float* p, float& a, float& b) {
  float2 t = *reinterpret_cast<const float2*>(p);
  a = t.x;
  b = t.y;
}

// stencil arithmetic from iteration arithmetic and back
__device__ __forceinline__ double to_cj(double x, double) { return x; }
__device__ __forceinline__ df to_cj(df x, df) { return x; }
__device__ __forceinline__ float to_cj(df x, float) { return x.hi; }
__device__ __forceinline__ float to_cj(float x, float) { return x; }
__device__ __forceinline__ double from_cj(double x, double) { return x; }
__device__ __forceinline__ df from_cj(df x, df) { return x; }
__device__ __forceinline__ df from_cj(float x, df) { return df_make(x, 0.f); }
__device__ __forceinline__ float from_cj(float x, float) { return x; }

// a * b + c in each arithmetic
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df mad(df a, df b, df c) { return df_fma(a, b, c); }

// squares for the norms
__device__ __forceinline__ void acc_sq(double& a, double x) { a = fma(x, x, a); }
__device__ __forceinline__ void acc_sq(float& a, df x) { a = fmaf(x.hi, x.hi, a); }
__device__ __forceinline__ void acc_sq(float& a, float x) { a = fmaf(x, x, a); }
__device__ __forceinline__ void acc_sq(df& a, df x) { a = df_fma(x, x, a); }

__device__ __forceinline__ double acc_to_double(double a) { return a; }
__device__ __forceinline__ double acc_to_double(float a) { return (double)a; }
__device__ __forceinline__ double acc_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df shfl_down(df v, int o) {
  return df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ float acc_add(float a, float b) { return a + b; }
__device__ __forceinline__ df acc_add(df a, df b) { return df_add(a, b); }

template <typename A>
__device__ __forceinline__ A acc_zero();
template <>
__device__ __forceinline__ double acc_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float acc_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ df acc_zero<df>() { return df_make(0.f, 0.f); }

// Deterministic two-level reduction of NV accumulators: each block reduces its
// values (warp shuffles, warps in order) into partials[blockIdx.x * (KMAX+1) + j];
// the block that finishes last sums the partials in a fixed order.  GB300
// issues float64 at 1/64 of the float32 rate (a warp-wide float64 add holds the
// pipe ~64 cycles), so float and double-float accumulators keep their partials
// and the final tree in double-float (float2 bits in the double slots); float64
// accumulators keep float64 throughout.
template <typename A>
struct PartialsDF {
  static constexpr bool value = !std::is_same<A, double>::value;
};
__device__ __forceinline__ df acc_to_df(float a) { return df_make(a, 0.f); }
__device__ __forceinline__ df acc_to_df(df a) { return a; }

// true in the block that arrived last (all partials visible)
template <typename A, int NV>
__device__ bool block_partials_and_last(A (&acc)[NV], double* partials, unsigned int* count) {
  __shared__ double sred[THREADS / 32][KMAX + 1];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    A v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = acc_add(v, shfl_down(v, o));
    if (lane == 0) {
      if constexpr (PartialsDF<A>::value) {
        const df d = acc_to_df(v);
        reinterpret_cast<float2*>(&sred[warp][j])[0] = make_float2(d.hi, d.lo);
      } else {
        sred[warp][j] = v;
      }
    }
  }
  __syncthreads();
  if (tid < NV) {
    if constexpr (PartialsDF<A>::value) {
      df s = df_make(0.f, 0.f);
      for (int w = 0; w < THREADS / 32; ++w) s = df_add(s, cv(reinterpret_cast<const float2*>(&sred[w][tid])[0]));
      reinterpret_cast<float2*>(partials + (size_t)blockIdx.x * (KMAX + 1) + tid)[0] = make_float2(s.hi, s.lo);
    } else {
      double s = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) s += sred[w][tid];
      partials[(size_t)blockIdx.x * (KMAX + 1) + tid] = s;
    }
    __threadfence();  // the writers' partials visible before the arrival count
  }
  __syncthreads();
  if (tid == 0) {
    unsigned int t = atomicAdd(count, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// Persistent chains: the block's sums into partials[blockIdx.x * (KMAX+1) + j]
// (the same block-level reduction as above, no arrival count).
template <typename A, int NV>
__device__ void block_partials_only(A (&acc)[NV], double* partials) {
  __shared__ double sred[THREADS / 32][KMAX + 1];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    A v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = acc_add(v, shfl_down(v, o));
    if (lane == 0) {
      if constexpr (PartialsDF<A>::value) {
        const df d = acc_to_df(v);
        reinterpret_cast<float2*>(&sred[warp][j])[0] = make_float2(d.hi, d.lo);
      } else {
        sred[warp][j] = v;
      }
    }
  }
  __syncthreads();
  if (tid < NV) {
    if constexpr (PartialsDF<A>::value) {
      df s = df_make(0.f, 0.f);
      for (int w = 0; w < THREADS / 32; ++w) s = df_add(s, cv(reinterpret_cast<const float2*>(&sred[w][tid])[0]));
      reinterpret_cast<float2*>(partials + (size_t)blockIdx.x * (KMAX + 1) + tid)[0] = make_float2(s.hi, s.lo);
    } else {
      double s = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) s += sred[w][tid];
      partials[(size_t)blockIdx.x * (KMAX + 1) + tid] = s;
    }
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch (every block resident): arrival
// count and generation in device memory, both zero at the chain's start.
// The wait is bounded (2 s of %globaltimer): on expiry the barrier returns
// false in every thread of the block, which must then leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire(gen);  // the generation before this block arrives
    __threadfence();                         // the block's writes visible before its arrival
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire(gen) == g) {
        if (globaltimer_ns() - t0 > 2000000000ull) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Last block: totals[j] = sum over blocks of the partials (fixed order: up to
// four strided partials per thread loaded at once, then a tree).  The totals
// are valid in thread 0 only.  Double-float partials: the tree runs on warp
// shuffles (float32 lanes) with one barrier between the warp and block levels;
// the last block's reduction is on the critical path of every launch.
struct NoHook {
  __device__ void operator()() const {}
};
// `hook` runs in every thread just before the block barrier (work that the
// caller wants overlapped with the partials' latency and published by it).
// `nv` <= NV: only the first nv totals are formed (the others are returned as 0).
template <typename A, int NV, typename H = NoHook>
__device__ void reduce_partials(const double* partials, double (&tot)[NV], H hook = H{}, int nv = NV) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if constexpr (PartialsDF<A>::value) {
    constexpr int NW = THREADS / 32;
    __shared__ float2 swarp[NW][KMAX + 1];
    const int lane = tid & 31, warp = tid >> 5;
    df s[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = df_make(0.f, 0.f);
    const float2* pf = reinterpret_cast<const float2*>(partials);
    for (int b0 = tid; b0 < (int)gridDim.x; b0 += 4 * THREADS) {
      float2 v[4][NV];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = b0 + q * THREADS;
#pragma unroll
        for (int j = 0; j < NV; ++j)
          v[q][j] = (b < (int)gridDim.x && j < nv) ? __ldcg(pf + (size_t)b * (KMAX + 1) + j) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < NV; ++j)
          if (j < nv) s[j] = df_add(s[j], cv(v[q][j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j)
        if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < NV; ++j) swarp[warp][j] = make_float2(s[j].hi, s[j].lo);
    hook();
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = 0.0;
    if (warp == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) s[j] = lane < NW ? cv(swarp[lane][j]) : df_make(0.f, 0.f);
#pragma unroll
      for (int o = NW / 2; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NV; ++j)
          if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
      // float64 work in one thread only (a warp's float64 instruction holds the pipe ~64 cycles)
      if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j)
          if (j < nv) tot[j] = (double)s[j].hi + (double)s[j].lo;
    }
  } else {
    __shared__ double sfin[THREADS][KMAX + 1];
    double s[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += THREADS) {
#pragma unroll
      for (int j = 0; j < NV; ++j) s[j] += __ldcg(partials + (size_t)b * (KMAX + 1) + j);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) sfin[tid][j] = s[j];
    hook();
    __syncthreads();
    for (int w = THREADS / 2; w > 0; w >>= 1) {
      if (tid < w) {
#pragma unroll
        for (int j = 0; j < NV; ++j) sfin[tid][j] += sfin[tid + w][j];
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = sfin[0][j];
  }
}

// As reduce_partials for double-float partials, the totals returned as
// double-float pairs (valid in thread 0): no float64 instruction at all.
template <typename A, int NV>
__device__ void reduce_partials_df(const double* partials, df (&tot)[NV], int nv = NV) {
  static_assert(PartialsDF<A>::value, "double-float partials only");
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  constexpr int NW = THREADS / 32;
  __shared__ float2 swarp[NW][KMAX + 1];
  const int lane = tid & 31, warp = tid >> 5;
  df s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) s[j] = df_make(0.f, 0.f);
  const float2* pf = reinterpret_cast<const float2*>(partials);
  for (int b0 = tid; b0 < (int)gridDim.x; b0 += 4 * THREADS) {
    float2 v[4][NV];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b = b0 + q * THREADS;
#pragma unroll
      for (int j = 0; j < NV; ++j)
        v[q][j] = (b < (int)gridDim.x && j < nv) ? __ldcg(pf + (size_t)b * (KMAX + 1) + j) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < NV; ++j)
        if (j < nv) s[j] = df_add(s[j], cv(v[q][j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) swarp[warp][j] = make_float2(s[j].hi, s[j].lo);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = df_make(0.f, 0.f);
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] = lane < NW ? cv(swarp[lane][j]) : df_make(0.f, 0.f);
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j)
        if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = s[j];
  }
}

// a <= b for normalised double-float values (|lo| <= ulp(hi)/2)
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// Stop test of the Newton-Leja chain at iteration m (Sec. 2.2):
// |d_k[m]| ||y_m|| <= tol ||p_m^(k)|| for every k, compared as squares (no
// square root on the critical path between launches); tot holds the squared
// norms.
__device__ inline void leja_test(LejaCtl* ctl, int m, int K, int m_min, int m_max, double tol,
                          const double* dkd, const double* tot) {
  const double ny2 = tot[0];
  bool finite = isfinite(ny2);
  bool conv = (m >= m_min);
  const double tol2 = tol * tol;
  for (int k = 0; k < K; ++k) {
    const double np2 = tot[1 + k];
    ctl->psq[k] = np2;
    finite = finite && isfinite(np2);
    conv = conv && (dkd[k] * dkd[k] * ny2 <= tol2 * np2);
  }
  ctl->ysq = ny2;
  if (!finite) {
    ctl->status = PHIX_ENAN;
    ctl->iters = m;
    ctl->done = 1;
  } else if (conv) {
    ctl->status = PHIX_OK;
    ctl->iters = m;
    ctl->done = 1;
  } else if (m >= m_max) {
    ctl->status = PHIX_ENOTCONV;
    ctl->iters = m;
    ctl->done = 1;
  }
}

// The same test on double-float totals: ||y_m||^2 q_k <= ||p_m^(k)||^2 with
// q_k = (d_k[m] / tol)^2 from the parameter block (float32 instructions only;
// a decision differs from the float64 form only at a relative tie ~2^-47).
__device__ inline void leja_test_df(LejaCtl* ctl, int m, int K, int m_min, int m_max, const float2* qk,
                                    const df* tot) {
  const df ny2 = tot[0];
  bool finite = isfinite(ny2.hi);
  bool conv = (m >= m_min);
  for (int k = 0; k < K; ++k) {
    const df np2 = tot[1 + k];
    finite = finite && isfinite(np2.hi);
    conv = conv && df_le(df_mul(ny2, cv(qk[k])), np2);
  }
  if (!finite) {
    ctl->status = PHIX_ENAN;
    ctl->iters = m;
    ctl->done = 1;
  } else if (conv) {
    ctl->status = PHIX_OK;
    ctl->iters = m;
    ctl->done = 1;
  } else if (m >= m_max) {
    ctl->status = PHIX_ENOTCONV;
    ctl->iters = m;
    ctl->done = 1;
  }
}

// ---------------------------------------------------------------------------
// Stencils.  Each returns J*y at one point in the stencil arithmetic CJ.
// ---------------------------------------------------------------------------
template <typename CJ>
__device__ __forceinline__ CJ stencil_advdiff(const CJ (&k)[8], CJ e, CJ w, CJ n, CJ s, CJ c) {
  return k[0] * e + k[1] * w + k[2] * n + k[3] * s + k[4] * c;
}

// GS species u: ku = {x, y, C}; returns J_u, J_v together, given the state
// terms a1 = ga V^2, a2 = ga 2UV at the point.
template <typename CJ>
__device__ __forceinline__ void stencil_gs_a(const CJ (&k)[8], CJ ue, CJ uw, CJ un, CJ us, CJ uc, CJ ve, CJ vw,
                                             CJ vn, CJ vs, CJ vc, CJ a1, CJ a2, CJ& ju, CJ& jv) {
  ju = k[0] * (ue + uw) + k[1] * (un + us) + (k[2] - a1) * uc - a2 * vc;
  jv = k[3] * (ve + vw) + k[4] * (vn + vs) + a1 * uc + (k[5] + a2) * vc;
}
template <typename CJ>
__device__ __forceinline__ void stencil_gs(const CJ (&k)[8], CJ ga, CJ ue, CJ uw, CJ un, CJ us, CJ uc,
                                           CJ ve, CJ vw, CJ vn, CJ vs, CJ vc, CJ g1, CJ g2, CJ& ju,
                                           CJ& jv) {
  stencil_gs_a<CJ>(k, ue, uw, un, us, uc, ve, vw, vn, vs, vc, ga * g1, ga * g2, ju, jv);
}

// double-float forms: the products of each row summed as unnormalised pairs
template <>
__device__ __forceinline__ df stencil_advdiff<df>(const df (&k)[8], df e, df w, df n, df s, df c) {
  float p[5], q[5];
  df_prod(k[0], e, p[0], q[0]);
  df_prod(k[1], w, p[1], q[1]);
  df_prod(k[2], n, p[2], q[2]);
  df_prod(k[3], s, p[3], q[3]);
  df_prod(k[4], c, p[4], q[4]);
  return df_sum_pairs<5>(p, q);
}

template <>
__device__ __forceinline__ void stencil_gs_a<df>(const df (&k)[8], df ue, df uw, df un, df us, df uc, df ve, df vw,
                                                 df vn, df vs, df vc, df a1, df a2, df& ju, df& jv) {
  float p[4], q[4];
  df_prod(k[0], ue + uw, p[0], q[0]);
  df_prod(k[1], un + us, p[1], q[1]);
  df_prod(k[2] - a1, uc, p[2], q[2]);
  df_prod(df_neg(a2), vc, p[3], q[3]);
  ju = df_sum_pairs<4>(p, q);
  df_prod(k[3], ve + vw, p[0], q[0]);
  df_prod(k[4], vn + vs, p[1], q[1]);
  df_prod(a1, uc, p[2], q[2]);
  df_prod(k[5] + a2, vc, p[3], q[3]);
  jv = df_sum_pairs<4>(p, q);
}

template <typename CJ>
__device__ __forceinline__ CJ stencil_burgers(const CJ (&k)[8], CJ ga, CJ e, CJ w, CJ n, CJ s, CJ c,
                                              CJ Ue, CJ Uw, CJ Un, CJ Us, CJ Uc) {
  // nu lap y - (U_x + U_y) y - U (y_x + y_y), all centred
  CJ divU = k[3] * (Ue - Uw) + k[4] * (Un - Us);
  CJ dy = k[3] * (e - w) + k[4] * (n - s);
  return k[0] * (e + w) + k[1] * (n + s) + k[2] * c - ga * (divU * c + Uc * dy);
}


// ---------------------------------------------------------------------------
// Chain parameter block: PassParams | beta_d[M] | beta_f[M] | dk_d[KMAX][M] | dk_f[KMAX][M] | q_f[KMAX][M]
// (q = (d_k[m] / tol)^2 in double-float: the stop test without float64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ const PassParams* pp_of(const unsigned char* t) {
  return reinterpret_cast<const PassParams*>(t);
}
__device__ __forceinline__ const double* beta_d_of(const unsigned char* t, int M) {
  return reinterpret_cast<const double*>(t + sizeof(PassParams));
}
__device__ __forceinline__ const float2* beta_f_of(const unsigned char* t, int M) {
  return reinterpret_cast<const float2*>(t + sizeof(PassParams) + 8 * (size_t)M);
}
__device__ __forceinline__ const double* dk_d_of(const unsigned char* t, int M) {
  return reinterpret_cast<const double*>(t + sizeof(PassParams) + 16 * (size_t)M);
}
__device__ __forceinline__ const float2* dk_f_of(const unsigned char* t, int M) {
  return reinterpret_cast<const float2*>(t + sizeof(PassParams) + 16 * (size_t)M + 8 * (size_t)KMAX * M);
}
__device__ __forceinline__ const float2* q_f_of(const unsigned char* t, int M) {
  return reinterpret_cast<const float2*>(t + sizeof(PassParams) + 16 * (size_t)M + 16 * (size_t)KMAX * M);
}

// centre-coefficient indices that the Newton shift beta is folded into
template <int OP>
struct Centre;
template <>
struct Centre<PHIX_OP_ADVDIFF> {
  static constexpr int a = 4, b = -1;
};
template <>
struct Centre<PHIX_OP_GRAYSCOTT> {
  static constexpr int a = 2, b = 5;
};
template <>
struct Centre<PHIX_OP_BURGERS> {
  static constexpr int a = 2, b = -1;
};

// a coefficient in the arithmetic X, from its float64 / double-float forms
template <typename X>
__device__ __forceinline__ X coef(double d, float2 f);
template <>
__device__ __forceinline__ double coef<double>(double d, float2) { return d; }
template <>
__device__ __forceinline__ df coef<df>(double, float2 f) { return df_make(f.x, f.y); }
template <>
__device__ __forceinline__ float coef<float>(double, float2 f) { return f.x; }

// SplitMix64 (Steele, Lea & Flood 2014): x_i = seed + (i+1)*golden; 64-bit
// finaliser; the top 53 bits mapped to [-0.5, 0.5).  The power iteration's
// start vector, element i of the stream `seed`.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

}  // namespace phix
