// KIOPS-style Krylov kernels (Sec. 2.1 of the paper): Arnoldi with window-2
// incomplete orthogonalisation on the augmented matrix
//   A~ = [[A, eta B], [0, K]],  A = h J,  B = [b_p, ..., b_1],  K = shift,
// the small exponential exp(tau Hbar) e_1 of the (tridiagonal) Hessenberg
// matrix with the corrected-Krylov error estimate, and the combination of the
// basis into the substep result.
//
// The basis is kept unnormalised, V_i = s_i Zhat_i; the N part of Zhat_i is
// stored in the iteration precision (float64 or double-float), the p tail
// entries in float64 inside the control block.  Each Arnoldi step is two
// grid passes:
//   pass 1: z = A~ V_j (5-point stencil + the eta b columns), partial dots
//           <Zhat_j, z>, <Zhat_{j-1}, z> and ||z||^2;
//   pass 2: z <- z - h_jj V_j - h_{j-1,j} V_{j-1} in place, partial ||z||^2;
// the last block of each pass adds the tail terms, forms h_jj, h_{j-1,j},
// h_{j+1,j}, s_{j+1} and writes the coefficients of the next launch.
#include <algorithm>
#include "iter_common.cuh"

namespace phix {

namespace {

// dot products: float64, or double-float accumulation
__device__ __forceinline__ void acc_dot(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_dot(df& a, df x, df y) { a = df_fma(x, y, a); }

// accumulator of <z, z> in pass 1: float64 in the float64 path, float32 otherwise
template <typename A>
struct AccSq {
  using F = float;
};
template <>
struct AccSq<double> {
  using F = double;
};
__device__ __forceinline__ double acc_sq_f(double a, double z) { return fma(z, z, a); }
__device__ __forceinline__ float acc_sq_f(float a, df z) { return fmaf(z.hi, z.hi, a); }
template <typename A>
__device__ __forceinline__ A acc_from_f(typename AccSq<A>::F v);
template <>
__device__ __forceinline__ double acc_from_f<double>(double v) { return v; }
template <>
__device__ __forceinline__ df acc_from_f<df>(float v) { return df_make(v, 0.f); }

template <int P>
struct KTr;
template <>
struct KTr<P_FP64> {
  using T = double;
  using C = double;
  using S = double;
  using Acc = double;
};
template <>
struct KTr<P_DF64> {
  using T = float2;
  using C = df;
  using S = float2;
  using Acc = df;
};

struct ArnArgs {
  const void* zj;
  const void* zjm1;  // NULL for j = 0
  void* zout;        // slot j + 1
  const void* bz[KIOPS_PMAX];
  int bslot[KIOPS_PMAX];
  int nb;
  const void* st;
  KiopsCtl* kc;
  double* partials;
  int j, p, nx, ny, ntiles, tiles_x, nscaled;
  double h;
  double kJ[8];
};

// next pass-1 coefficients from s[j] (single thread)
__device__ void prepare_pass1(KiopsCtl* kc, int j, int p, double h, const double* kJ, int nscaled) {
  const double sj = kc->s[j];
  for (int i = 0; i < 8; ++i) {
    double v = i < nscaled ? kJ[i] * h * sj : kJ[i];
    kc->kd[i] = v;
    float hi = (float)v;
    kc->kf[i] = make_float2(hi, (float)(v - (double)hi));
  }
  const double g = h * sj;
  kc->gad = g;
  float gh = (float)g;
  kc->gaf = make_float2(gh, (float)(g - (double)gh));
  for (int t = 0; t < p; ++t) {
    double b = kc->eta * sj * kc->tail[j * KIOPS_PMAX + t];
    kc->bd[t] = b;
    float bh = (float)b;
    kc->bf[t] = make_float2(bh, (float)(b - (double)bh));
  }
}

__device__ __forceinline__ float2 split2d(double v) {
  float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

template <int P, int OP, int V>
__global__ void __launch_bounds__(THREADS) k_arn1(ArnArgs a) {
  using T = typename KTr<P>::T;
  using C = typename KTr<P>::C;
  using S = typename KTr<P>::S;
  using Acc = typename KTr<P>::Acc;
  constexpr int NC = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 1;
  KiopsCtl* kc = a.kc;
  if (__ldcg(&kc->stop)) return;
  C kk[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) kk[i] = coef<C>(__ldcg(&kc->kd[i]), __ldcg(&kc->kf[i]));
  const C ga = coef<C>(__ldcg(&kc->gad), __ldcg(&kc->gaf));
  C bw[KIOPS_PMAX];
#pragma unroll
  for (int b = 0; b < KIOPS_PMAX; ++b)
    bw[b] = b < a.nb ? coef<C>(__ldcg(&kc->bd[a.bslot[b]]), __ldcg(&kc->bf[a.bslot[b]])) : C{};

  Acc acc[3] = {acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>()};
  // <z, z> only sets the happy-breakdown threshold: float32 in the double-float path
  typename AccSq<Acc>::F zz = 0;
  const T* __restrict__ zj = static_cast<const T*>(a.zj);
  const T* __restrict__ zm = static_cast<const T*>(a.zjm1);
  T* __restrict__ zo = static_cast<T*>(a.zout);
  const S* __restrict__ st = static_cast<const S*>(a.st);
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;

  // a contiguous, balanced range of tiles per block (neighbouring tiles share
  // their halo rows in L1/L2; blocks differ by at most one tile)
  const int t_begin = (int)(((long long)blockIdx.x * a.ntiles) / gridDim.x);
  const int t_end = (int)(((long long)(blockIdx.x + 1) * a.ntiles) / gridDim.x);
  for (int tile = t_begin; tile < t_end; ++tile) {
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int iy = ty * TILE_Y + threadIdx.y;
    const int ix = (tx * 32 + threadIdx.x) * V;
    if (iy >= ny || ix >= nx) continue;
    const int iym = iy == 0 ? ny - 1 : iy - 1;
    const int iyp = iy == ny - 1 ? 0 : iy + 1;
    const int ixm = ix == 0 ? nx - 1 : ix - 1;
    const int ixp = (ix + V == nx) ? 0 : ix + V;
    const size_t row = (size_t)iy * nx, rowp = (size_t)iyp * nx, rowm = (size_t)iym * nx;
    C c[NC][V], nn[NC][V], ss[NC][V], we[NC], ea[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const T* b = zj + q * plane;
      if constexpr (V == 2) {
        ldr2(b + row + ix, c[q][0], c[q][1]);
        ldr2(b + rowp + ix, nn[q][0], nn[q][1]);
        ldr2(b + rowm + ix, ss[q][0], ss[q][1]);
      } else {
        c[q][0] = ldr1(b + row + ix);
        nn[q][0] = ldr1(b + rowp + ix);
        ss[q][0] = ldr1(b + rowm + ix);
      }
      we[q] = ldr1(b + row + ixm);
      ea[q] = ldr1(b + row + ixp);
    }
    // every load of the tile issued before its arithmetic: z_{j-1} for the
    // second dot and the augmented columns B t (sum_b bw_b b-copy_b)
    C cm[NC][V], zb[NC][V];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const size_t i0 = q * plane + row + ix;
      if (zm) {
        if constexpr (V == 2)
          ldr2(zm + i0, cm[q][0], cm[q][1]);
        else
          cm[q][0] = ldr1(zm + i0);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) cm[q][v] = C{};
      }
#pragma unroll
      for (int v = 0; v < V; ++v) zb[q][v] = C{};
#pragma unroll
      for (int bq = 0; bq < KIOPS_PMAX; ++bq) {
        if (bq < a.nb) {
          const T* bb = static_cast<const T*>(a.bz[bq]) + i0;
          if constexpr (V == 2) {
            C b0, b1;
            ldr2(bb, b0, b1);
            zb[q][0] = zb[q][0] + bw[bq] * b0;
            zb[q][1] = zb[q][1] + bw[bq] * b1;
          } else {
            zb[q][0] = zb[q][0] + bw[bq] * ldr1(bb);
          }
        }
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      C J[NC];
      if constexpr (OP == PHIX_OP_ADVDIFF) {
        C e = (v == V - 1) ? ea[0] : c[0][v + 1];
        C w = (v == 0) ? we[0] : c[0][v - 1];
        J[0] = stencil_advdiff<C>(kk, e, w, nn[0][v], ss[0][v], c[0][v]);
      } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
        C eu = (v == V - 1) ? ea[0] : c[0][v + 1];
        C wu = (v == 0) ? we[0] : c[0][v - 1];
        C ev = (v == V - 1) ? ea[NC - 1] : c[NC - 1][v + 1];
        C wv = (v == 0) ? we[NC - 1] : c[NC - 1][v - 1];
        C g1 = cv(__ldg(st + row + ix + v));
        C g2 = cv(__ldg(st + plane + row + ix + v));
        stencil_gs<C>(kk, ga, eu, wu, nn[0][v], ss[0][v], c[0][v], ev, wv, nn[NC - 1][v], ss[NC - 1][v],
                      c[NC - 1][v], g1, g2, J[0], J[NC - 1]);
      } else {
        C e = (v == V - 1) ? ea[0] : c[0][v + 1];
        C w = (v == 0) ? we[0] : c[0][v - 1];
        const int vx = ix + v;
        const int vxm = (v == 0) ? ixm : vx - 1;
        const int vxp = (v == V - 1) ? ixp : vx + 1;
        C Uc = cv(__ldg(st + row + vx));
        C Ue = cv(__ldg(st + row + vxp));
        C Uw = cv(__ldg(st + row + vxm));
        C Un = cv(__ldg(st + rowp + vx));
        C Us = cv(__ldg(st + rowm + vx));
        J[0] = stencil_burgers<C>(kk, ga, e, w, nn[0][v], ss[0][v], c[0][v], Ue, Uw, Un, Us, Uc);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const size_t idx = q * plane + row + ix + v;
        const C z = J[q] + zb[q][v];
        st1(zo + idx, z);
        acc_dot(acc[0], c[q][v], z);
        acc_dot(acc[1], cm[q][v], z);
        zz = acc_sq_f(zz, z);
      }
    }
  }

  acc[2] = acc_from_f<Acc>(zz);
  if (block_partials_and_last<Acc, 3>(acc, a.partials, &kc->count)) {
    double tot[3];
    reduce_partials<Acc, 3>(a.partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int j = a.j, p = a.p;
      const double sj = kc->s[j];
      const double* tj = kc->tail + j * KIOPS_PMAX;
      double tz[KIOPS_PMAX];
      for (int t = 0; t < p; ++t) tz[t] = (t + 1 < p) ? sj * tj[t + 1] : 0.0;
      double d1 = tot[0], d0 = tot[1], zz = tot[2];
      for (int t = 0; t < p; ++t) {
        d1 += tj[t] * tz[t];
        zz += tz[t] * tz[t];
        if (j >= 1) d0 += kc->tail[(j - 1) * KIOPS_PMAX + t] * tz[t];
      }
      const double hjj = sj * d1;
      const double hjm = j >= 1 ? kc->s[j - 1] * d0 : 0.0;
      kc->hd[j] = hjj;
      kc->hu[j] = hjm;
      kc->z0[j] = sqrt(zz);
      for (int t = 0; t < p; ++t) kc->tail[(j + 1) * KIOPS_PMAX + t] = tz[t];
      const double c1 = hjj * sj, c0 = j >= 1 ? hjm * kc->s[j - 1] : 0.0;
      kc->c1d = c1;
      kc->c0d = c0;
      kc->c1f = split2d(c1);
      kc->c0f = split2d(c0);
      if (!isfinite(hjj) || !isfinite(hjm) || !isfinite(zz)) {
        kc->status = PHIX_ENAN;
        kc->stop = 1;
      }
      kc->count = 0;
      __threadfence();
    }
  }
}

template <int P>
__global__ void __launch_bounds__(THREADS) k_arn2(ArnArgs a, size_t n) {
  using T = typename KTr<P>::T;
  using C = typename KTr<P>::C;
  using Acc = typename KTr<P>::Acc;
  KiopsCtl* kc = a.kc;
  if (__ldcg(&kc->stop)) return;
  const C c1 = coef<C>(__ldcg(&kc->c1d), __ldcg(&kc->c1f));
  const C c0 = coef<C>(__ldcg(&kc->c0d), __ldcg(&kc->c0f));
  const T* __restrict__ zj = static_cast<const T*>(a.zj);
  const T* __restrict__ zm = static_cast<const T*>(a.zjm1);
  T* __restrict__ zo = static_cast<T*>(a.zout);
  Acc acc[1] = {acc_zero<Acc>()};
  // element pairs (16-byte accesses; every vector starts 256-byte aligned), two
  // pairs per thread per trip so that six loads are in flight
  const size_t np = n / 2;
  const size_t t0 = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * THREADS;
  auto pair = [&](size_t q) {
    const size_t i = 2 * q;
    C w0, w1, a0, a1, b0 = C{}, b1 = C{};
    ldw2(zo + i, w0, w1);
    ldr2(zj + i, a0, a1);
    if (zm) ldr2(zm + i, b0, b1);
    C z0 = w0 - c1 * a0, z1 = w1 - c1 * a1;
    if (zm) {
      z0 = z0 - c0 * b0;
      z1 = z1 - c0 * b1;
    }
    st2(zo + i, z0, z1);
    acc_dot(acc[0], z0, z0);
    acc_dot(acc[0], z1, z1);
  };
  auto single = [&](size_t i) {
    C z = ldw1(zo + i) - c1 * ldr1(zj + i);
    if (zm) z = z - c0 * ldr1(zm + i);
    st1(zo + i, z);
    acc_dot(acc[0], z, z);
  };
  // basis slots lie N elements apart: with N odd every other slot is only
  // 8-byte aligned, and the pairs would be misaligned
  const bool vec = ((reinterpret_cast<uintptr_t>(zo) | reinterpret_cast<uintptr_t>(zj) |
                     reinterpret_cast<uintptr_t>(zm)) & 15) == 0;
  if (vec) {
    size_t q = t0;
    for (; q + stride < np; q += 2 * stride) {
      pair(q);
      pair(q + stride);
    }
    if (q < np) pair(q);
    if ((n & 1) && t0 == 0) single(n - 1);  // odd length: the last element
  } else {
    for (size_t i = t0; i < n; i += stride) single(i);
  }
  if (block_partials_and_last<Acc, 1>(acc, a.partials, &kc->count)) {
    double tot[1];
    reduce_partials<Acc, 1>(a.partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int j = a.j, p = a.p;
      double* tz = kc->tail + (j + 1) * KIOPS_PMAX;
      const double c1d = kc->c1d, c0d = kc->c0d;
      double nz = tot[0];
      for (int t = 0; t < p; ++t) {
        double v = tz[t] - c1d * kc->tail[j * KIOPS_PMAX + t];
        if (j >= 1) v -= c0d * kc->tail[(j - 1) * KIOPS_PMAX + t];
        tz[t] = v;
        nz += v * v;
      }
      const double hn = sqrt(nz);
      kc->hl[j] = hn;
      if (!isfinite(hn)) {
        kc->status = PHIX_ENAN;
        kc->stop = 1;
      } else if (hn <= 1e-12 * kc->z0[j]) {
        kc->stop = 1;  // happy breakdown: exact invariant subspace of dimension j+1
        kc->happy_m = j + 1;
      } else {
        kc->s[j + 1] = 1.0 / hn;
        kc->sf[j + 1] = split2d(1.0 / hn);
        prepare_pass1(kc, j + 1, p, a.h, a.kJ, a.nscaled);
      }
      kc->count = 0;
      __threadfence();
    }
  }
}

// F = exp(tau Hbar) e_1 for the tridiagonal Hbar (one CTA of 128 threads).
//
// Main method: Chebyshev expansion on [lo, hi], the exact range of the real
// parts of the field of values W(X), X = tau Hbar, i.e. the extreme
// eigenvalues of the symmetric part (X + X^T)/2 (Bendixson):
//   e^{c + r t} = e^{c + r} (I~_0(r) + 2 sum_k I~_k(r) T_k(t)),  I~_k = e^{-r} I_k,
// applied with the three-term recurrence to Y = (X - c I)/r, in S segments
// exp(X) e_1 = exp(X/S)^S e_1 (the expansion at r/S, applied S times): one
// segment at r ~ 100 needs terms whose size 2 I~_k rho^k reaches 2^16 and
// amplifies rounding as much; S segments of r/S keep it below 100 at about
// 1.5x the terms of one, against ~15 r terms for the Taylor series.  The extreme
// eigenvalues come from Sturm-sequence multisection (float32 counts, then a
// 1e-5 relative safety margin); the imaginary extent iota is the spectral
// radius of the skew part (same routine on |skew| entries).  The scaled
// modified Bessel values come from Miller's backward recurrence normalised by
// I~_0 + 2 sum_k I~_k = 1; the term count makes 2 I~_k rho^k <= 1e-16, rho the
// Bernstein-ellipse parameter holding the box [lo, hi] x [-iota, iota].  With
// Crouzeix's bound the error of a segment is ~1e-16 of its input times
// e^{hi/S} >= ||exp(X/S)||, so ~S 1e-16 e^{hi} >= S 1e-16 ||exp(X)|| in all,
// normwise like a dense expm.  Fallback (iota > r/2, no admissible term count
// within 64 segments, or more serial terms than the Taylor series): Taylor
// series in segments of norm <= 4 after the shift by the interval midpoint.
//
// GB300 issues float64 at 1/64 of the float32 rate, so a serial float64 chain
// costs ~70 cycles per operation: the recurrences (Bessel values, Chebyshev
// and Taylor terms) run in double-float (~2^-47 per operation, far below the
// tolerances the result serves) and every loop over rows or terms is spread
// over the block.
constexpr int CHEB_MAX = 600;
constexpr int SEG_MAX = 64;  // Chebyshev segments
constexpr int SX = 128;  // threads

__device__ __forceinline__ df dfd(double v) { return df_from_double(v); }
__device__ __forceinline__ double dd(df v) { return (double)v.hi + (double)v.lo; }

// block reductions over SX threads (sh: 4 entries of scratch, reused after a barrier)
__device__ df blk_dfsum(df v, df* sh, int tid) {
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)));
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  const df r = df_add(df_add(sh[0], sh[1]), df_add(sh[2], sh[3]));
  __syncthreads();
  return r;
}
__device__ float blk_maxf(float v, float* sh, int tid) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  const float r = fmaxf(fmaxf(sh[0], sh[1]), fmaxf(sh[2], sh[3]));
  __syncthreads();
  return r;
}
__device__ int blk_imin(int v, int* sh, int tid) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  const int r = min(min(sh[0], sh[1]), min(sh[2], sh[3]));
  __syncthreads();
  return r;
}

// number of eigenvalues < x of the symmetric tridiagonal (diag a, squared off-diagonal b2);
// the division is the fast reciprocal form (the bounds carry a 1e-5 relative margin)
__device__ int sturm_count(int n, const float* a, const float* b2, float x) {
  int cnt = 0;
  float q = a[0] - x;
  cnt += q < 0.f;
  for (int i = 1; i < n; ++i) {
    if (q == 0.f) q = 1e-30f;
    q = (a[i] - x) - __fdividef(b2[i - 1], q);
    cnt += q < 0.f;
  }
  return cnt;
}

struct SmallExpWork {
  double x[KIOPS_MMAX + 2];           // result (float64)
  float2 nb[2][KIOPS_MMAX + 4];       // recurrence rows for the neighbours (ping-pong; row i at i + 1,
                                      // zero pads at 0 and n + 1)
  df bes[CHEB_MAX + 2];
  df invk[32];
  float fa[KIOPS_MMAX + 2], fs2[KIOPS_MMAX + 2], fk2[KIOPS_MMAX + 2], fz[KIOPS_MMAX + 2];
  int cnt[SX];
  float pts[SX];
  float br[4];
  float shf[4];
  df shd[4];
  int shi[4];
  int mode, S, K;
  double lead;
};

// One round of Sturm multisection of the brackets [lo[g], hi[g]] (g = 0: the
// largest eigenvalue, threads 0..np-1; g = 1: the smallest, threads np..2np-1;
// ng groups): each thread counts at one of np interior points, the first
// thread of each group narrows its bracket to one cell.  All SX threads call
// it (barriers).  The points are kept in shared memory so the bracket update
// uses exactly the values that were counted.
__device__ void msect_round(int n, const float* a, const float* b2, float (&lo)[2], float (&hi)[2], int ng,
                            int np, SmallExpWork& w, int tid) {
  const int g = tid / np, t = tid - g * np;
  if (g < ng) {
    const float x = __fmaf_rn(hi[g] - lo[g], (float)(t + 1) / (float)(np + 1), lo[g]);
    w.pts[tid] = x;
    w.cnt[tid] = sturm_count(n, a, b2, x);
  }
  __syncthreads();
  if (g < ng && t == 0) {
    const int o = g * np;
    float nlo = lo[g], nhi = hi[g];
    if (g == 0) {  // smallest point with all eigenvalues below it
      int s = 0;
      while (s < np && w.cnt[o + s] < n) ++s;
      nhi = (s < np) ? w.pts[o + s] : hi[g];
      nlo = (s > 0) ? w.pts[o + s - 1] : lo[g];
    } else {  // largest point with no eigenvalue below it
      int s = np - 1;
      while (s >= 0 && w.cnt[o + s] > 0) --s;
      nlo = (s >= 0) ? w.pts[o + s] : lo[g];
      nhi = (s < np - 1) ? w.pts[o + s + 1] : hi[g];
    }
    w.br[2 * g] = nlo;
    w.br[2 * g + 1] = nhi;
  }
  __syncthreads();
  for (int q = 0; q < ng; ++q) {
    lo[q] = w.br[2 * q];
    hi[q] = w.br[2 * q + 1];
  }
  __syncthreads();
}

// Chebyshev segments: x <- I~_0 x + 2 sum_{k=1}^{K-1} I~_k T_k(Y) x, S times,
// with M = 2Y in (ma, mu, ml); x renormalised by a power of two before every
// segment but the first (lead collects the exponents).  R rows per thread.
template <int R>
__device__ void cheb_segments(int n, int S, int K, const df (&ma)[R], const df (&mu)[R], const df (&ml)[R],
                              df (&xr)[R], double& lead, SmallExpWork& w, int tid) {
  const df b0 = w.bes[0], b1 = df_scale2(w.bes[1], 2.f);
  for (int seg = 0; seg < S; ++seg) {
    if (seg > 0) {
      float mx = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) mx = fmaxf(mx, fabsf(xr[q].hi));
      mx = blk_maxf(mx, w.shf, tid);
      int e = 0;
      if (mx > 0.f) (void)frexpf(mx, &e);
      const float f = ldexpf(1.f, -e);
#pragma unroll
      for (int q = 0; q < R; ++q) xr[q] = df_scale2(xr[q], f);
      lead += e * 0.69314718055994530942;
    }
    df tm[R], tc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = tid + q * SX;
      if (i < n) w.nb[0][i + 1] = make_float2(xr[q].hi, xr[q].lo);
    }
    __syncthreads();
    // T_1 = Y x (half the row of M); x <- I~_0 x + 2 I~_1 T_1
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = tid + q * SX;
      tm[q] = xr[q];
      tc[q] = df_make(0.f, 0.f);
      if (i < n) {
        float p[3], e[3];
        df_prod(ma[q], xr[q], p[0], e[0]);
        df_prod(mu[q], cv(w.nb[0][i + 2]), p[1], e[1]);
        df_prod(ml[q], cv(w.nb[0][i]), p[2], e[2]);
        const df v = df_scale2(df_sum_pairs<3>(p, e), 0.5f);
        w.nb[1][i + 1] = make_float2(v.hi, v.lo);
        xr[q] = df_fma(b1, v, df_mul(b0, xr[q]));
        tc[q] = v;
      }
    }
    __syncthreads();
    // T_k = M T_{k-1} - T_{k-2}; term k reads nb[(k - 1) & 1], writes nb[k & 1]
    df bk = df_scale2(w.bes[2], 2.f);
    for (int k = 2; k < K; ++k) {
      const float2* src = w.nb[(k - 1) & 1];
      float2* dst = w.nb[k & 1];
      const df bnext = df_scale2(w.bes[k + 1], 2.f);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = tid + q * SX;
        if (i < n) {
          float p[4], e[4];
          df_prod(ma[q], tc[q], p[0], e[0]);
          df_prod(mu[q], cv(src[i + 2]), p[1], e[1]);
          df_prod(ml[q], cv(src[i]), p[2], e[2]);
          p[3] = -tm[q].hi;
          e[3] = -tm[q].lo;
          const df v = df_sum_pairs<4>(p, e);
          dst[i + 1] = make_float2(v.hi, v.lo);
          xr[q] = df_fma(bk, v, xr[q]);
          tm[q] = tc[q];
          tc[q] = v;
        }
      }
      bk = bnext;
      __syncthreads();
    }
  }
}

// Taylor segments: x <- sum_{k=0}^{30} M^k x / k!, S times, M = (T - cI)/S in
// (ma, mu, ml); renormalised like the Chebyshev segments.
template <int R>
__device__ void taylor_segments(int n, int S, const df (&ma)[R], const df (&mu)[R], const df (&ml)[R],
                                df (&xr)[R], double& lead, SmallExpWork& w, int tid) {
  for (int seg = 0; seg < S; ++seg) {
    if (seg > 0) {
      float mx = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) mx = fmaxf(mx, fabsf(xr[q].hi));
      mx = blk_maxf(mx, w.shf, tid);
      int e = 0;
      if (mx > 0.f) (void)frexpf(mx, &e);
      const float f = ldexpf(1.f, -e);
#pragma unroll
      for (int q = 0; q < R; ++q) xr[q] = df_scale2(xr[q], f);
      lead += e * 0.69314718055994530942;
    }
    df tc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = tid + q * SX;
      tc[q] = xr[q];
      if (i < n) w.nb[0][i + 1] = make_float2(xr[q].hi, xr[q].lo);
    }
    __syncthreads();
    for (int k = 1; k <= 30; ++k) {
      const float2* src = w.nb[(k - 1) & 1];
      float2* dst = w.nb[k & 1];
      const df ik = w.invk[k];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = tid + q * SX;
        if (i < n) {
          float p[3], e[3];
          df_prod(ma[q], tc[q], p[0], e[0]);
          df_prod(mu[q], cv(src[i + 2]), p[1], e[1]);
          df_prod(ml[q], cv(src[i]), p[2], e[2]);
          const df v = df_mul(df_sum_pairs<3>(p, e), ik);
          dst[i + 1] = make_float2(v.hi, v.lo);
          xr[q] = df_add(xr[q], v);
          tc[q] = v;
        }
      }
      __syncthreads();
    }
  }
}

// The recurrence matrix rows of this thread (M = (T - cI) cscale), the
// starting vector e_1, and the chosen recurrence; x returned in w.x.
template <int R>
__device__ void run_recurrence(int n, const double* dg, const double* up, const double* lo, double c,
                               double cscale, int mode, int S, int K, double& lead, SmallExpWork& w, int tid) {
  df ma[R], mu[R], ml[R], xr[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = tid + q * SX;
    const bool in = i < n;
    ma[q] = dfd(in ? (dg[i] - c) * cscale : 0.0);
    mu[q] = dfd((in && i + 1 < n) ? up[i] * cscale : 0.0);
    ml[q] = dfd((in && i >= 1) ? lo[i - 1] * cscale : 0.0);
    xr[q] = df_make((i == 0) ? 1.f : 0.f, 0.f);
  }
  if (mode == 0)
    cheb_segments<R>(n, S, K, ma, mu, ml, xr, lead, w, tid);
  else
    taylor_segments<R>(n, S, ma, mu, ml, xr, lead, w, tid);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = tid + q * SX;
    if (i < n) w.x[i] = dd(xr[q]);
  }
}

// x = exp(T) e_1 for the n x n tridiagonal T = tridiag(lo, dg, up) (already
// scaled by tau); lead: on return x holds exp(T) e_1 / e^{lead}.  Block-wide
// (SX threads); work arrays in shared memory.  The set-up (bounds, counts)
// runs in float32 and a few float64 scalars: float64 issues at 1/64 rate.
__device__ void small_exp_e1(int n, const double* dg, const double* up, const double* lo, SmallExpWork& w,
                             int tid) {
  // symmetric / skew parts in float32, Gershgorin box of each (one row per thread)
  float glo = 3e38f, ghi = -3e38f, kb = 0.f;
  for (int i = tid; i < n; i += SX) {
    const float ui = (i + 1 < n) ? (float)up[i] : 0.f, li = (i + 1 < n) ? (float)lo[i] : 0.f;
    const float s = 0.5f * (ui + li), k = 0.5f * (ui - li);
    const float di = (float)dg[i];
    w.fa[i] = di;
    w.fs2[i] = s * s;
    w.fk2[i] = k * k;
    w.fz[i] = 0.f;
    float rs = fabsf(s), rk = fabsf(k);
    if (i >= 1) {
      const float um = (float)up[i - 1], lm = (float)lo[i - 1];
      rs += 0.5f * fabsf(um + lm);
      rk += 0.5f * fabsf(um - lm);
    }
    glo = fminf(glo, di - rs);
    ghi = fmaxf(ghi, di + rs);
    kb = fmaxf(kb, rk);
  }
  glo = -blk_maxf(-glo, w.shf, tid);
  ghi = blk_maxf(ghi, w.shf, tid);
  kb = blk_maxf(kb, w.shf, tid);
  // float32 rounding of the entries and sums: 1e-5 relative outward
  glo -= 1e-5f * (fabsf(glo) + 1.f);
  ghi += 1e-5f * (fabsf(ghi) + 1.f);
  kb = kb * (1.f + 1e-5f) + 1e-30f;
  // both real-part bounds in the same rounds (64 points each, 2 rounds: 65^-2 of
  // the box), then iota (128 points, 1 round: 1/129 of its Gershgorin bound);
  // looser bounds only widen the box and the ellipse
  float lo2[2] = {glo, glo}, hi2[2] = {ghi, ghi};
  for (int round = 0; round < 2; ++round) msect_round(n, w.fa, w.fs2, lo2, hi2, 2, 64, w, tid);
  const double lam_hi = (double)hi2[0] + (1e-5 * (fabs((double)lo2[0]) + fabs((double)hi2[0])) + 1e-300);
  const double lam_lo = (double)lo2[1] - (1e-5 * (fabs((double)lo2[1]) + fabs((double)hi2[1])) + 1e-300);
  double iota = 0.0;
  if (n > 1) {
    float lo1[2] = {0.f, 0.f}, hi1[2] = {kb, kb};
    msect_round(n, w.fz, w.fk2, lo1, hi1, 1, SX, w, tid);
    iota = (double)hi1[0] * (1.0 + 1e-5) + 1e-300;
  }
  const double r = 0.5 * (lam_hi - lam_lo), c = 0.5 * (lam_hi + lam_lo);
  // Taylor segment count (norm <= 4 each) about the centre of the box:
  // ||T - cI||_2 <= 2 sqrt(r^2 + iota^2) (numerical radius), or the 1-norm if smaller
  const float cf = (float)c;
  float cs = 0.f;
  for (int i = tid; i < n; i += SX) {
    float v = fabsf((float)dg[i] - cf);
    if (i >= 1) v += fabsf((float)up[i - 1]);
    if (i + 1 < n) v += fabsf((float)lo[i]);
    cs = fmaxf(cs, v);
  }
  const float nrm1 = blk_maxf(cs, w.shf, tid) * (1.f + 1e-5f);
  const float rf = (float)r, iof = (float)iota;
  const float tnrm = fminf(nrm1, 2.f * sqrtf(rf * rf + iof * iof) * (1.f + 1e-5f));
  const int S_taylor = tnrm > 4.f ? (int)ceilf(tnrm / 4.f) : 1;
  int mode = (!(r >= 1e-3) || iota > 0.5 * r) ? 1 : 0;
  int K = -1, S = 1;
  if (mode == 0) {
    // Bernstein ellipse holding the box [-1, 1] x [-iota/r, iota/r] (the same for
    // every segment: exp(X) = exp(X/S)^S scales the box, not its aspect)
    const float y0 = iof / rf;
    const float b2 = 0.5f * (y0 * y0 + sqrtf(y0 * y0 * y0 * y0 + 4.f * y0 * y0));
    const float lnrho = logf(sqrtf(1.f + b2) + sqrtf(b2)) * (1.f + 1e-5f);
    // first segment count: the scaled Bessel values are close to
    // e^{-k^2/(2 rs)} / sqrt(2 pi rs), so max_k 2 I~_k(rs) rho^k is close to
    // 2 e^{rs ln(rho)^2 / 2} / sqrt(2 pi rs); take the smallest S whose estimate
    // is <= 2^6 (the exact amplification test below decides)
    while (S < SEG_MAX) {
      const float rs = rf / (float)S;
      const float est = 0.5f * rs * lnrho * lnrho * 1.44269504f + 1.f - 0.5f * log2f(6.28318531f * rs);
      if (est <= 6.f) break;
      ++S;
    }
    for (int attempt = 0; attempt < 4; ++attempt) {
      const double rs = r / S;
      const float rsf = (float)rs;
      // kmax: an upper bound of the term count from
      //   I~_k(x) <= (x/2)^k / k! e^{x^2/(4(k+1)) - x}
      // (the series of I_k term by term against that of the exponential) and
      // Robbins' ln k! >= k ln k - k + ln(2 pi k)/2: the first k > 2 where that
      // bound of 2 I~_k rho^k and of its predecessor is <= 1e-16 (every thread
      // tests some k, one block minimum)
      const float lstep = lnrho + logf(0.5f * rsf);
      auto lbound = [&](int k) -> float {
        const float kf = (float)k;
        const float lfact = kf * logf(kf) - kf + 0.5f * logf(6.28318531f * kf);
        return 0.69314718f + kf * lstep - lfact - rsf + rsf * rsf / (4.f * (kf + 1.f));
      };
      int kb_min = CHEB_MAX;
      for (int k = 3 + tid; k <= CHEB_MAX - 2; k += SX)
        if (lbound(k) <= -36.8413615f && lbound(k - 1) <= -36.8413615f) kb_min = min(kb_min, k + 2);  // ln(1e-16)
      const int kmax = blk_imin(kb_min, w.shi, tid);
      if (tid == 0) {
        // Miller's backward recurrence I_{k-1} = (2k/rs) I_k + I_{k+1} in double-float,
        // rescaled by powers of two; started 24 indices beyond both kmax and 2 rs, where
        // each step down shrinks the start error by a factor >= 2
        const int kstart = max(kmax, 2 * (int)rs) + 24;
        const df ir2 = dfd(2.0 / rs);
        df ip1 = df_make(0.f, 0.f), ik = df_make(1e-30f, 0.f);
        for (int k = kstart; k >= 0; --k) {
          if (k <= kmax) w.bes[k] = ik;
          const df im1 = df_fma(df_mul(df_make((float)k, 0.f), ir2), ik, ip1);
          ip1 = ik;
          ik = im1;
          if (fabsf(ik.hi) > 1e30f) {
            ik = df_scale2(ik, 0x1p-100f);
            ip1 = df_scale2(ip1, 0x1p-100f);
            for (int q = k; q <= kmax; ++q) w.bes[q] = df_scale2(w.bes[q], 0x1p-100f);
          }
        }
      }
      __syncthreads();
      // normalise: I~_0 + 2 sum_{k >= 1} I~_k = 1
      df part = df_make(0.f, 0.f);
      for (int k = tid; k <= kmax; k += SX) part = df_add(part, k == 0 ? w.bes[0] : df_scale2(w.bes[k], 2.f));
      const df sum = blk_dfsum(part, w.shd, tid);
      const df isum = dfd(1.0 / dd(sum));
      for (int k = tid; k <= kmax; k += SX) w.bes[k] = df_mul(w.bes[k], isum);
      // one more entry, zero, for the look-ahead of the recurrence
      if (tid == 0) w.bes[kmax + 1] = df_make(0.f, 0.f);
      __syncthreads();
      // term count: the first k > 2 with 2 I~_k rho^k and 2 I~_{k-1} rho^{k-1} <= 1e-16
      // (log2 in float32: a threshold test); no count before rho^k > 2^96 (T_k(Y) x
      // must stay inside the double-float range)
      const float l2r = lnrho * 1.44269504f;
      const float lim = -53.15f;  // log2(1e-16)
      auto lv = [&](int k) -> float {
        const float b = 2.f * w.bes[k].hi;
        return (b > 0.f ? log2f(b) : -1e30f) + (float)k * l2r;
      };
      int kc = 1 << 30;
      for (int k = 3 + tid; k <= kmax; k += SX)
        if (lv(k) <= lim && lv(k - 1) <= lim && (float)k * l2r <= 96.f) kc = min(kc, k);
      kc = blk_imin(kc, w.shi, tid);
      if (kc < (1 << 30)) {
        // amplification of rounding errors: max_{k < K} 2 I~_k rho^k
        float amp = -1e30f;
        for (int k = tid; k < kc; k += SX) amp = fmaxf(amp, lv(k));
        amp = blk_maxf(amp, w.shf, tid);
        if (amp <= 6.644f) K = kc;  // log2(100)
      }
      if (K >= 0 || S >= SEG_MAX) break;
      ++S;
    }
    // Chebyshev only while it needs fewer serial terms than the Taylor fallback
    if (K < 0 || (long)S * K > 30L * S_taylor) mode = 1;
  }
  if (mode == 1) S = S_taylor;

  // The recurrence in double-float.  Each thread keeps its rows (i = tid + q SX)
  // of the matrix, of the last two terms and of the sum in registers; the rows
  // its neighbours need pass through a ping-pong buffer (term k writes nb[k & 1]
  // and reads nb[(k - 1) & 1]), one barrier per term.  The new row is one sum of
  // product pairs with a single renormalisation.
  // Matrix of the recurrence: Chebyshev 2Y = 2(T - cI)/r, Taylor (T - cI)/S.
  for (int i = tid; i < KIOPS_MMAX + 4; i += SX) {
    w.nb[0][i] = make_float2(0.f, 0.f);
    w.nb[1][i] = make_float2(0.f, 0.f);
  }
  if (tid < 32) w.invk[tid] = dfd(tid > 0 ? 1.0 / tid : 0.0);
  __syncthreads();  // pads and invk before the first rows are written
  double lead = (mode == 0) ? lam_hi : c;  // Chebyshev: S (c + r)/S; Taylor: the shift
  const double cscale = (mode == 0) ? 2.0 / r : 1.0 / S;
  if (n <= SX)
    run_recurrence<1>(n, dg, up, lo, c, cscale, mode, S, K, lead, w, tid);
  else
    run_recurrence<2>(n, dg, up, lo, c, cscale, mode, S, K, lead, w, tid);
  if (tid == 0) {
    w.mode = mode;
    w.lead = lead;
    w.K = K;
    w.S = S;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SX) k_kexp(KiopsCtl* kc, int m, double tau, double tau_end, double tol) {
  __shared__ double dg[KIOPS_MMAX + 2], up[KIOPS_MMAX + 2], lo[KIOPS_MMAX + 2];
  __shared__ SmallExpWork w;
  __shared__ int n_s;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int hm = kc->happy_m;
    const int mm = hm > 0 ? hm : m;
    n_s = hm > 0 ? hm : m + 1;
    const int n = n_s;
    for (int i = 0; i < n; ++i) {
      dg[i] = tau * (i < mm ? kc->hd[i] : 0.0);          // row m of Hbar has no diagonal
      up[i] = tau * ((i + 1 < mm) ? kc->hu[i + 1] : 0.0);  // (i, i+1); column m is zero
      lo[i] = tau * ((i + 1 < n) ? kc->hl[i] : 0.0);       // (i+1, i)
    }
  }
  __syncthreads();
  const int n = n_s;
  small_exp_e1(n, dg, up, lo, w, tid);
  const double e = exp(w.lead);
  for (int i = tid; i < n; i += 128) {
    const double Fi = e * w.x[i];
    kc->F[i] = Fi;
    const double cf = kc->beta * Fi * kc->s[i];
    kc->coef[i] = cf;
    kc->coeff[i] = split2d(cf);
  }
  __syncthreads();
  if (tid == 0) {
    double omega = 0.0, err = 0.0;
    if (kc->happy_m == 0) {
      err = kc->beta * fabs(e * w.x[m]);
      omega = (tau_end / tau) * err / (tol * kc->beta);
    }
    kc->err = err;
    kc->omega = omega;
    if (!isfinite(omega)) kc->status = PHIX_ENAN;
    __threadfence();
  }
}

// exp(tau T) e_1 for a caller's tridiagonal T (device arrays), out[n]
__global__ void __launch_bounds__(128) k_smallexp(int n, const double* d, const double* u, const double* l,
                                                  double tau, double* out, int* mode_out) {
  __shared__ double dg[KIOPS_MMAX + 2], up[KIOPS_MMAX + 2], lo[KIOPS_MMAX + 2];
  __shared__ SmallExpWork w;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += 128) {
    dg[i] = tau * d[i];
    up[i] = (i + 1 < n) ? tau * u[i] : 0.0;
    lo[i] = (i + 1 < n) ? tau * l[i] : 0.0;
  }
  __syncthreads();
  small_exp_e1(n, dg, up, lo, w, tid);
  const double e = exp(w.lead);
  for (int i = tid; i < n; i += 128) out[i] = e * w.x[i];
  if (tid == 0 && mode_out) *mode_out = w.mode;
}

struct CombArgs {
  const void* const* Z;  // device array of slot pointers
  int n;
  KiopsCtl* kc;
  double* partials;
  double* out;
  double scale;
  int p, nscaled;
  double h;
  double kJ[8];
};

template <int P>
__global__ void __launch_bounds__(THREADS) k_kcomb(CombArgs a, size_t N) {
  using T = typename KTr<P>::T;
  using C = typename KTr<P>::C;
  using Acc = typename KTr<P>::Acc;
  KiopsCtl* kc = a.kc;
  __shared__ C cf[KIOPS_MMAX + 2];
  __shared__ const T* zp[KIOPS_MMAX + 2];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int i = tid; i < a.n; i += THREADS) {
    cf[i] = coef<C>(__ldcg(&kc->coef[i]), __ldcg(&kc->coeff[i]));
    zp[i] = static_cast<const T*>(a.Z[i]);
  }
  __syncthreads();
  T* z0 = const_cast<T*>(zp[0]);
  Acc acc[1] = {acc_zero<Acc>()};
  const size_t stride = (size_t)gridDim.x * THREADS;
  for (size_t i = (size_t)blockIdx.x * THREADS + tid; i < N; i += stride) {
    C w = cf[0] * ldr1(zp[0] + i);
    for (int k = 1; k < a.n; ++k) w = w + cf[k] * ldr1(zp[k] + i);
    st1(z0 + i, w);
    if (a.out) {
      double d;
      if constexpr (P == P_FP64)
        d = w;
      else
        d = (double)w.hi + (double)w.lo;
      a.out[i] = a.scale * d;
    }
    acc_dot(acc[0], w, w);
  }
  if (block_partials_and_last<Acc, 1>(acc, a.partials, &kc->count)) {
    double tot[1];
    reduce_partials<Acc, 1>(a.partials, tot);
    if (tid == 0) {
      double tw[KIOPS_PMAX];
      double nz = tot[0];
      for (int t = 0; t < a.p; ++t) {
        double v = 0.0;
        for (int k = 0; k < a.n; ++k) v += kc->coef[k] * kc->tail[k * KIOPS_PMAX + t];
        tw[t] = v;
        nz += v * v;
      }
      for (int t = 0; t < a.p; ++t) kc->tail[t] = tw[t];
      const double beta = sqrt(nz);
      kc->beta = beta;
      kc->s[0] = beta > 0 ? 1.0 / beta : 0.0;
      kc->sf[0] = split2d(kc->s[0]);
      kc->stop = 0;
      kc->happy_m = 0;
      if (!isfinite(beta)) kc->status = PHIX_ENAN;
      prepare_pass1(kc, 0, a.p, a.h, a.kJ, a.nscaled);
      kc->count = 0;
      __threadfence();
    }
  }
}

template <int P>
__global__ void __launch_bounds__(THREADS)
    k_kstart(const double* __restrict__ b0, typename KTr<P>::T* __restrict__ z0, size_t N, CombArgs a, double eta,
             double c) {
  using C = typename KTr<P>::C;
  using Acc = typename KTr<P>::Acc;
  KiopsCtl* kc = a.kc;
  Acc acc[1] = {acc_zero<Acc>()};
  const size_t stride = (size_t)gridDim.x * THREADS;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (size_t i = (size_t)blockIdx.x * THREADS + tid; i < N; i += stride) {
    double x = b0 ? c * b0[i] : 0.0;  // c: a power of two, exact
    C w;
    if constexpr (P == P_FP64)
      w = x;
    else
      w = df_from_double(x);
    st1(z0 + i, w);
    acc_dot(acc[0], w, w);
  }
  if (block_partials_and_last<Acc, 1>(acc, a.partials, &kc->count)) {
    double tot[1];
    reduce_partials<Acc, 1>(a.partials, tot);
    if (tid == 0) {
      kc->eta = eta;
      for (int t = 0; t < KIOPS_PMAX; ++t) kc->tail[t] = 0.0;
      double nz = tot[0];
      if (a.p > 0) {
        kc->tail[a.p - 1] = c / eta;
        nz += (c / eta) * (c / eta);
      }
      const double beta = sqrt(nz);
      kc->beta = beta;
      kc->s[0] = beta > 0 ? 1.0 / beta : 0.0;
      kc->sf[0] = split2d(kc->s[0]);
      kc->stop = 0;
      kc->happy_m = 0;
      kc->status = isfinite(beta) ? PHIX_OK : PHIX_ENAN;
      prepare_pass1(kc, 0, a.p, a.h, a.kJ, a.nscaled);
      kc->count = 0;
      __threadfence();
    }
  }
}

template <int P>
__global__ void __launch_bounds__(THREADS)
    k_kconvert(const double* __restrict__ b, typename KTr<P>::T* __restrict__ out, size_t n, double* partials,
               unsigned int* counter, double* norm1) {
  double acc[1] = {0.0};
  const size_t stride = (size_t)gridDim.x * THREADS;
  for (size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x; i < n; i += stride) {
    double x = b[i];
    acc[0] += fabs(x);
    if (!out) continue;  // norm only
    if constexpr (P == P_FP64)
      out[i] = x;
    else {
      df w = df_from_double(x);
      out[i] = make_float2(w.hi, w.lo);
    }
  }
  if (block_partials_and_last<double, 1>(acc, partials, counter)) {
    double tot[1];
    reduce_partials<double, 1>(partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      *norm1 = tot[0];
      *counter = 0;
      __threadfence();
    }
  }
}

ArnArgs make_arn(const KiopsSpec& s, int j, int V) {
  ArnArgs a{};
  a.zj = s.Zh[j];
  a.zjm1 = j >= 1 ? s.Zh[j - 1] : nullptr;
  a.zout = s.Zh[j + 1];
  for (int b = 0; b < s.nb; ++b) {
    a.bz[b] = s.bz[b];
    a.bslot[b] = s.bslot[b];
  }
  a.nb = s.nb;
  a.st = s.st;
  a.kc = s.kc;
  a.partials = s.partials;
  a.j = j;
  a.p = s.p;
  a.nx = s.nx;
  a.ny = s.ny;
  a.tiles_x = (s.nx / V + 31) / 32;
  a.ntiles = a.tiles_x * ((s.ny + TILE_Y - 1) / TILE_Y);
  a.nscaled = s.nscaled;
  a.h = s.h;
  for (int i = 0; i < 8; ++i) a.kJ[i] = s.kJ[i];
  return a;
}

CombArgs make_comb(const KiopsSpec& s, int n, double* out, double scale) {
  CombArgs c{};
  c.Z = s.Z;
  c.n = n;
  c.kc = s.kc;
  c.partials = s.partials;
  c.out = out;
  c.scale = scale;
  c.p = s.p;
  c.nscaled = s.nscaled;
  c.h = s.h;
  for (int i = 0; i < 8; ++i) c.kJ[i] = s.kJ[i];
  return c;
}

// resident blocks per SM of a THREADS-thread kernel (at least 1)
int blocks_per_sm(const void* fn) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, THREADS, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 4;
  }
  return nb < 1 ? 1 : nb;
}

// Both passes run as one wave of resident blocks (SMs x occupancy): a grid
// beyond that leaves a partial second wave on a third of the SMs.
template <int P, int OP>
cudaError_t arn_t(const KiopsSpec& s, int j, cudaStream_t st) {
  static const int occ1v2 = blocks_per_sm(reinterpret_cast<const void*>(k_arn1<P, OP, 2>));
  static const int occ1v1 = blocks_per_sm(reinterpret_cast<const void*>(k_arn1<P, OP, 1>));
  static const int occ2 = blocks_per_sm(reinterpret_cast<const void*>(k_arn2<P>));
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  ArnArgs a = make_arn(s, j, V);
  const int g1 = std::min(s.nsm * (V == 2 ? occ1v2 : occ1v1), a.ntiles);
  if (V == 2)
    k_arn1<P, OP, 2><<<g1, dim3(32, TILE_Y), 0, st>>>(a);
  else
    k_arn1<P, OP, 1><<<g1, dim3(32, TILE_Y), 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t N = (size_t)s.nx * s.ny * (OP == PHIX_OP_GRAYSCOTT ? 2 : 1);
  k_arn2<P><<<s.nsm * occ2, dim3(32, TILE_Y), 0, st>>>(a, N);
  return cudaGetLastError();
}

template <int P>
cudaError_t arn_p(const KiopsSpec& s, int j, cudaStream_t st) {
  switch (s.op) {
    case PHIX_OP_ADVDIFF:
      return arn_t<P, PHIX_OP_ADVDIFF>(s, j, st);
    case PHIX_OP_GRAYSCOTT:
      return arn_t<P, PHIX_OP_GRAYSCOTT>(s, j, st);
    case PHIX_OP_BURGERS:
      return arn_t<P, PHIX_OP_BURGERS>(s, j, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t kiops_arnoldi(const KiopsSpec& s, int j, cudaStream_t st) {
  return s.prec == P_FP64 ? arn_p<P_FP64>(s, j, st) : arn_p<P_DF64>(s, j, st);
}

cudaError_t small_expm_e1(int n, const double* d, const double* u, const double* l, double tau, double* out,
                          int* mode, cudaStream_t st) {
  if (n < 1 || n > KIOPS_MMAX + 1) return cudaErrorInvalidValue;
  k_smallexp<<<1, 128, 0, st>>>(n, d, u, l, tau, out, mode);
  return cudaGetLastError();
}

cudaError_t kiops_smallexp(KiopsCtl* kc, int m, double tau, double tau_end, double tol, cudaStream_t st) {
  k_kexp<<<1, 128, 0, st>>>(kc, m, tau, tau_end, tol);
  return cudaGetLastError();
}

cudaError_t kiops_combine(const KiopsSpec& s, int n, double* out, double scale, cudaStream_t st) {
  const size_t N = (size_t)s.nx * s.ny * (s.op == PHIX_OP_GRAYSCOTT ? 2 : 1);
  CombArgs c = make_comb(s, n, out, scale);
  if (s.prec == P_FP64)
    k_kcomb<P_FP64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(c, N);
  else
    k_kcomb<P_DF64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(c, N);
  return cudaGetLastError();
}

cudaError_t kiops_start(const KiopsSpec& s, const double* b0, double eta, double cscale, cudaStream_t st) {
  const size_t N = (size_t)s.nx * s.ny * (s.op == PHIX_OP_GRAYSCOTT ? 2 : 1);
  CombArgs c = make_comb(s, 1, nullptr, 0.0);
  if (s.prec == P_FP64)
    k_kstart<P_FP64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(b0, static_cast<double*>(s.Zh[0]), N, c, eta, cscale);
  else
    k_kstart<P_DF64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(b0, static_cast<float2*>(s.Zh[0]), N, c, eta, cscale);
  return cudaGetLastError();
}

cudaError_t kiops_convert(int prec, size_t n, const double* b, void* out, double* partials,
                          unsigned int* counter, double* norm1, int grid, cudaStream_t st) {
  if (prec == P_FP64)
    k_kconvert<P_FP64><<<grid, dim3(32, TILE_Y), 0, st>>>(b, static_cast<double*>(out), n, partials, counter, norm1);
  else
    k_kconvert<P_DF64><<<grid, dim3(32, TILE_Y), 0, st>>>(b, static_cast<float2*>(out), n, partials, counter, norm1);
  return cudaGetLastError();
}

}  // namespace phix
