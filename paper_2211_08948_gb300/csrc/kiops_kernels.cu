// KIOPS-style Krylov kernels (Sec. 2.1 of the paper): Arnoldi with window-2
// incomplete orthogonalisation on the augmented matrix
//   A~ = [[A, eta B], [0, K]],  A = h J,  B = [b_p, ..., b_1],  K = shift,
// the small exponential exp(tau Hbar) e_1 of the (tridiagonal) Hessenberg
// matrix with the corrected-Krylov error estimate, and the combination of the
// basis into the substep result.
//
// The basis is kept unnormalised, V_i = s_i Zhat_i; the N part of Zhat_i is
// stored in the iteration precision (float64 or double-float), the p tail
// entries in float64 inside the control block.  An Arnoldi step has two grid
// passes with a reduction between them (the two inner products per step that
// incomplete orthogonalisation leaves, Sec. 2.1):
//   pass 1: z = A~ V_j (5-point stencil + the eta b columns), partial dots
//           <Zhat_j, z>, <Zhat_{j-1}, z> and ||z||^2;
//   pass 2: z <- z - h_jj V_j - h_{j-1,j} V_{j-1} in place, partial ||z||^2;
// the last block of each pass adds the tail terms, forms h_jj, h_{j-1,j},
// h_{j+1,j}, s_{j+1} and writes the coefficients of the next launch.  On grids
// of whole 64 x 8 tiles, pass 2 of step j and pass 1 of step j + 1 run as one
// launch (k_arnf): the orthogonalised vector is staged in shared memory with a
// one-point halo ring and the stencil of the next step reads it there.
#include <algorithm>
#include <cstdint>
#include "iter_common.cuh"
#include "op_points.cuh"

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

// ws w - c1 z - c0 y: float64, or one sum of double-float product pairs with a
// single renormalisation
__device__ __forceinline__ double orth3(double ws, double w, double c1, double z, double c0, double y) {
  return ws * w - c1 * z - c0 * y;
}
__device__ __forceinline__ df orth3(df ws, df w, df c1, df z, df c0, df y) {
  float p[3], e[3];
  df_prod(ws, w, p[0], e[0]);
  df_prod(df_neg(c1), z, p[1], e[1]);
  df_prod(df_neg(c0), y, p[2], e[2]);
  return df_sum_pairs<3>(p, e);
}

// r = 1/sqrt(x), s = sqrt(x): a float32 seed and two Newton steps
// y <- y (3/2 - x y^2 / 2) in float64 inside the float32 range, a float64
// square root and division outside it (and for 0, inf, NaN)
__device__ __forceinline__ void rsqrt_and_sqrt(double x, double& r, double& s) {
  if (x > 1e-30 && x < 1e30) {
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x * y, y, 1.5);
    y = y * fma(-0.5 * x * y, y, 1.5);
    r = y;
    s = x * y;
  } else {
    s = sqrt(x);
    r = 1.0 / s;
  }
}

// Asynchronous global -> shared copies (cp.async): 16-byte (L2 only) and
// 8-byte forms, the commit and the wait for all of this thread's groups.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// two adjacent values from shared memory as one 16-byte word (p 16-byte aligned)
__device__ __forceinline__ void lds2(const double* p, double& a, double& b) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  a = t.x;
  b = t.y;
}
__device__ __forceinline__ void lds2(const float2* p, df& a, df& b) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a = df_make(t.x, t.y);
  b = df_make(t.z, t.w);
}

// a value in its storage form (float64, or the two float32 parts)
__device__ __forceinline__ double stv(double v) { return v; }
__device__ __forceinline__ float2 stv(df v) { return make_float2(v.hi, v.lo); }

template <int P>
struct KTr;
template <>
struct KTr<P_FP64> {
  using T = double;
  using T2 = double2;
  using C = double;
  using S = double;
  using Acc = double;
};
template <>
struct KTr<P_DF64> {
  using T = float2;
  using T2 = float4;
  using C = df;
  using S = float2;
  using Acc = df;
};

struct ArnArgs {
  const void* zj;
  const void* zjm1;  // NULL for j = 0
  void* zout;        // slot j + 1 (fused first pass: the scratch vector W0)
  const void* win;   // fused step: W (pass-1 result of step j, scaled by ws)
  void* wout;        // fused step: u (pass-1 result of step j + 1, unscaled)
  int fused;         // pass 1 of step 0 feeding fused steps
  const void* bz[KIOPS_PMAX];
  int bslot[KIOPS_PMAX];
  int nb;
  const void* st;
  KiopsCtl* kc;
  double* partials;
  int j, p, nx, ny, ntiles, tiles_x, nscaled;
  double h;
  double kJ[8];
  int gkind;         // general operator (the no-flow problems): its kind, parameters;
  double gprm[8];    // st is then the raw float64 state
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

// After pass 1 of step j (tail[j + 1] = tail of A~ z_j, c1/c0 set): the
// orthogonalised tail of Zhat_{j+1}, the scale ws of the scratch vector W, and
// the coefficients of u = A~ [Zhat_{j+1}; tail_{j+1}] without the s_{j+1}
// factor (k h, ga = h, b-column weights eta tail_{j+1}).  Single thread.
__device__ void fused_prepare(KiopsCtl* kc, int j, int p, double ws, double h, const double* kJ, int nscaled) {
  double* t1 = kc->tail + (j + 1) * KIOPS_PMAX;
  const double* t0 = kc->tail + j * KIOPS_PMAX;
  for (int t = 0; t < p; ++t) {
    double v = t1[t] - kc->c1d * t0[t];
    if (j >= 1) v -= kc->c0d * kc->tail[(j - 1) * KIOPS_PMAX + t];
    t1[t] = v;
    const double b = kc->eta * v;
    kc->bud[t] = b;
    kc->buf[t] = split2d(b);
  }
  kc->wsd = ws;
  kc->wsf = split2d(ws);
  for (int i = 0; i < 8; ++i) {
    const double v = i < nscaled ? kJ[i] * h : kJ[i];
    kc->kud[i] = v;
    kc->kuf[i] = split2d(v);
  }
  kc->gud = h;
  kc->guf = split2d(h);
}

__device__ void arn1_finish(const ArnArgs& a, KiopsCtl* kc, const double (&tot)[3]);

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
    if (threadIdx.x == 0 && threadIdx.y == 0) arn1_finish(a, kc, tot);
  }
}

// Pass 1 of Arnoldi step j for a general operator (the no-flow problems),
// float64, one point per thread: z = A~ V_j = (h s_j) J Zhat_j + B t (the
// augmented columns), with <Zhat_j, z>, <Zhat_{j-1}, z>, ||z||^2.
__global__ void __launch_bounds__(THREADS) k_arn1g(ArnArgs a) {
  KiopsCtl* kc = a.kc;
  if (__ldcg(&kc->stop)) return;
  const double g = __ldcg(&kc->gad);  // h s_j
  double bw[KIOPS_PMAX];
  for (int b = 0; b < KIOPS_PMAX; ++b) bw[b] = b < a.nb ? __ldcg(&kc->bd[a.bslot[b]]) : 0.0;
  const Geo geo = make_geo(a.gkind, a.nx, a.ny);
  const int nc = op_ncomp(a.gkind);
  const size_t plane = (size_t)a.nx * a.ny;
  const double* zj = static_cast<const double*>(a.zj);
  const double* zm = static_cast<const double*>(a.zjm1);
  double* zo = static_cast<double*>(a.zout);
  const double* st = static_cast<const double*>(a.st);
  const Nbr zero{0, 0, 0, 0, 0};
  double acc[3] = {0.0, 0.0, 0.0};
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (size_t i = (size_t)blockIdx.x * THREADS + tid; i < plane; i += (size_t)gridDim.x * THREADS) {
    const int ix = (int)(i % (size_t)a.nx), iy = (int)(i / (size_t)a.nx);
    const Nbr xa = load_nbr(zj, geo, ix, iy);
    const Nbr xb = nc == 2 ? load_nbr(zj + plane, geo, ix, iy) : xa;
    const Nbr sa = st ? load_nbr(st, geo, ix, iy) : zero;
    const Nbr sb = (st && nc == 2) ? load_nbr(st + plane, geo, ix, iy) : sa;
    double J[2];
    jv_nbr(a.gkind, a.gprm, geo, xa, xb, sa, sb, J);
    const double xc[2] = {xa.c, xb.c};
    for (int q = 0; q < nc; ++q) {
      const size_t idx = q * plane + i;
      double z = g * J[q];
      for (int b = 0; b < a.nb; ++b) z += bw[b] * static_cast<const double*>(a.bz[b])[idx];
      zo[idx] = z;
      acc[0] += xc[q] * z;
      if (zm) acc[1] += zm[idx] * z;
      acc[2] += z * z;
    }
  }
  if (block_partials_and_last<double, 3>(acc, a.partials, &kc->count)) {
    double tot[3];
    reduce_partials<double, 3>(a.partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) arn1_finish(a, kc, tot);
  }
}

// The epilogue of pass 1 (single thread): h_{j,j}, h_{j-1,j}, ||A~ V_j||, the
// tail of A~ V_j, the pass-2 coefficients.
__device__ void arn1_finish(const ArnArgs& a, KiopsCtl* kc, const double (&tot)[3]) {
  {
    {
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
      if (a.fused) fused_prepare(kc, j, p, 1.0, a.h, a.kJ, a.nscaled);
      if (!isfinite(hjj) || !isfinite(hjm) || !isfinite(zz)) {
        kc->status = PHIX_ENAN;
        kc->stop = 1;
      }
      kc->count = 0;
      __threadfence();
    }
  }
}

// shared-memory layout of the fused step: the two staged-tile buffers, then the
// per-thread prefetch stage (pairs of W, Zhat_j, Zhat_{j-1}, the state planes
// and nb b-copies; the ring point's three values)
constexpr int ARNF_TW = 64, ARNF_SW = ARNF_TW + 2, ARNF_NRING = 2 * ARNF_TW + 2 * TILE_Y;
__host__ __device__ constexpr int arnf_tile_bytes(int nc, int elem) {
  return ((2 * nc * (TILE_Y + 2) * ARNF_SW * elem + 15) / 16) * 16;
}
__host__ __device__ constexpr int arnf_smem_bytes(int nc, int ng, int nb, int elem) {
  return arnf_tile_bytes(nc, elem) + (3 * nc + ng + nb * nc) * THREADS * 2 * elem + 3 * nc * ARNF_NRING * elem;
}

// Fused Arnoldi step j of the incomplete orthogonalisation (Sec. 2.1; grids of
// whole tiles: nx % 64 == 0, ny % TILE_Y == 0).
// Completes step j: Zhat_{j+1} = ws W - c1 Zhat_j - c0 Zhat_{j-1} (written to
// slot j + 1 and, with a one-point halo ring recomputed from W, Zhat_j,
// Zhat_{j-1}, staged in shared memory), and runs pass 1 of step j + 1 from
// the staged tile: u = A~ [Zhat_{j+1}; tail_{j+1}] without the factor s_{j+1}
// (written to the other scratch vector), with <Zhat_{j+1}, Zhat_{j+1}>,
// <Zhat_{j+1}, u>, <Zhat_j, u> and <u, u>.  Five vectors move per step instead
// of seven (two-pass); the recompute is the ring, 9/32 of the tile.
template <int P, int OP>
__global__ void __launch_bounds__(THREADS) k_arnf(ArnArgs a) {
  using T = typename KTr<P>::T;
  using C = typename KTr<P>::C;
  using S = typename KTr<P>::S;
  using Acc = typename KTr<P>::Acc;
  constexpr int V = 2;
  constexpr int NC = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 1;
  constexpr int TW = 32 * V, SW = TW + 2, NRING = 2 * TW + 2 * TILE_Y;
  static_assert(NRING <= THREADS, "one ring point per thread");
  static_assert(TW == ARNF_TW && SW == ARNF_SW && NRING == ARNF_NRING, "layout of arnf_smem_bytes");
  // Dynamic shared memory: the staged tile (two buffers, one barrier per tile:
  // a buffer is rewritten two tiles later, after every thread has passed the
  // next tile's barrier), then each thread's prefetch stage (see below).
  extern __shared__ __align__(16) unsigned char dsm[];
  using T2 = typename KTr<P>::T2;  // a pair of values, 16 bytes
  constexpr int NG = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 0;  // state planes staged per point pair
  T (*smb)[NC][TILE_Y + 2][SW] = reinterpret_cast<T (*)[NC][TILE_Y + 2][SW]>(dsm);
  T2* stW = reinterpret_cast<T2*>(dsm + arnf_tile_bytes(NC, (int)sizeof(T)));
  T2* stZ = stW + NC * THREADS;
  T2* stM = stZ + NC * THREADS;
  T2* stG = stM + NC * THREADS;
  T2* stB = stG + NG * THREADS;
  T* rgW = reinterpret_cast<T*>(stB + a.nb * NC * THREADS);
  T* rgZ = rgW + NC * NRING;
  T* rgM = rgZ + NC * NRING;
  KiopsCtl* kc = a.kc;
  // the stop flag and the step's coefficients: independent loads, issued
  // together (the flag is tested after them)
  const int stop0 = __ldcg(&kc->stop);
  const C ws = coef<C>(__ldcg(&kc->wsd), __ldcg(&kc->wsf));
  const C c1 = coef<C>(__ldcg(&kc->c1d), __ldcg(&kc->c1f));
  const C c0 = coef<C>(__ldcg(&kc->c0d), __ldcg(&kc->c0f));
  C kk[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) kk[i] = coef<C>(__ldcg(&kc->kud[i]), __ldcg(&kc->kuf[i]));
  const C ga = coef<C>(__ldcg(&kc->gud), __ldcg(&kc->guf));
  C bw[KIOPS_PMAX];
#pragma unroll
  for (int b = 0; b < KIOPS_PMAX; ++b)
    bw[b] = b < a.nb ? coef<C>(__ldcg(&kc->bud[a.bslot[b]]), __ldcg(&kc->buf[a.bslot[b]])) : C{};
  if (stop0) return;

  Acc acc[4] = {acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>()};
  // ||Zhat_{j+1}||^2 and <u, u> in float32 on the double-float path: an error d
  // in ||Zhat_{j+1}|| scales z_{j+1} by 1 + d and h_{j+1,j} by 1/(1 + d), a
  // diagonal similarity of the Hessenberg matrix that leaves V exp(tau H) e_1
  // and the error estimate unchanged (and <u, u> only sets a threshold)
  typename AccSq<Acc>::F zz2 = 0, uu = 0;
  const T* __restrict__ W = static_cast<const T*>(a.win);
  const T* __restrict__ zj = static_cast<const T*>(a.zj);
  const T* __restrict__ zm = static_cast<const T*>(a.zjm1);
  T* __restrict__ zo = static_cast<T*>(a.zout);
  T* __restrict__ uo = static_cast<T*>(a.wout);
  const S* __restrict__ st = static_cast<const S*>(a.st);
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  auto orth = [&](C w, C z, C y) -> C { return orth3(ws, w, c1, z, c0, y); };

  const int t_begin = (int)(((long long)blockIdx.x * a.ntiles) / gridDim.x);
  const int t_end = (int)(((long long)(blockIdx.x + 1) * a.ntiles) / gridDim.x);
  // the ring point of this thread (tid < NRING): its staged-tile row and column
  int rr = 0, rc = 0;
  if (tid < TW) {  // south row
    rr = 0;
    rc = tid + 1;
  } else if (tid < 2 * TW) {  // north row
    rr = TILE_Y + 1;
    rc = tid - TW + 1;
  } else if (tid < 2 * TW + TILE_Y) {  // west column
    rr = tid - 2 * TW + 1;
    rc = 0;
  } else if (tid < NRING) {  // east column
    rr = tid - 2 * TW - TILE_Y + 1;
    rc = TW + 1;
  }
  // Prefetch stage: every thread copies (cp.async) exactly the values it will
  // read itself — its point pairs of W, Zhat_j, Zhat_{j-1}, the state planes
  // and the b-copies, and its ring point — so the stage needs no barrier; the
  // copies of tile k+1 are requested once tile k's staged values are consumed
  // and arrive while tile k is computed.
  auto prefetch = [&](int tile) {
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int iy0 = ty * TILE_Y, ix0 = tx * TW;
    const size_t row = (size_t)(iy0 + threadIdx.y) * nx;
    const int ix = ix0 + V * threadIdx.x;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const size_t i0 = q * plane + row + ix;
      cp_async16(stW + q * THREADS + tid, W + i0);
      cp_async16(stZ + q * THREADS + tid, zj + i0);
      if (zm) cp_async16(stM + q * THREADS + tid, zm + i0);
#pragma unroll
      for (int bq = 0; bq < KIOPS_PMAX; ++bq)
        if (bq < a.nb) cp_async16(stB + (bq * NC + q) * THREADS + tid, static_cast<const T*>(a.bz[bq]) + i0);
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) cp_async16(stG + g * THREADS + tid, st + g * plane + row + ix);
    if (tid < NRING) {
      const int gy = (iy0 + rr - 1 + ny) % ny, gx = (ix0 + rc - 1 + nx) % nx;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const size_t gq = q * plane + (size_t)gy * nx + gx;
        cp_async8(rgW + q * NRING + tid, W + gq);
        cp_async8(rgZ + q * NRING + tid, zj + gq);
        if (zm) cp_async8(rgM + q * NRING + tid, zm + gq);
      }
    }
    cp_async_commit();
  };
  if (t_begin < t_end) prefetch(t_begin);
  for (int tile = t_begin; tile < t_end; ++tile) {
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int iy0 = ty * TILE_Y, ix0 = tx * TW;
    T (*sm)[TILE_Y + 2][SW] = smb[(tile - t_begin) & 1];
    const int iy = iy0 + threadIdx.y, ix = ix0 + V * threadIdx.x;
    const size_t row = (size_t)iy * nx;
    cp_async_wait_all();  // this thread's copies of the tile have landed
    C wv[NC][V], zc[NC][V], mv[NC][V], zb[NC][V];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      lds2(reinterpret_cast<const T*>(stW + q * THREADS + tid), wv[q][0], wv[q][1]);
      lds2(reinterpret_cast<const T*>(stZ + q * THREADS + tid), zc[q][0], zc[q][1]);
      if (zm) {
        lds2(reinterpret_cast<const T*>(stM + q * THREADS + tid), mv[q][0], mv[q][1]);
      } else {
        mv[q][0] = C{};
        mv[q][1] = C{};
      }
      zb[q][0] = C{};
      zb[q][1] = C{};
#pragma unroll
      for (int bq = 0; bq < KIOPS_PMAX; ++bq) {
        if (bq < a.nb) {
          C b0, b1;
          lds2(reinterpret_cast<const T*>(stB + (bq * NC + q) * THREADS + tid), b0, b1);
          zb[q][0] = zb[q][0] + bw[bq] * b0;
          zb[q][1] = zb[q][1] + bw[bq] * b1;
        }
      }
    }
    C rv[NC];
    if (tid < NRING) {
#pragma unroll
      for (int q = 0; q < NC; ++q)
        rv[q] = orth(cv(rgW[q * NRING + tid]), cv(rgZ[q * NRING + tid]), zm ? cv(rgM[q * NRING + tid]) : C{});
    }
    // Gray-Scott state terms ga V^2, ga 2UV, formed now so that every staged
    // value is consumed before the next request overwrites the stage
    C a1[V], a2[V];
    if constexpr (OP == PHIX_OP_GRAYSCOTT) {
      C g1[V], g2[V];
      lds2(reinterpret_cast<const T*>(stG + tid), g1[0], g1[1]);
      lds2(reinterpret_cast<const T*>(stG + THREADS + tid), g2[0], g2[1]);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        a1[v] = ga * g1[v];
        a2[v] = ga * g2[v];
      }
    }
    // Zhat_{j+1} at the own points: to slot j + 1 and the staged tile
    C zn[NC][V];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        zn[q][v] = orth(wv[q][v], zc[q][v], mv[q][v]);
        sm[q][threadIdx.y + 1][V * threadIdx.x + 1 + v] = stv(zn[q][v]);
      }
      st2(zo + q * plane + row + ix, zn[q][0], zn[q][1]);
      if (tid < NRING) sm[q][rr][rc] = stv(rv[q]);
    }
    // every staged value is consumed (zn, zb, rv, a1, a2 depend on them): request
    // the next tile into the stage while this one is computed
    if (tile + 1 < t_end) prefetch(tile + 1);
    __syncthreads();
    // pass 1 of step j + 1 from the staged tile
    const int sr = threadIdx.y + 1;
    C u[NC][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int sc = V * threadIdx.x + 1 + v;
      C J[NC];
      if constexpr (OP == PHIX_OP_ADVDIFF) {
        J[0] = stencil_advdiff<C>(kk, cv(sm[0][sr][sc + 1]), cv(sm[0][sr][sc - 1]), cv(sm[0][sr + 1][sc]),
                                  cv(sm[0][sr - 1][sc]), zn[0][v]);
      } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
        stencil_gs_a<C>(kk, cv(sm[0][sr][sc + 1]), cv(sm[0][sr][sc - 1]), cv(sm[0][sr + 1][sc]),
                        cv(sm[0][sr - 1][sc]), zn[0][v], cv(sm[NC - 1][sr][sc + 1]), cv(sm[NC - 1][sr][sc - 1]),
                        cv(sm[NC - 1][sr + 1][sc]), cv(sm[NC - 1][sr - 1][sc]), zn[NC - 1][v], a1[v], a2[v], J[0],
                        J[NC - 1]);
      } else {
        const int vx = ix + v;
        const int vxm = vx == 0 ? nx - 1 : vx - 1;
        const int vxp = vx == nx - 1 ? 0 : vx + 1;
        const size_t rowp = (size_t)(iy == ny - 1 ? 0 : iy + 1) * nx;
        const size_t rowm = (size_t)(iy == 0 ? ny - 1 : iy - 1) * nx;
        C Uc = cv(__ldg(st + row + vx));
        C Ue = cv(__ldg(st + row + vxp));
        C Uw = cv(__ldg(st + row + vxm));
        C Un = cv(__ldg(st + rowp + vx));
        C Us = cv(__ldg(st + rowm + vx));
        J[0] = stencil_burgers<C>(kk, ga, cv(sm[0][sr][sc + 1]), cv(sm[0][sr][sc - 1]), cv(sm[0][sr + 1][sc]),
                                  cv(sm[0][sr - 1][sc]), zn[0][v], Ue, Uw, Un, Us, Uc);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        u[q][v] = J[q] + zb[q][v];
        zz2 = acc_sq_f(zz2, zn[q][v]);
        acc_dot(acc[1], zn[q][v], u[q][v]);
        acc_dot(acc[2], zc[q][v], u[q][v]);
        uu = acc_sq_f(uu, u[q][v]);
      }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) st2(uo + q * plane + row + ix, u[q][0], u[q][1]);
  }

  acc[0] = acc_from_f<Acc>(zz2);
  acc[3] = acc_from_f<Acc>(uu);
  if (block_partials_and_last<Acc, 4>(acc, a.partials, &kc->count)) {
    // Epilogue, a chain of float64 scalars on the critical path of every step
    // (a float64 instruction holds a pipe ~64 cycles):
    // - thread 32 reads the control values before the partials and, in the
    //   reduction's hook, forms the sums that need only the tails;
    // - thread 0 runs the short chain from the totals;
    // - one lane per warp splits one result into its float32 pair.
    constexpr int PM = KIOPS_PMAX;
    __shared__ double sx[2 * PM + 7];
    __shared__ double sv[3 + PM];
    __shared__ int s_go;
    const int j = a.j, p = a.p;
    double t1[PM], t0[PM], sj = 0.0, z0j = 0.0, eta = 0.0;
#pragma unroll
    for (int t = 0; t < PM; ++t) {
      t1[t] = (tid == 32 && t < p) ? kc->tail[(j + 1) * PM + t] : 0.0;  // tail_{j+1}, orthogonalised
      t0[t] = (tid == 32 && t < p) ? kc->tail[j * PM + t] : 0.0;        // tail_j
    }
    if (tid == 32) {
      sj = kc->s[j];
      z0j = kc->z0[j];
      eta = kc->eta;
    }
    double tot[4];
    reduce_partials<Acc, 4>(a.partials, tot, [&]() {
      if (tid == 32) {
        double T2 = 0.0, A1 = 0.0, A0 = 0.0, A2 = 0.0;
#pragma unroll
        for (int t = 0; t < PM; ++t) {
          T2 = fma(t1[t], t1[t], T2);
          if (t + 1 < PM) {
            A1 = fma(t1[t], t1[t + 1], A1);
            A0 = fma(t0[t], t1[t + 1], A0);
            A2 = fma(t1[t + 1], t1[t + 1], A2);
          }
          sx[7 + t] = t1[t];
          sx[7 + PM + t] = t0[t];
        }
        sx[0] = T2;
        sx[1] = A1;
        sx[2] = A0;
        sx[3] = A2;
        sx[4] = sj;
        sx[5] = z0j;
        sx[6] = eta;
      }
    });
    if (tid == 0) {
      // A~ z_{j+1} = s_{j+1} [u; K tail_{j+1}] with K the shift: its tail is
      // s_{j+1} tail_{j+1}[t + 1], so with 1/nz = s_{j+1}^2
      //   h_{j+1,j+1} = (<Zhat_{j+1}, u> + A1) / nz,   h_{j,j+1} = s_j s_{j+1} (<Zhat_j, u> + A0),
      //   ||A~ z_{j+1}||^2 = (<u, u> + A2) / nz
      const double nz = tot[0] + sx[0];
      double s1, hn;
      rsqrt_and_sqrt(nz, s1, hn);
      kc->hl[j] = hn;
      int go = 0;
      if (!isfinite(hn)) {
        kc->status = PHIX_ENAN;
        kc->stop = 1;
      } else if (hn <= 1e-12 * sx[5]) {
        kc->stop = 1;  // happy breakdown: exact invariant subspace of dimension j+1
        kc->happy_m = j + 1;
      } else {
        const double r2 = s1 * s1, sj2 = sx[4];
        const double h11 = (tot[1] + sx[1]) * r2, h01 = sj2 * s1 * (tot[2] + sx[2]);
        const double zz = (tot[3] + sx[3]) * r2;
        const double cc1 = h11 * s1, cc0 = h01 * sj2;
        kc->s[j + 1] = s1;
        kc->wsd = s1;
        kc->hd[j + 1] = h11;
        kc->hu[j + 1] = h01;
        kc->c1d = cc1;
        kc->c0d = cc0;
        sv[0] = s1;
        sv[1] = cc1;
        sv[2] = cc0;
        // tail_{j+2} = s_{j+1} tail_{j+1}[t + 1] - c1 tail_{j+1} - c0 tail_j (orthogonalised)
        // and the b-column weights of the next fused step
        double* t2 = kc->tail + (j + 2) * PM;
        for (int t = 0; t < p; ++t) {
          const double tz = (t + 1 < p) ? s1 * sx[7 + t + 1] : 0.0;
          const double v = tz - cc1 * sx[7 + t] - cc0 * sx[7 + PM + t];
          t2[t] = v;
          const double bb = sx[6] * v;
          kc->bud[t] = bb;
          sv[3 + t] = bb;
        }
        // ||A~ z_{j+1}|| only sets the happy-breakdown threshold: float32 square root in range
        kc->z0[j + 1] = (zz > 1e-30 && zz < 1e30) ? (double)sqrtf((float)zz) : sqrt(zz);
        if (!isfinite(h11) || !isfinite(h01) || !isfinite(zz)) {
          kc->status = PHIX_ENAN;
          kc->stop = 1;
        } else {
          go = 1;
        }
      }
      s_go = go;
      kc->count = 0;
    }
    __syncthreads();
    // float32 pairs of s_{j+1} (twice), c1, c0 and the b weights: one lane per warp
    if (s_go && (tid & 31) == 0) {
      const int k = tid >> 5;
      if (k < 3 + p) {
        const float2 f = split2d(sv[k]);
        if (k == 0) {
          kc->sf[j + 1] = f;
          kc->wsf = f;
        } else if (k == 1) {
          kc->c1f = f;
        } else if (k == 2) {
          kc->c0f = f;
        } else {
          kc->buf[k - 3] = f;
        }
      }
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
  // ||z||^2 in float32 on the double-float path (the normalisation error is a
  // diagonal similarity of the Hessenberg matrix: no effect on the result)
  typename AccSq<Acc>::F zz = 0;
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
    zz = acc_sq_f(zz, z0);
    zz = acc_sq_f(zz, z1);
  };
  auto single = [&](size_t i) {
    C z = ldw1(zo + i) - c1 * ldr1(zj + i);
    if (zm) z = z - c0 * ldr1(zm + i);
    st1(zo + i, z);
    zz = acc_sq_f(zz, z);
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
  acc[0] = acc_from_f<Acc>(zz);
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
  float2 n2[2][2][KIOPS_MMAX + 6];  // Chebyshev pairs (T_{k-1}, T_k), ping-pong; row i at i + 2, zero pads
  df bes[CHEB_MAX + 2];
  short bres[CHEB_MAX + 2];           // rescalings of the Miller recurrence before bes[k] was stored
  int nres;                           // and in all
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
// Terms advance two at a time from (T_{k-1}, T_k):
//   T_{k+1} = M T_k - T_{k-1},   T_{k+2} = (M^2 - I) T_k - M T_{k-1},
// the pentadiagonal M^2 - I in pc (columns i-2 .. i+2 of row i): both new
// terms depend only on the pair before, so a pair of terms takes one exchange
// through shared memory and one barrier (the arithmetic per term is not
// reduced: the step is bound by each row's dependent double-float operations).
template <int R>
__device__ void cheb_segments(int n, int S, int K, const df (&ma)[R], const df (&mu)[R], const df (&ml)[R],
                              const df (&pc)[R][5], df (&xr)[R], double& lead, SmallExpWork& w, int tid) {
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
    // rows of the exchanged terms: row i at index i + 2, zero pads around
    df tm[R], tc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = tid + q * SX;
      if (i < n) w.n2[0][0][i + 2] = make_float2(xr[q].hi, xr[q].lo);
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
        df_prod(mu[q], cv(w.n2[0][0][i + 3]), p[1], e[1]);
        df_prod(ml[q], cv(w.n2[0][0][i + 1]), p[2], e[2]);
        const df v = df_scale2(df_sum_pairs<3>(p, e), 0.5f);
        w.n2[0][1][i + 2] = make_float2(v.hi, v.lo);
        xr[q] = df_fma(b1, v, df_mul(b0, xr[q]));
        tc[q] = v;
      }
    }
    __syncthreads();
    // pairs: tm = T_{k-1}, tc = T_k, also in n2[par][0], n2[par][1]
    int k = 1, par = 0;
    for (; k + 2 < K; k += 2) {
      const float2* om = w.n2[par][0];
      const float2* oc = w.n2[par][1];
      float2* nm = w.n2[par ^ 1][0];
      float2* nc = w.n2[par ^ 1][1];
      const df c1 = df_scale2(w.bes[k + 1], 2.f), c2 = df_scale2(w.bes[k + 2], 2.f);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = tid + q * SX;
        if (i < n) {
          const df cw2 = cv(oc[i]), cw1 = cv(oc[i + 1]), ce1 = cv(oc[i + 3]), ce2 = cv(oc[i + 4]);
          const df mw1 = cv(om[i + 1]), me1 = cv(om[i + 3]);
          float p[4], e[4];
          df_prod(ma[q], tc[q], p[0], e[0]);
          df_prod(mu[q], ce1, p[1], e[1]);
          df_prod(ml[q], cw1, p[2], e[2]);
          p[3] = -tm[q].hi;
          e[3] = -tm[q].lo;
          const df v1 = df_sum_pairs<4>(p, e);
          float P[8], E[8];
          df_prod(pc[q][0], cw2, P[0], E[0]);
          df_prod(pc[q][1], cw1, P[1], E[1]);
          df_prod(pc[q][2], tc[q], P[2], E[2]);
          df_prod(pc[q][3], ce1, P[3], E[3]);
          df_prod(pc[q][4], ce2, P[4], E[4]);
          df_prod(df_neg(ma[q]), tm[q], P[5], E[5]);
          df_prod(df_neg(mu[q]), me1, P[6], E[6]);
          df_prod(df_neg(ml[q]), mw1, P[7], E[7]);
          const df v2 = df_sum_pairs<8>(P, E);
          nm[i + 2] = make_float2(v1.hi, v1.lo);
          nc[i + 2] = make_float2(v2.hi, v2.lo);
          xr[q] = df_fma(c2, v2, df_fma(c1, v1, xr[q]));
          tm[q] = v1;
          tc[q] = v2;
        }
      }
      par ^= 1;
      __syncthreads();
    }
    // one last term when K - 2 is odd
    if (k + 1 < K) {
      const float2* oc = w.n2[par][1];
      const df c1 = df_scale2(w.bes[k + 1], 2.f);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = tid + q * SX;
        if (i < n) {
          float p[4], e[4];
          df_prod(ma[q], tc[q], p[0], e[0]);
          df_prod(mu[q], cv(oc[i + 3]), p[1], e[1]);
          df_prod(ml[q], cv(oc[i + 1]), p[2], e[2]);
          p[3] = -tm[q].hi;
          e[3] = -tm[q].lo;
          xr[q] = df_fma(c1, df_sum_pairs<4>(p, e), xr[q]);
        }
      }
    }
    __syncthreads();  // every read of n2 done before the next segment writes it
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
  if (mode == 0) {
    // row i of M^2 - I (float64 from the float64 entries of M: a diagonal,
    // u super-, l sub-diagonal; entries outside the matrix are zero)
    df pc[R][5];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = tid + q * SX;
      const bool in = i < n;
      auto a_ = [&](int j) { return (j >= 0 && j < n) ? (dg[j] - c) * cscale : 0.0; };
      auto u_ = [&](int j) { return (j >= 0 && j + 1 < n) ? up[j] * cscale : 0.0; };
      auto l_ = [&](int j) { return (j >= 1 && j < n) ? lo[j - 1] * cscale : 0.0; };
      const double ai = a_(i), ui = u_(i), li = l_(i);
      pc[q][0] = dfd(in ? li * l_(i - 1) : 0.0);
      pc[q][1] = dfd(in ? li * (ai + a_(i - 1)) : 0.0);
      pc[q][2] = dfd(in ? ai * ai + ui * l_(i + 1) + li * u_(i - 1) - 1.0 : 0.0);
      pc[q][3] = dfd(in ? ui * (ai + a_(i + 1)) : 0.0);
      pc[q][4] = dfd(in ? ui * u_(i + 1) : 0.0);
    }
    cheb_segments<R>(n, S, K, ma, mu, ml, pc, xr, lead, w, tid);
  } else
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
        // The values already stored are rescaled with the recurrence; a stored
        // value only records how many rescalings preceded it (bres), and the
        // ones that follow are applied below, in parallel, off this serial chain.
        df ip1 = df_make(0.f, 0.f), ik = df_make(1e-30f, 0.f);
        int nres = 0;
        for (int k = kstart; k >= 0; --k) {
          if (k <= kmax) {
            w.bes[k] = ik;
            w.bres[k] = (short)nres;
          }
          const df im1 = df_fma(df_mul(df_make((float)k, 0.f), ir2), ik, ip1);
          ip1 = ik;
          ik = im1;
          if (fabsf(ik.hi) > 1e30f) {
            ik = df_scale2(ik, 0x1p-100f);
            ip1 = df_scale2(ip1, 0x1p-100f);
            ++nres;
          }
        }
        w.nres = nres;
      }
      __syncthreads();
      // each stored value times 2^-100 once per later rescaling, in sequence (the
      // same products as rescaling every stored value at each event)
      for (int k = tid; k <= kmax; k += SX) {
        df bv = w.bes[k];
        for (int q = w.bres[k]; q < w.nres; ++q) bv = df_scale2(bv, 0x1p-100f);
        w.bes[k] = bv;
      }
      // normalise: I~_0 + 2 sum_{k >= 1} I~_k = 1 (each thread sums the entries it rescaled)
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
  for (int i = tid; i < KIOPS_MMAX + 6; i += SX)
    for (int a = 0; a < 4; ++a) w.n2[a >> 1][a & 1][i] = make_float2(0.f, 0.f);
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

__global__ void __launch_bounds__(SX) k_kexp(KiopsCtl* kc, int m, double tau, double tau_end, double tol,
                                              KiopsMailbox* mbox, unsigned int seq) {
  __shared__ double dg[KIOPS_MMAX + 2], up[KIOPS_MMAX + 2], lo[KIOPS_MMAX + 2];
  __shared__ SmallExpWork w;
  const int tid = threadIdx.x;
  // one row of the matrix per thread (independent loads, not a serial chain)
  const int hm = __ldcg(&kc->happy_m);
  const int mm = hm > 0 ? hm : m;
  const int n = hm > 0 ? hm : m + 1;
  for (int i = tid; i < n; i += 128) {
    dg[i] = tau * (i < mm ? __ldcg(&kc->hd[i]) : 0.0);          // row m of Hbar has no diagonal
    up[i] = tau * ((i + 1 < mm) ? __ldcg(&kc->hu[i + 1]) : 0.0);  // (i, i+1); column m is zero
    lo[i] = tau * ((i + 1 < n) ? __ldcg(&kc->hl[i]) : 0.0);       // (i+1, i)
  }
  __syncthreads();
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
    if (mbox) {
      // the decision's inputs to the host: the header, then its sequence number
      const unsigned int* src = reinterpret_cast<const unsigned int*>(kc);
      unsigned int* dst = reinterpret_cast<unsigned int*>(mbox->header);
      for (int i = 0; i < (int)(KIOPS_HOST_BYTES / 4); ++i) dst[i] = __ldcg(src + i);
      __threadfence_system();
      mbox->seq = seq;
    }
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
  int pairs;  // N even, slots and out 16-byte aligned: 16-byte loads of element pairs
  double h;
  double kJ[8];
};

template <int P>
__global__ void __launch_bounds__(THREADS, 4) k_kcomb(CombArgs a, size_t N) {
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
  // Double-float path: pairs of elements, one 16-byte load per basis vector
  // (a.pairs: N even, every slot and the output 16-byte aligned).  The loads
  // of KC basis vectors are issued before their products are summed, so a
  // thread waits for memory once per KC terms instead of once per term; the
  // sum runs in the basis order, the same arithmetic as the element loop
  // below.  (The float64 path is bound by GB300's float64 rate, not by these
  // latencies: it keeps the element loop.)
  size_t i0 = 0;
  if (P == P_DF64 && a.pairs) {
    constexpr int KC = 8;
    const size_t np = N / 2;
    for (size_t v = (size_t)blockIdx.x * THREADS + tid; v < np; v += stride) {
      C w0{}, w1{};
      for (int k0 = 0; k0 < a.n; k0 += KC) {
        C x0[KC], x1[KC];
#pragma unroll
        for (int q = 0; q < KC; ++q)
          if (k0 + q < a.n) ldr2(zp[k0 + q] + 2 * v, x0[q], x1[q]);
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          if (k0 + q < a.n) {
            const C c = cf[k0 + q];
            if (k0 + q == 0) {
              w0 = c * x0[q];
              w1 = c * x1[q];
            } else {
              w0 = w0 + c * x0[q];
              w1 = w1 + c * x1[q];
            }
          }
        }
      }
      st2(z0 + 2 * v, w0, w1);
      if (a.out) {
        double d0, d1;
        if constexpr (P == P_FP64) {
          d0 = w0;
          d1 = w1;
        } else {
          d0 = df_to_double_pow2(w0, 0);
          d1 = df_to_double_pow2(w1, 0);
        }
        *reinterpret_cast<double2*>(a.out + 2 * v) = make_double2(a.scale * d0, a.scale * d1);
      }
      acc_dot(acc[0], w0, w0);
      acc_dot(acc[0], w1, w1);
    }
    i0 = 2 * np;
  }
  for (size_t i = i0 + (size_t)blockIdx.x * THREADS + tid; i < N; i += stride) {
    C w = cf[0] * ldr1(zp[0] + i);
    for (int k = 1; k < a.n; ++k) w = w + cf[k] * ldr1(zp[k] + i);
    st1(z0 + i, w);
    if (a.out) {
      double d;
      if constexpr (P == P_FP64)
        d = w;
      else
        d = df_to_double_pow2(w, 0);
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
  auto body = [&](size_t i, double x) {
    C w;
    if constexpr (P == P_FP64)
      w = x;
    else
      w = df_split_pow2(x, 0);
    st1(z0 + i, w);
    acc_dot(acc[0], w, w);
  };
  size_t i = (size_t)blockIdx.x * THREADS + tid;
  for (; i + (UNR - 1) * stride < N; i += UNR * stride) {
    double x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = b0 ? c * __ldg(b0 + i + u * stride) : 0.0;  // c: a power of two, exact
#pragma unroll
    for (int u = 0; u < UNR; ++u) body(i + u * stride, x[u]);
  }
  for (; i < N; i += stride) body(i, b0 ? c * __ldg(b0 + i) : 0.0);
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
  auto body = [&](size_t i, double x) {
    acc[0] += fabs(x);
    if (!out) return;  // norm only
    if constexpr (P == P_FP64)
      out[i] = x;
    else {
      df w = df_split_pow2(x, 0);
      out[i] = make_float2(w.hi, w.lo);
    }
  };
  // the thread's elements in grid-stride order, their loads issued UNR at a time
  size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
  for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
    double x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = __ldg(b + i + u * stride);
#pragma unroll
    for (int u = 0; u < UNR; ++u) body(i + u * stride, x[u]);
  }
  for (; i < n; i += stride) body(i, __ldg(b + i));
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
  a.gkind = s.op;
  for (int i = 0; i < 8; ++i) a.gprm[i] = s.prm[i];
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
int blocks_per_sm(const void* fn, size_t dsmem = 0) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, THREADS, dsmem) != cudaSuccess) {
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
  const size_t N = (size_t)s.nx * s.ny * op_ncomp(OP);
  k_arn2<P><<<s.nsm * occ2, dim3(32, TILE_Y), 0, st>>>(a, N);
  return cudaGetLastError();
}

// pass 1 of step 0 into W0, fused steps feeding on it
template <int P, int OP>
cudaError_t fused_first_t(const KiopsSpec& s, cudaStream_t st) {
  static const int occ = blocks_per_sm(reinterpret_cast<const void*>(k_arn1<P, OP, 2>));
  ArnArgs a = make_arn(s, 0, 2);
  a.zout = s.W[0];
  a.fused = 1;
  k_arn1<P, OP, 2><<<std::min(s.nsm * occ, a.ntiles), dim3(32, TILE_Y), 0, st>>>(a);
  return cudaGetLastError();
}

// dynamic shared memory of a fused launch with nb b-columns
template <int P, int OP>
int arnf_smem(int nb) {
  constexpr int nc = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 1, ng = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 0;
  return arnf_smem_bytes(nc, ng, nb, (int)sizeof(typename KTr<P>::T));
}

// the kernel's dynamic shared-memory limit raised to its largest layout (once),
// and its occupancy at that layout
template <int P, int OP>
int arnf_setup() {
  const void* fn = reinterpret_cast<const void*>(k_arnf<P, OP>);
  const int smax = arnf_smem<P, OP>(KIOPS_PMAX);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smax) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return blocks_per_sm(fn, (size_t)smax);
}

template <int P, int OP>
cudaError_t fused_step_t(const KiopsSpec& s, int j, cudaStream_t st) {
  static const int occ = arnf_setup<P, OP>();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  ArnArgs a = make_arn(s, j, 2);
  a.win = s.W[j & 1];
  a.wout = s.W[(j + 1) & 1];
  k_arnf<P, OP><<<std::min(s.nsm * occ, a.ntiles), dim3(32, TILE_Y), arnf_smem<P, OP>(s.nb), st>>>(a);
  return cudaGetLastError();
}

template <int P>
cudaError_t fused_p(const KiopsSpec& s, int j, bool first, cudaStream_t st) {
  switch (s.op) {
    case PHIX_OP_ADVDIFF:
      return first ? fused_first_t<P, PHIX_OP_ADVDIFF>(s, st) : fused_step_t<P, PHIX_OP_ADVDIFF>(s, j, st);
    case PHIX_OP_GRAYSCOTT:
      return first ? fused_first_t<P, PHIX_OP_GRAYSCOTT>(s, st) : fused_step_t<P, PHIX_OP_GRAYSCOTT>(s, j, st);
    case PHIX_OP_BURGERS:
      return first ? fused_first_t<P, PHIX_OP_BURGERS>(s, st) : fused_step_t<P, PHIX_OP_BURGERS>(s, j, st);
  }
  return cudaErrorInvalidValue;
}

// general operators: float64 pass 1 on k_arn1g, then the common pass 2
cudaError_t arn_general(const KiopsSpec& s, int j, cudaStream_t st) {
  static const int occ1 = blocks_per_sm(reinterpret_cast<const void*>(k_arn1g));
  static const int occ2 = blocks_per_sm(reinterpret_cast<const void*>(k_arn2<P_FP64>));
  ArnArgs a = make_arn(s, j, 1);
  const size_t plane = (size_t)s.nx * s.ny;
  const int g1 = (int)std::min<size_t>((size_t)s.nsm * occ1, (plane + THREADS - 1) / THREADS);
  k_arn1g<<<g1, dim3(32, TILE_Y), 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_arn2<P_FP64><<<s.nsm * occ2, dim3(32, TILE_Y), 0, st>>>(a, plane * op_ncomp(s.op));
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
  if (P == P_FP64 && s.op >= PHIX_OP_ADR) return arn_general(s, j, st);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t kiops_arnoldi(const KiopsSpec& s, int j, cudaStream_t st) {
  return s.prec == P_FP64 ? arn_p<P_FP64>(s, j, st) : arn_p<P_DF64>(s, j, st);
}

bool kiops_fused_ok(const KiopsSpec& s) {
  return s.op <= PHIX_OP_BURGERS && s.nx % 64 == 0 && s.ny % TILE_Y == 0 && s.W[0] != nullptr &&
         s.W[1] != nullptr;
}

cudaError_t kiops_fused_first(const KiopsSpec& s, cudaStream_t st) {
  return s.prec == P_FP64 ? fused_p<P_FP64>(s, 0, true, st) : fused_p<P_DF64>(s, 0, true, st);
}

cudaError_t kiops_fused_step(const KiopsSpec& s, int j, cudaStream_t st) {
  return s.prec == P_FP64 ? fused_p<P_FP64>(s, j, false, st) : fused_p<P_DF64>(s, j, false, st);
}

cudaError_t small_expm_e1(int n, const double* d, const double* u, const double* l, double tau, double* out,
                          int* mode, cudaStream_t st) {
  if (n < 1 || n > KIOPS_MMAX + 1) return cudaErrorInvalidValue;
  k_smallexp<<<1, 128, 0, st>>>(n, d, u, l, tau, out, mode);
  return cudaGetLastError();
}

cudaError_t kiops_smallexp(KiopsCtl* kc, int m, double tau, double tau_end, double tol, KiopsMailbox* mbox,
                           unsigned int seq, cudaStream_t st) {
  k_kexp<<<1, 128, 0, st>>>(kc, m, tau, tau_end, tol, mbox, seq);
  return cudaGetLastError();
}

cudaError_t kiops_combine(const KiopsSpec& s, int n, double* out, double scale, cudaStream_t st) {
  const size_t N = (size_t)s.nx * s.ny * op_ncomp(s.op);
  CombArgs c = make_comb(s, n, out, scale);
  bool al = N % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  for (int k = 0; k < n; ++k) al = al && (reinterpret_cast<uintptr_t>(s.Zh[k]) & 15) == 0;
  c.pairs = al ? 1 : 0;
  if (s.prec == P_FP64)
    k_kcomb<P_FP64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(c, N);
  else
    k_kcomb<P_DF64><<<s.grid, dim3(32, TILE_Y), 0, st>>>(c, N);
  return cudaGetLastError();
}

cudaError_t kiops_start(const KiopsSpec& s, const double* b0, double eta, double cscale, cudaStream_t st) {
  const size_t N = (size_t)s.nx * s.ny * op_ncomp(s.op);
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
