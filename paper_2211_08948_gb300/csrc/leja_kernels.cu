// Iteration kernels of the real-Leja phi-action (Sec. 2.2 of the paper) and
// of the power iteration that estimates the spectral interval.
//
// One launch = one iteration over the whole grid:
//   MODE_NEWTON: y_m = ((J - c)/gamma - xi_{m-1}) y_{m-1}          (Newton basis)
//                p_m^(k) = p_{m-1}^(k) + d_k[m] y_m,  k < K          (vertical, Sec. 4)
//                partial sums of ||y_m||^2 and ||p_m^(k)||^2
//   MODE_POWER:  y_k = J y_{k-1} / ||y_{k-1}||, partial sums of ||y_k||^2
// and the last block to finish reduces the partials in block order
// (deterministic), applies the stop test |d_k[m]| ||y_m|| <= tol ||p_m^(k)||
// (m >= m_min) or the power-iteration relative-change test, and sets
// ctl->done.  Every launch first reads ctl->done and returns if set, so a
// chain of launches stops itself on the device.
//
// Layout: planar float64-sized elements (double, or a float2 hi/lo pair),
// 2D periodic grid, 32 x 8 thread tiles, V = 2 consecutive x points per
// thread (16-byte loads) when nx is even, grid-stride over tiles.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "iter_common.cuh"

namespace phix {

// ---------------------------------------------------------------------------
// Kernel arguments (identical for every launch of a chain) and parameter access
// ---------------------------------------------------------------------------
struct IterDev {
  const void* y[2];
  void* p[KMAX];
  const void* st;
  LejaCtl* ctl;
  double* partials;
  const unsigned char* ptab;
  int nx, ny, ntiles, tiles_x;
  int use_cond;
  cudaGraphConditionalHandle cond;
};

// Inside a conditional WHILE node: stop the loop (one thread per launch).
__device__ __forceinline__ void stop_loop(const IterDev& a) {
  if (a.use_cond) cudaGraphSetConditional(a.cond, 0);
}


// ---------------------------------------------------------------------------
// The iteration kernel.
// ---------------------------------------------------------------------------
template <int P, int OP, int V, int MODE, int PERSIST>
__global__ void __launch_bounds__(THREADS, 2) k_iter(IterDev a) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  using CJ = typename Tr<P>::CJ;
  using S = typename Tr<P>::S;
  using Acc = typename std::conditional<MODE == MODE_NEWTON, typename Tr<P>::AccN,
                                        typename Tr<P>::AccP>::type;
  constexpr int NC = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 1;
  // FP32_JV keeps the stencil in float32 and the shift in double-float: no folding
  constexpr bool FOLD = (MODE == MODE_NEWTON) && std::is_same<C, CJ>::value;

  // the control word, the iteration index and the parameter header are
  // independent loads: issued together, one round trip before the
  // coefficient and tile loads (the stop flag is tested after them)
  const int done0 = __ldcg(&a.ctl->done);
  int m = __ldcg(&a.ctl->m);
  const PassParams* pp = pp_of(a.ptab);
  const int M = pp->M;
  const int K = (MODE == MODE_NEWTON) ? pp->K : 0;
  const CJ ga = coef<CJ>(pp->gad, pp->gaf);
  const bool prescaled = MODE == MODE_NEWTON && pp->prescaled;
  if (done0) {  // the chain already stopped
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) stop_loop(a);
    return;
  }
  // PERSIST: every iteration of the chain in this one (cooperative) launch,
  // one grid barrier per iteration; otherwise one iteration per launch
  for (;;) {
  CJ kk[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) kk[j] = coef<CJ>(pp->kd[j], pp->kf[j]);
  C beta{};
  C dk[KMAX];
  C alpha_pw{};
  if (MODE == MODE_NEWTON) {
    beta = coef<C>(beta_d_of(a.ptab, M)[m], beta_f_of(a.ptab, M)[m]);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      dk[k] = (k < K) ? coef<C>(dk_d_of(a.ptab, M)[k * M + m], dk_f_of(a.ptab, M)[k * M + m]) : C{};
    if constexpr (FOLD) {
      kk[Centre<OP>::a] = kk[Centre<OP>::a] + from_cj(beta, CJ());
      if constexpr (Centre<OP>::b >= 0) kk[Centre<OP>::b] = kk[Centre<OP>::b] + from_cj(beta, CJ());
    }
  } else {
    if constexpr (P == P_FP64) {
      alpha_pw = __ldcg(&a.ctl->alpha);
    } else if constexpr (P == P_FP32) {
      alpha_pw = __ldcg(&a.ctl->alpha_hi);
    } else {
      alpha_pw = df_make(__ldcg(&a.ctl->alpha_hi), __ldcg(&a.ctl->alpha_lo));
    }
  }

  Acc acc[KMAX + 1];
#pragma unroll
  for (int j = 0; j <= KMAX; ++j) acc[j] = acc_zero<Acc>();

  // (selects, not a runtime index into the argument block, which would copy
  // the block to local memory)
  const bool odd = m & 1;
  const T* __restrict__ yin = static_cast<const T*>(odd ? a.y[0] : a.y[1]);
  T* __restrict__ yout = static_cast<T*>(const_cast<void*>(odd ? a.y[1] : a.y[0]));
  const S* __restrict__ st = static_cast<const S*>(a.st);
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int iy = ty * TILE_Y + threadIdx.y;
    const int ix = (tx * 32 + threadIdx.x) * V;
    if (iy >= ny || ix >= nx) continue;
    const int iym = iy == 0 ? ny - 1 : iy - 1;
    const int iyp = iy == ny - 1 ? 0 : iy + 1;
    const int ixm = ix == 0 ? nx - 1 : ix - 1;
    const int ixp = (ix + V == nx) ? 0 : ix + V;
    const size_t row = (size_t)iy * nx, rowp = (size_t)iyp * nx, rowm = (size_t)iym * nx;

    // load y (both species for GS): centre pair, north/south pairs, west/east
    C c[NC][V], nn[NC][V], ss[NC][V], we[NC], ea[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const T* b = yin + q * plane;
      if constexpr (V == 2) {
        ldy2<PERSIST>(b + row + ix, c[q][0], c[q][1]);
        ldy2<PERSIST>(b + rowp + ix, nn[q][0], nn[q][1]);
        ldy2<PERSIST>(b + rowm + ix, ss[q][0], ss[q][1]);
      } else {
        c[q][0] = ldy1<PERSIST>(b + row + ix);
        nn[q][0] = ldy1<PERSIST>(b + rowp + ix);
        ss[q][0] = ldy1<PERSIST>(b + rowm + ix);
      }
      we[q] = ldy1<PERSIST>(b + row + ixm);
      ea[q] = ldy1<PERSIST>(b + row + ixp);
    }

    // accumulators p_k, loaded before any store of this tile so that all
    // loads are in flight together (p and y may alias as far as the compiler
    // knows, so it would not move these loads above the stores by itself)
    C pv[NC][KMAX][V];
    if constexpr (MODE == MODE_NEWTON) {
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int kq = 0; kq < KMAX; ++kq) {
          if (kq < K) {
            const T* pp2 = static_cast<const T*>(a.p[kq]) + q * plane + row + ix;
            if constexpr (V == 2)
              ldw2(pp2, pv[q][kq][0], pv[q][kq][1]);
            else
              pv[q][kq][0] = ldw1(pp2);
          }
        }
    }

    C out[NC][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      CJ J[NC];
      if constexpr (OP == PHIX_OP_ADVDIFF) {
        C e = (v == V - 1) ? ea[0] : c[0][v + 1];
        C w = (v == 0) ? we[0] : c[0][v - 1];
        J[0] = stencil_advdiff<CJ>(kk, to_cj(e, CJ()), to_cj(w, CJ()), to_cj(nn[0][v], CJ()),
                                   to_cj(ss[0][v], CJ()), to_cj(c[0][v], CJ()));
      } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
        C eu = (v == V - 1) ? ea[0] : c[0][v + 1];
        C wu = (v == 0) ? we[0] : c[0][v - 1];
        C ev = (v == V - 1) ? ea[NC - 1] : c[NC - 1][v + 1];
        C wv = (v == 0) ? we[NC - 1] : c[NC - 1][v - 1];
        CJ g1 = to_cj(cv(__ldg(st + row + ix + v)), CJ());
        CJ g2 = to_cj(cv(__ldg(st + plane + row + ix + v)), CJ());
        if (!prescaled) {
          g1 = ga * g1;
          g2 = ga * g2;
        }
        stencil_gs_a<CJ>(kk, to_cj(eu, CJ()), to_cj(wu, CJ()), to_cj(nn[0][v], CJ()), to_cj(ss[0][v], CJ()),
                         to_cj(c[0][v], CJ()), to_cj(ev, CJ()), to_cj(wv, CJ()), to_cj(nn[NC - 1][v], CJ()),
                         to_cj(ss[NC - 1][v], CJ()), to_cj(c[NC - 1][v], CJ()), g1, g2, J[0], J[NC - 1]);
      } else {
        C e = (v == V - 1) ? ea[0] : c[0][v + 1];
        C w = (v == 0) ? we[0] : c[0][v - 1];
        const int vx = ix + v;
        const int vxm = (v == 0) ? ixm : vx - 1;
        const int vxp = (v == V - 1) ? ixp : vx + 1;
        CJ Uc = to_cj(cv(__ldg(st + row + vx)), CJ());
        CJ Ue = to_cj(cv(__ldg(st + row + vxp)), CJ());
        CJ Uw = to_cj(cv(__ldg(st + row + vxm)), CJ());
        CJ Un = to_cj(cv(__ldg(st + rowp + vx)), CJ());
        CJ Us = to_cj(cv(__ldg(st + rowm + vx)), CJ());
        J[0] = stencil_burgers<CJ>(kk, ga, to_cj(e, CJ()), to_cj(w, CJ()), to_cj(nn[0][v], CJ()),
                                   to_cj(ss[0][v], CJ()), to_cj(c[0][v], CJ()), Ue, Uw, Un, Us, Uc);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if constexpr (MODE == MODE_NEWTON) {
          if constexpr (FOLD)
            out[q][v] = from_cj(J[q], C());
          else
            out[q][v] = from_cj(J[q], C()) + beta * c[q][v];
        } else {
          out[q][v] = alpha_pw * from_cj(J[q], C());
        }
      }
    }

    // store y, accumulate p_k, norms
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      T* yo = yout + q * plane + row + ix;
      if constexpr (V == 2) {
        st2(yo, out[q][0], out[q][1]);
      } else {
        st1(yo, out[q][0]);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) acc_sq(acc[0], out[q][v]);
      if (MODE == MODE_NEWTON) {
#pragma unroll
        for (int kq = 0; kq < KMAX; ++kq) {
          if (kq < K) {
            T* pp2 = static_cast<T*>(a.p[kq]) + q * plane + row + ix;
            if constexpr (V == 2) {
              const C p0 = mad(dk[kq], out[q][0], pv[q][kq][0]);
              const C p1 = mad(dk[kq], out[q][1], pv[q][kq][1]);
              st2(pp2, p0, p1);
              acc_sq(acc[1 + kq], p0);
              acc_sq(acc[1 + kq], p1);
            } else {
              const C p0 = mad(dk[kq], out[q][0], pv[q][kq][0]);
              st1(pp2, p0);
              acc_sq(acc[1 + kq], p0);
            }
          }
        }
      }
    }
  }

  if constexpr (PERSIST) {
    // block partials into this iteration's half of the partials buffer (the
    // halves alternate, so a block can write iteration m + 1's sums while a
    // slower one still reads iteration m's), the grid barrier, then every
    // block forms the same totals in the same order and takes the same stop
    // decision; block 0 records it in the control block
    static_assert(MODE == MODE_NEWTON, "persistent chains run Newton-Leja passes");
    double* part = a.partials + (size_t)(m & 1) * gridDim.x * (KMAX + 1);
    block_partials_only<Acc, KMAX + 1>(acc, part);
    if (!grid_barrier(&a.ctl->bar_count, &a.ctl->bar_gen)) {
      if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        a.ctl->status = PHIX_ETIMEOUT;
        a.ctl->iters = m;
        a.ctl->done = 1;
      }
      return;
    }
    __shared__ int s_done;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    LejaCtl local{};
    if constexpr (PartialsDF<Acc>::value) {
      float2 qk[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        qk[k] = (tid == 0 && k < K) ? q_f_of(a.ptab, M)[k * M + m] : make_float2(0.f, 0.f);
      df tot[KMAX + 1];
      reduce_partials_df<Acc, KMAX + 1>(part, tot, K + 1);
      if (tid == 0) leja_test_df(&local, m, K, pp->m_min, pp->m_max, qk, tot);
    } else {
      double dkd[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) dkd[k] = (tid == 0 && k < K) ? dk_d_of(a.ptab, M)[k * M + m] : 0.0;
      double tot[KMAX + 1];
      reduce_partials<Acc, KMAX + 1>(part, tot, NoHook{}, K + 1);
      if (tid == 0) leja_test(&local, m, K, pp->m_min, pp->m_max, pp->tol, dkd, tot);
    }
    if (tid == 0) {
      s_done = local.done;
      if (blockIdx.x == 0) {
        LejaCtl* ctl = a.ctl;
        if (local.done) {
          ctl->status = local.status;
          ctl->iters = local.iters;
          ctl->ysq = local.ysq;
          for (int k = 0; k < KMAX; ++k) ctl->psq[k] = local.psq[k];
          ctl->done = 1;
        }
        ctl->m = m + 1;
      }
    }
    __syncthreads();
    if (s_done) return;
    ++m;
    continue;
  }
  if (block_partials_and_last<Acc, KMAX + 1>(acc, a.partials, &a.ctl->count)) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if constexpr (MODE == MODE_NEWTON && PartialsDF<Acc>::value) {
      // the test's factors (d_k[m]/tol)^2, read before the partials so that their
      // latency overlaps the reduction; totals and test in double-float
      float2 qk[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        qk[k] = (tid == 0 && k < K) ? q_f_of(a.ptab, M)[k * M + m] : make_float2(0.f, 0.f);
      df tot[KMAX + 1];
      reduce_partials_df<Acc, KMAX + 1>(a.partials, tot, K + 1);
      if (tid == 0) {
        LejaCtl* ctl = a.ctl;
        leja_test_df(ctl, m, K, pp->m_min, pp->m_max, qk, tot);
        ctl->m = m + 1;
        ctl->count = 0;
        if (ctl->done) stop_loop(a);
      }
    } else {
      // the stop test's coefficients, read before the partials so that their
      // latency overlaps the reduction
      double dkd[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) dkd[k] = (MODE == MODE_NEWTON && tid == 0 && k < K) ? dk_d_of(a.ptab, M)[k * M + m] : 0.0;
      double tot[KMAX + 1];
      reduce_partials<Acc, KMAX + 1>(a.partials, tot, NoHook{}, MODE == MODE_NEWTON ? K + 1 : 1);
      if (tid == 0) {
        LejaCtl* ctl = a.ctl;
        if (MODE == MODE_NEWTON) {
          leja_test(ctl, m, K, pp->m_min, pp->m_max, pp->tol, dkd, tot);
        } else {
          // power iteration: y_k = J v_{k-1}, v_{k-1} unit  =>  rho_k = ||y_k||
          double rho = sqrt(tot[0]);
          double prev = ctl->rho;
          ctl->rho_prev = prev;
          ctl->rho = rho;
          ctl->iters = m;
          if (!isfinite(rho)) {
            ctl->status = PHIX_ENAN;
            ctl->done = 1;
          } else if (rho == 0.0) {
            ctl->status = PHIX_OK;
            ctl->done = 1;
          } else if ((m >= 2 && fabs(rho - prev) <= pp->rel * rho) || m >= pp->m_max) {
            ctl->status = PHIX_OK;
            ctl->done = 1;
          }
          double al = 1.0 / rho;
          ctl->alpha = al;
          float ah = (float)al;
          ctl->alpha_hi = ah;
          ctl->alpha_lo = (float)(al - (double)ah);
        }
        ctl->m = m + 1;
        ctl->count = 0;
        // no fence: the next launch, the loop condition and the host's copy all
        // follow the kernel's completion
        if (ctl->done) stop_loop(a);
      }
    }
  }
  return;
  }  // for (;;)
}

// ---------------------------------------------------------------------------
// init: y0 = v / sigma, p_k = d_k[0] y0, norms, test at m = 0, ctl->m = 1
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(THREADS)
    k_init(const double* __restrict__ v, typename Tr<P>::T* __restrict__ y0, IterDev a, size_t n) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  using Acc = typename Tr<P>::AccN;
  const PassParams* pp = pp_of(a.ptab);
  const int M = pp->M, K = pp->K;
  C dk[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    dk[k] = (k < K) ? coef<C>(dk_d_of(a.ptab, M)[k * M], dk_f_of(a.ptab, M)[k * M]) : C{};
  Acc acc[KMAX + 1];
#pragma unroll
  for (int j = 0; j <= KMAX; ++j) acc[j] = acc_zero<Acc>();
  const double is = __ldcg(&a.ctl->inv_sigma);
  const int se = __ldcg(&a.ctl->sigma_e);
  const size_t stride = (size_t)gridDim.x * THREADS;
  auto body = [&](size_t i, double vi) {
    C y;
    if constexpr (P == P_FP64) {
      const double x = vi * is;
      y = x;
      y0[i] = x;
    } else if constexpr (P == P_FP32) {
      y = (float)(vi * is);
      y0[i] = y;
    } else {
      y = df_split_pow2(vi, -se);  // v / sigma, sigma a power of two
      y0[i] = make_float2(y.hi, y.lo);
    }
    acc_sq(acc[0], y);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < K) {
        C p = dk[k] * y;
        st1(static_cast<T*>(a.p[k]) + i, p);
        acc_sq(acc[1 + k], p);
      }
    }
  };
  // the thread's elements in grid-stride order, their loads issued UNR at a time
  size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
  for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
    double x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = __ldg(v + i + u * stride);
#pragma unroll
    for (int u = 0; u < UNR; ++u) body(i + u * stride, x[u]);
  }
  for (; i < n; i += stride) body(i, __ldg(v + i));
  if (block_partials_and_last<Acc, KMAX + 1>(acc, a.partials, &a.ctl->count)) {
    double tot[KMAX + 1];
    reduce_partials<Acc, KMAX + 1>(a.partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double dkd[KMAX];
      for (int k = 0; k < K; ++k) dkd[k] = dk_d_of(a.ptab, M)[k * M];
      if (!a.ctl->done) leja_test(a.ctl, 0, K, pp->m_min, pp->m_max, pp->tol, dkd, tot);
      a.ctl->m = 1;
      a.ctl->count = 0;
      __threadfence();
    }
  }
}

// sigma = 2^round(log2(rms(v))); ENAN on a non-finite input
__global__ void __launch_bounds__(THREADS)
    k_scale(const double* __restrict__ v, size_t n, LejaCtl* ctl, double* partials) {
  double acc[1] = {0.0};
  const size_t stride = (size_t)gridDim.x * THREADS;
  size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
  for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
    double x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = __ldg(v + i + u * stride);
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[0] = fma(x[u], x[u], acc[0]);
  }
  for (; i < n; i += stride) {
    const double x = __ldg(v + i);
    acc[0] = fma(x, x, acc[0]);
  }
  if (block_partials_and_last<double, 1>(acc, partials, &ctl->count)) {
    double tot[1];
    reduce_partials<double, 1>(partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double s = tot[0];
      double sig = 1.0;
      if (!isfinite(s)) {
        ctl->status = PHIX_ENAN;
        ctl->done = 1;
      } else if (s > 0.0) {
        double rms = sqrt(s / (double)n);
        int e = (int)rint(log2(rms));
        sig = ldexp(1.0, e);
      }
      ctl->sigma = sig;
      ctl->sigma_e = (int)ilogb(sig);
      ctl->inv_sigma = 1.0 / sig;
      ctl->count = 0;
      __threadfence();
    }
  }
}

template <int P>
__global__ void __launch_bounds__(THREADS) k_finalize(size_t n, int K, PtrPack pk, const LejaCtl* ctl, FusedOut fo) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  const double s = __ldcg(&ctl->sigma);
  const int se = __ldcg(&ctl->sigma_e);
  // a two-iteration chain that stopped at an even m >= 2: p_m = p_{m-1} + d_k[m] y_m
  const int it = __ldcg(&ctl->iters);
  const bool def = fo.ptab != nullptr && it >= 2 && !(it & 1);
  const T* yd = def ? static_cast<const T*>(((it >> 1) & 1) ? fo.y[1] : fo.y[0]) : nullptr;
  const unsigned char* tab = static_cast<const unsigned char*>(fo.ptab);
  const size_t stride = (size_t)gridDim.x * THREADS;
  for (int k = 0; k < K; ++k) {
    const T* p = static_cast<const T*>(pk.p[k]);
    double* o = pk.o[k];
    C dk{};
    if (def) {
      const int M = pp_of(tab)->M;
      dk = coef<C>(dk_d_of(tab, M)[k * M + it], dk_f_of(tab, M)[k * M + it]);
    }
    auto body = [&](size_t i, C x, C yv) {
      if (def) x = mad(dk, yv, x);
      if constexpr (P == P_FP64 || P == P_FP32) {
        o[i] = s * (double)x;
      } else {
        o[i] = df_to_double_pow2(x, se);  // sigma (hi + lo), sigma a power of two
      }
    };
    size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
    for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
      C x[UNR], yv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        x[u] = cv(p[i + u * stride]);
        yv[u] = def ? cv(yd[i + u * stride]) : C{};
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) body(i + u * stride, x[u], yv[u]);
    }
    for (; i < n; i += stride) body(i, cv(p[i]), def ? cv(yd[i]) : C{});
  }
}

template <int P>
__global__ void __launch_bounds__(THREADS)
    k_power_start(size_t n, uint64_t seed, typename Tr<P>::T* __restrict__ y0, LejaCtl* ctl, double* partials) {
  using C = typename Tr<P>::C;
  using Acc = typename Tr<P>::AccP;
  Acc acc[1] = {acc_zero<Acc>()};
  const size_t stride = (size_t)gridDim.x * THREADS;
  for (size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x; i < n; i += stride) {
    double x = splitmix_uniform(seed, i);
    C y;
    if constexpr (P == P_FP64) {
      y = x;
      y0[i] = x;
    } else if constexpr (P == P_FP32) {
      y = (float)x;
      y0[i] = y;
    } else {
      y = df_split_pow2(x, 0);
      y0[i] = make_float2(y.hi, y.lo);
    }
    acc_sq(acc[0], y);
  }
  if (block_partials_and_last<Acc, 1>(acc, partials, &ctl->count)) {
    double tot[1];
    reduce_partials<Acc, 1>(partials, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double al = 1.0 / sqrt(tot[0]);
      ctl->alpha = al;
      float ah = (float)al;
      ctl->alpha_hi = ah;
      ctl->alpha_lo = (float)(al - (double)ah);
      ctl->rho = 0.0;
      ctl->m = 1;
      ctl->count = 0;
      __threadfence();
    }
  }
}

// GS: st = [V^2, 2UV]; Burgers: st = [U]; computed in float64 then stored in S.
template <int P>
__global__ void __launch_bounds__(THREADS)
    k_prep_state(int op, size_t plane, const double* __restrict__ state, typename Tr<P>::S* __restrict__ st,
                 double scale) {
  using S = typename Tr<P>::S;
  const size_t stride = (size_t)gridDim.x * THREADS;
  const bool gs = op == PHIX_OP_GRAYSCOTT;
  auto body = [&](size_t i, double U, double Vv) {
    double g[2];
    int ng = 1;
    if (gs) {
      g[0] = scale * (Vv * Vv);
      g[1] = scale * (2.0 * U * Vv);
      ng = 2;
    } else {
      g[0] = scale * U;
    }
    for (int j = 0; j < ng; ++j) {
      S s;
      if constexpr (P == P_FP64) {
        s = g[j];
      } else if constexpr (P == P_DF64) {
        df d = df_split_pow2(g[j], 0);
        s = make_float2(d.hi, d.lo);
      } else {
        s = (float)g[j];
      }
      st[j * plane + i] = s;
    }
  };
  size_t i = (size_t)blockIdx.x * THREADS + threadIdx.y * 32 + threadIdx.x;
  for (; i + (UNR - 1) * stride < plane; i += UNR * stride) {
    double U[UNR], Vv[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      U[u] = __ldg(state + i + u * stride);
      Vv[u] = gs ? __ldg(state + plane + i + u * stride) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) body(i + u * stride, U[u], Vv[u]);
  }
  for (; i < plane; i += stride) body(i, __ldg(state + i), gs ? __ldg(state + plane + i) : 0.0);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static float2 split2(double x) {
  float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

void ptab_fill(void* host, int K, int m_min, int m_max, double tol, double rel, const double* k8,
               double ga, const double* beta, const double* const* dk, int prescaled) {
  const int M = m_max + 1;
  unsigned char* b = static_cast<unsigned char*>(host);
  PassParams* pp = reinterpret_cast<PassParams*>(b);
  std::memset(b, 0, ptab_bytes(M));
  pp->K = K;
  pp->m_min = m_min;
  pp->m_max = m_max;
  pp->M = M;
  pp->tol = tol;
  pp->rel = rel;
  for (int j = 0; j < 8; ++j) {
    pp->kd[j] = k8[j];
    pp->kf[j] = split2(k8[j]);
  }
  pp->gad = ga;
  pp->gaf = split2(ga);
  pp->prescaled = prescaled;
  double* bd = reinterpret_cast<double*>(b + sizeof(PassParams));
  float2* bf = reinterpret_cast<float2*>(b + sizeof(PassParams) + 8 * (size_t)M);
  double* dd = reinterpret_cast<double*>(b + sizeof(PassParams) + 16 * (size_t)M);
  float2* df2 = reinterpret_cast<float2*>(b + sizeof(PassParams) + 16 * (size_t)M + 8 * (size_t)KMAX * M);
  if (beta)
    for (int m = 0; m < M; ++m) {
      bd[m] = beta[m];
      bf[m] = split2(beta[m]);
    }
  float2* qf = reinterpret_cast<float2*>(b + sizeof(PassParams) + 16 * (size_t)M + 16 * (size_t)KMAX * M);
  if (dk)
    for (int k = 0; k < K; ++k)
      for (int m = 0; m < M; ++m) {
        dd[k * M + m] = dk[k][m];
        df2[k * M + m] = split2(dk[k][m]);
        const double r = tol > 0 ? dk[k][m] / tol : 0.0;
        // beyond the float32 range: +inf (the test never passes there)
        qf[k * M + m] = r * r > 3.0e38 ? make_float2(INFINITY, 0.f) : split2(r * r);
      }
}

static IterDev make_dev(const ChainSpec& s, int V) {
  IterDev a{};
  a.y[0] = s.y[0];
  a.y[1] = s.y[1];
  for (int k = 0; k < KMAX; ++k) a.p[k] = s.p[k];
  a.st = s.st;
  a.ctl = s.ctl;
  a.partials = s.partials;
  a.ptab = static_cast<const unsigned char*>(s.ptab);
  a.nx = s.nx;
  a.ny = s.ny;
  a.tiles_x = (s.nx / V + 31) / 32;
  a.ntiles = a.tiles_x * ((s.ny + TILE_Y - 1) / TILE_Y);
  a.use_cond = s.use_cond;
  a.cond = s.cond;
  return a;
}

// the kernel function of a spec
template <int P, int OP, int MODE>
static void* kfn_t(int V) {
  return V == 2 ? (void*)k_iter<P, OP, 2, MODE, 0> : (void*)k_iter<P, OP, 1, MODE, 0>;
}
template <int P, int OP>
static void* kfn_chain_op(int V) {
  return V == 2 ? (void*)k_iter<P, OP, 2, MODE_NEWTON, 1> : (void*)k_iter<P, OP, 1, MODE_NEWTON, 1>;
}
template <int P>
static void* kfn_chain_p(int op, int V) {
  switch (op) {
    case PHIX_OP_ADVDIFF:
      return kfn_chain_op<P, PHIX_OP_ADVDIFF>(V);
    case PHIX_OP_GRAYSCOTT:
      return kfn_chain_op<P, PHIX_OP_GRAYSCOTT>(V);
    case PHIX_OP_BURGERS:
      return kfn_chain_op<P, PHIX_OP_BURGERS>(V);
  }
  return nullptr;
}
// the persistent (whole-chain) Newton kernel of a spec
static void* kfn_chain(const ChainSpec& s, int V) {
  switch (s.prec) {
    case P_FP64:
      return kfn_chain_p<P_FP64>(s.op, V);
    case P_DF64:
      return kfn_chain_p<P_DF64>(s.op, V);
    case P_FP32JV:
      return kfn_chain_p<P_FP32JV>(s.op, V);
    case P_FP32:
      return kfn_chain_p<P_FP32>(s.op, V);
  }
  return nullptr;
}
template <int P, int MODE>
static void* kfn_op(int op, int V) {
  switch (op) {
    case PHIX_OP_ADVDIFF:
      return kfn_t<P, PHIX_OP_ADVDIFF, MODE>(V);
    case PHIX_OP_GRAYSCOTT:
      return kfn_t<P, PHIX_OP_GRAYSCOTT, MODE>(V);
    case PHIX_OP_BURGERS:
      return kfn_t<P, PHIX_OP_BURGERS, MODE>(V);
  }
  return nullptr;
}
template <int P>
static void* kfn_mode(int op, int mode, int V) {
  return mode == MODE_NEWTON ? kfn_op<P, MODE_NEWTON>(op, V) : kfn_op<P, MODE_POWER>(op, V);
}
static void* kfn(const ChainSpec& s, int V) {
  switch (s.prec) {
    case P_FP64:
      return kfn_mode<P_FP64>(s.op, s.mode, V);
    case P_DF64:
      return kfn_mode<P_DF64>(s.op, s.mode, V);
    case P_FP32JV:
      return kfn_mode<P_FP32JV>(s.op, s.mode, V);
    case P_FP32:
      return kfn_mode<P_FP32>(s.op, s.mode, V);
  }
  return nullptr;
}

cudaError_t iter_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage,
                             size_t arg_bytes) {
  if (s.tma) return tma_node_params(s, np, arg_storage, arg_bytes);
  if (s.fused2) return fused2_node_params(s, np, arg_storage, arg_bytes);
  if (arg_bytes < sizeof(IterDev)) return cudaErrorInvalidValue;
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  IterDev a = make_dev(s, V);
  std::memcpy(arg_storage, &a, sizeof a);
  void* fn = kfn(s, V);
  if (!fn) return cudaErrorInvalidValue;
  std::memset(np, 0, sizeof *np);
  np->func = fn;
  np->gridDim = dim3(s.grid < a.ntiles ? s.grid : a.ntiles);
  np->blockDim = dim3(32, TILE_Y);
  np->sharedMemBytes = 0;
  static thread_local void* argp[1];
  argp[0] = arg_storage;
  np->kernelParams = argp;
  np->extra = nullptr;
  return cudaSuccess;
}

cudaError_t launch_iter(const ChainSpec& s, cudaStream_t st) {
  if (s.fused2 || s.tma) {
    alignas(64) unsigned char argbuf[2048];
    cudaKernelNodeParams np;
    const cudaError_t e = iter_node_params(s, &np, argbuf, sizeof argbuf);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(np.func, np.gridDim, np.blockDim, np.kernelParams, np.sharedMemBytes, st);
  }
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  IterDev a = make_dev(s, V);
  void* fn = kfn(s, V);
  if (!fn) return cudaErrorInvalidValue;
  void* args[1] = {&a};
  dim3 grid(s.grid < a.ntiles ? s.grid : a.ntiles);
  return cudaLaunchKernel(fn, grid, dim3(32, TILE_Y), args, 0, st);
}

int chain_grid(const ChainSpec& s, int nsm) {
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn_chain(s, V), THREADS, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  // every resident block (the same count on every SM; an even tile split over
  // fewer blocks leaves some SMs with one block fewer, measured no faster)
  const int ntiles = make_dev(s, V).ntiles;
  const int g = nb * nsm;
  return g < ntiles ? g : ntiles;
}

cudaError_t launch_chain(const ChainSpec& s, cudaStream_t st) {
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  IterDev a = make_dev(s, V);
  void* fn = kfn_chain(s, V);
  if (!fn || s.grid < 1) return cudaErrorInvalidValue;
  void* args[1] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3(s.grid), dim3(32, TILE_Y), args, 0, st);
}

int iter_tiles(const ChainSpec& s) {
  if (s.fused2) return fused2_tiles(s);
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  return make_dev(s, V).ntiles;
}

int iter_blocks_per_sm(const ChainSpec& s) {
  const int V = (s.nx % 2 == 0) ? 2 : 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn(s, V), THREADS, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 4;
  }
  return nb < 1 ? 1 : nb;
}

template <int P>
static cudaError_t launch_init_t(const InitLaunch& L, cudaStream_t s) {
  ChainSpec cs{};
  cs.nx = L.nx;
  cs.ny = L.ny;
  for (int k = 0; k < KMAX; ++k) cs.p[k] = L.p[k];
  cs.ctl = L.ctl;
  cs.partials = L.partials;
  cs.ptab = L.ptab;
  IterDev a = make_dev(cs, 1);
  size_t n = (size_t)L.ncomp * L.nx * L.ny;
  k_init<P><<<L.grid, dim3(32, TILE_Y), 0, s>>>(L.v, static_cast<typename Tr<P>::T*>(L.y0), a, n);
  return cudaGetLastError();
}

cudaError_t launch_init(const InitLaunch& L, cudaStream_t s) {
  switch (L.prec) {
    case P_FP64:
      return launch_init_t<P_FP64>(L, s);
    case P_DF64:
      return launch_init_t<P_DF64>(L, s);
    case P_FP32JV:
      return launch_init_t<P_FP32JV>(L, s);
    case P_FP32:
      return launch_init_t<P_FP32>(L, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_scale(const double* v, size_t n, LejaCtl* ctl, double* partials, int grid,
                         cudaStream_t s) {
  k_scale<<<grid, dim3(32, TILE_Y), 0, s>>>(v, n, ctl, partials);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int prec, size_t n, int K, void* const* p, double* const* out,
                            const LejaCtl* ctl, int grid, cudaStream_t s, const FusedOut* fo) {
  PtrPack pk{};
  for (int k = 0; k < K && k < KMAX; ++k) {
    pk.p[k] = p[k];
    pk.o[k] = out[k];
  }
  const FusedOut f = fo ? *fo : FusedOut{};
  switch (prec) {
    case P_FP64:
      k_finalize<P_FP64><<<grid, dim3(32, TILE_Y), 0, s>>>(n, K, pk, ctl, f);
      break;
    case P_DF64:
    case P_FP32JV:
      k_finalize<P_DF64><<<grid, dim3(32, TILE_Y), 0, s>>>(n, K, pk, ctl, f);
      break;
    case P_FP32:
      k_finalize<P_FP32><<<grid, dim3(32, TILE_Y), 0, s>>>(n, K, pk, ctl, f);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_power_start(int prec, size_t n, uint64_t seed, void* y0, LejaCtl* ctl,
                               double* partials, int grid, cudaStream_t s) {
  dim3 b(32, TILE_Y);
  switch (prec) {
    case P_FP64:
      k_power_start<P_FP64><<<grid, b, 0, s>>>(n, seed, static_cast<double*>(y0), ctl, partials);
      break;
    case P_DF64:
      k_power_start<P_DF64><<<grid, b, 0, s>>>(n, seed, static_cast<float2*>(y0), ctl, partials);
      break;
    case P_FP32JV:
      k_power_start<P_FP32JV><<<grid, b, 0, s>>>(n, seed, static_cast<float2*>(y0), ctl, partials);
      break;
    case P_FP32:
      k_power_start<P_FP32><<<grid, b, 0, s>>>(n, seed, static_cast<float*>(y0), ctl, partials);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prep_state(int prec, int op, int nx, int ny, const double* state, void* st,
                              int grid, cudaStream_t s, double scale) {
  size_t plane = (size_t)nx * ny;
  dim3 b(32, TILE_Y);
  switch (prec) {
    case P_FP64:
      k_prep_state<P_FP64><<<grid, b, 0, s>>>(op, plane, state, static_cast<double*>(st), scale);
      break;
    case P_DF64:
      k_prep_state<P_DF64><<<grid, b, 0, s>>>(op, plane, state, static_cast<float2*>(st), scale);
      break;
    case P_FP32JV:
      k_prep_state<P_FP32JV><<<grid, b, 0, s>>>(op, plane, state, static_cast<float*>(st), scale);
      break;
    case P_FP32:
      k_prep_state<P_FP32><<<grid, b, 0, s>>>(op, plane, state, static_cast<float*>(st), scale);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace phix
