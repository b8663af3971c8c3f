// Newton-Leja iteration (Sec. 2.2) with the operands staged by the Tensor
// Memory Accelerator.
//
// Persistent CTAs of 128 threads, four per SM, walk tiles of 128 x 2 points.
// For every tile one thread issues 3-D tensor copies of
//   y_{m-1} with a one-row / HX-column halo (both species in one box),
//   the state planes (with a halo where the Jacobian needs neighbours),
//   each accumulator p_k,
// into one of 2-4 shared-memory stages, completing on that stage's mbarrier;
// the copies of the next tiles are in flight while the CTA computes the
// current one, and they hold no registers.  Four independent CTAs per SM keep
// copies and arithmetic overlapped (one CTA of 512 threads on 128 x 8 tiles
// ran 40 us per iteration on the 1024^2 Gray-Scott pass, four of 128 on
// 128 x 2 tiles 28 us; the y halo then costs two extra rows per two, read
// from L2).  Halo cells that wrap around the
// periodic domain lie outside the tensor (the copy fills them with zeros)
// and are patched with plain loads on the tiles that touch the domain edge.
// The arithmetic per point is the single-step kernel's: same stencil, same
// folded shift, same update order; y_m and p_k are stored with plain
// coalesced stores.  The stop test runs in the last CTA to finish, as there.
//
// Every mbarrier wait has a time limit (1 s on %globaltimer); a CTA that
// times out marks the chain PHIX_ETIMEOUT, waits (again bounded) for its own
// copies in flight and leaves.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "iter_common.cuh"

namespace phix {

namespace {

constexpr int TW = 128, TR = 2;  // interior tile
constexpr int TT = 128;          // threads: 64 column pairs x 2 rows
constexpr int CTAS_PER_SM = 4;
constexpr int STAGES_MAX = 4;
constexpr unsigned SMEM_BUDGET = 58u * 1024u;  // per CTA: two stages of the largest layout (K = 4)

struct TmaDev {
  CUtensorMap my[2];     // y ping-pong, box (TW + 2 HX) x (TR + 2) x NC
  CUtensorMap mp[KMAX];  // accumulators, box TW x TR x NC
  CUtensorMap ms;        // state planes: Gray-Scott TW x TR x 2, Burgers (TW + 2 HXS) x (TR + 2) x 1
  void* y[2];
  void* p[KMAX];
  const void* st;
  LejaCtl* ctl;
  double* partials;
  const unsigned char* ptab;
  int nx, ny, tiles_x, ntiles, stages, K;
  unsigned off_s, off_p, p_box, stage_bytes, tx_bytes;  // bytes within a stage; bytes delivered per stage
  int use_cond;
  cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for phase `parity` of `bar`, at most ~1 s
__device__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ int wrap(int v, int n) {
  if (v >= 0 && v < n) return v;
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// Deterministic reduction of NV accumulators over a block of TT threads into
// partials[blockIdx.x * (KMAX + 1) + j]; true in the block that arrived last.
template <typename A, int NV>
__device__ bool tma_partials_and_last(A (&acc)[NV], double* partials, unsigned int* count, double (*sw)[KMAX + 1]) {
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // float and double-float accumulators: double-float partials (float2 in the
  // double slots), no float64 instruction; float64 accumulators: float64
  constexpr bool DFP = !std::is_same<A, double>::value;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    A v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = acc_add(v, shfl_down(v, o));
    if (lane == 0) {
      if constexpr (DFP) {
        const df d = acc_to_df(v);
        reinterpret_cast<float2*>(&sw[warp][j])[0] = make_float2(d.hi, d.lo);
      } else {
        sw[warp][j] = v;
      }
    }
  }
  __syncthreads();
  if (tid < NV) {
    if constexpr (DFP) {
      df s = df_make(0.f, 0.f);
      for (int w = 0; w < TT / 32; ++w) s = df_add(s, cv(reinterpret_cast<const float2*>(&sw[w][tid])[0]));
      reinterpret_cast<float2*>(partials + (size_t)blockIdx.x * (KMAX + 1) + tid)[0] = make_float2(s.hi, s.lo);
    } else {
      double s = 0.0;
      for (int w = 0; w < TT / 32; ++w) s += sw[w][tid];
      partials[(size_t)blockIdx.x * (KMAX + 1) + tid] = s;
    }
    __threadfence();  // the writers' partials visible before the arrival count
  }
  __syncthreads();
  if (tid == 0) last = (atomicAdd(count, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

// Last block, double-float partials: totals as double-float pairs in thread 0
// (strided per thread, then float32-lane shuffles; no float64 instruction).
template <int NV>
__device__ void tma_reduce_df(const double* partials, df (&tot)[NV], int nv, double (*sw)[KMAX + 1]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TT / 32;
  df s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) s[j] = df_make(0.f, 0.f);
  const float2* pf = reinterpret_cast<const float2*>(partials);
  for (int b = tid; b < (int)gridDim.x; b += TT) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nv) s[j] = df_add(s[j], cv(__ldcg(pf + (size_t)b * (KMAX + 1) + j)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
  __syncthreads();  // sw is reused
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) reinterpret_cast<float2*>(&sw[warp][j])[0] = make_float2(s[j].hi, s[j].lo);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = df_make(0.f, 0.f);
  if (tid == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      df t = df_make(0.f, 0.f);
      for (int w = 0; w < NW; ++w) t = df_add(t, cv(reinterpret_cast<const float2*>(&sw[w][j])[0]));
      tot[j] = t;
    }
}

template <int NV>
__device__ void tma_reduce(const double* partials, double (&tot)[NV], double (*sw)[KMAX + 1]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) s[j] = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += TT) {
#pragma unroll
    for (int j = 0; j < NV; ++j) s[j] += __ldcg(partials + (size_t)b * (KMAX + 1) + j);
  }
  __syncthreads();  // sw is reused
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double v = s[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sw[warp][j] = v;
  }
  __syncthreads();
  // the totals in thread 0 only (float64 instructions hold the pipe ~64 cycles per warp)
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = 0.0;
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = 0.0;
      for (int w = 0; w < TT / 32; ++w) t += sw[w][j];
      tot[j] = t;
    }
  }
}

template <int P, int OP>
__global__ void __launch_bounds__(TT, CTAS_PER_SM) k_iter_tma(const __grid_constant__ TmaDev a) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  using CJ = typename Tr<P>::CJ;
  using S = typename Tr<P>::S;
  using Acc = typename Tr<P>::AccN;
  constexpr int NC = (OP == PHIX_OP_GRAYSCOTT) ? 2 : 1;
  constexpr int HX = 16 / (int)sizeof(T);   // y box starts HX columns left of the tile (16-byte x)
  constexpr int BW = TW + 2 * HX;           // y box width
  constexpr int HXS = 16 / (int)sizeof(S);  // the same for a state box with a halo
  constexpr int BWS = TW + 2 * HXS;
  constexpr bool FOLD = std::is_same<C, CJ>::value;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[STAGES_MAX];
  __shared__ double sw[TT / 32][KMAX + 1];
  __shared__ int s_abort;

  LejaCtl* ctl = a.ctl;
  // the stop flag, the iteration index and the table length: independent
  // loads, issued together (the flag is tested after them)
  const int done0 = __ldcg(&ctl->done);
  const int m = __ldcg(&ctl->m);
  const PassParams* pp = pp_of(a.ptab);
  const int M = pp->M;
  if (done0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.use_cond) cudaGraphSetConditional(a.cond, 0);
    return;
  }
  const int K = a.K;
  const int tid = threadIdx.x;

  CJ kk[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) kk[j] = coef<CJ>(pp->kd[j], pp->kf[j]);
  const CJ ga = coef<CJ>(pp->gad, pp->gaf);
  const bool prescaled = pp->prescaled != 0;
  const C beta = coef<C>(beta_d_of(a.ptab, M)[m], beta_f_of(a.ptab, M)[m]);
  C dk[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
    dk[k] = (k < K) ? coef<C>(dk_d_of(a.ptab, M)[k * M + m], dk_f_of(a.ptab, M)[k * M + m]) : C{};
  if constexpr (FOLD) {
    kk[Centre<OP>::a] = kk[Centre<OP>::a] + from_cj(beta, CJ());
    if constexpr (Centre<OP>::b >= 0) kk[Centre<OP>::b] = kk[Centre<OP>::b] + from_cj(beta, CJ());
  }

  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const int pin = (m - 1) & 1;
  // selects, not a runtime index into the argument block (which would copy
  // the block to local memory)
  const T* __restrict__ yin = static_cast<const T*>(pin ? a.y[1] : a.y[0]);
  T* __restrict__ yout = static_cast<T*>(pin ? a.y[0] : a.y[1]);
  const S* __restrict__ stg = static_cast<const S*>(a.st);
  const int nst = a.stages;
  const int nt = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles of this CTA

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();

  // tiles run down the columns first: with the grid a multiple of the tile
  // columns, row-major order would hand every tile at the periodic x edge
  // (halo patches) to the same few CTAs
  const int tiles_y = a.ntiles / a.tiles_x;
  auto tile_xy = [&](int j, int& x0, int& y0) {
    const int t = (int)blockIdx.x + j * (int)gridDim.x;
    y0 = (t % tiles_y) * TR;
    x0 = (t / tiles_y) * TW;
  };
  auto issue = [&](int j) {  // one thread
    const int s = j % nst;
    unsigned char* base = smem + (size_t)s * a.stage_bytes;
    int x0, y0;
    tile_xy(j, x0, y0);
    // threads read (and on edge tiles wrote) this stage through the generic
    // proxy; order that before the copies of the async proxy overwrite it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&full[s], a.tx_bytes);
    tma_load3(base, &a.my[pin], x0 - HX, y0 - 1, 0, &full[s]);
    if constexpr (OP == PHIX_OP_GRAYSCOTT) tma_load3(base + a.off_s, &a.ms, x0, y0, 0, &full[s]);
    if constexpr (OP == PHIX_OP_BURGERS) tma_load3(base + a.off_s, &a.ms, x0 - HXS, y0 - 1, 0, &full[s]);
    for (int k = 0; k < K; ++k) tma_load3(base + a.off_p + (size_t)k * a.p_box, &a.mp[k], x0, y0, 0, &full[s]);
  };
  if (tid == 0)
    for (int j = 0; j < nst && j < nt; ++j) issue(j);

  Acc acc[KMAX + 1];
#pragma unroll
  for (int j = 0; j <= KMAX; ++j) acc[j] = acc_zero<Acc>();
  const int r = tid >> 6;          // tile row of this thread
  const int c2 = (tid & 63) * 2;   // first of its two columns

  int issued = nst < nt ? nst : nt;
  int j = 0;
  for (; j < nt; ++j) {
    const int s = j % nst;
    int x0, y0;
    tile_xy(j, x0, y0);
    if (!mbar_wait(&full[s], (unsigned)(j / nst) & 1u)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    unsigned char* base = smem + (size_t)s * a.stage_bytes;
    T* ys = reinterpret_cast<T*>(base);                  // [NC][TR + 2][BW]
    S* ss = reinterpret_cast<S*>(base + a.off_s);        // GS [2][TR][TW]; Burgers [TR + 2][BWS]
    // accumulator k: [NC][TR][TW] at base + off_p + k p_box
    const int wv = min(TW, nx - x0), rv = min(TR, ny - y0);
    if (x0 == 0 || x0 + wv >= nx || y0 == 0 || y0 + rv >= ny) {
      // halo cells across the periodic boundary: rows 0 and rv + 1 over the
      // valid columns, columns HX - 1 and HX + wv over the valid rows
      const int nrow = 2 * wv, ncol = 2 * rv;
      for (int i = tid; i < nrow + ncol; i += TT) {
        int lr, lc, gy, gx;
        if (i < nrow) {
          const int side = i / wv, c = i - side * wv;
          lr = side ? rv + 1 : 0;
          lc = HX + c;
          gy = wrap(side ? y0 + rv : y0 - 1, ny);
          gx = x0 + c;
        } else {
          const int i2 = i - nrow, side = i2 / rv, rr = i2 - side * rv;
          lr = 1 + rr;
          lc = side ? HX + wv : HX - 1;
          gy = y0 + rr;
          gx = wrap(side ? x0 + wv : x0 - 1, nx);
        }
        const size_t g = (size_t)gy * nx + gx;
#pragma unroll
        for (int q = 0; q < NC; ++q) ys[(q * (TR + 2) + lr) * BW + lc] = yin[q * plane + g];
        if constexpr (OP == PHIX_OP_BURGERS) ss[lr * BWS + (lc - HX + HXS)] = stg[g];
      }
      __syncthreads();
    }

    if (r < rv && c2 < wv) {  // nx is even: both columns are inside
      const int gy = y0 + r, gx = x0 + c2;
      const size_t g = (size_t)gy * nx + gx;
      C pv[NC][KMAX][2];
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
          if (k < K) {
            const T* pk = reinterpret_cast<const T*>(base + a.off_p + (size_t)k * a.p_box) +
                          ((size_t)q * TR + r) * TW + c2;
            ldw2(pk, pv[q][k][0], pv[q][k][1]);
          }
      // centre, north and south pairs as 16-byte shared loads (HX + c2 is a
      // 16-byte column); east and west from the neighbours
      C cc[NC][2], ee[NC][2], ww[NC][2], nn[NC][2], so[NC][2];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const T* row = ys + (q * (TR + 2) + r + 1) * BW + HX + c2;
        ldw2(row, cc[q][0], cc[q][1]);
        ldw2(row + BW, nn[q][0], nn[q][1]);
        ldw2(row - BW, so[q][0], so[q][1]);
        ww[q][0] = cv(row[-1]);
        ww[q][1] = cc[q][0];
        ee[q][0] = cc[q][1];
        ee[q][1] = cv(row[2]);
      }
      using SC = decltype(cv(S{}));
      SC g1v[2], g2v[2];
      if constexpr (OP == PHIX_OP_GRAYSCOTT) {
        ldw2(ss + r * TW + c2, g1v[0], g1v[1]);
        ldw2(ss + (TR + r) * TW + c2, g2v[0], g2v[1]);
      }
      C out[NC][2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        CJ J[NC];
        if constexpr (OP == PHIX_OP_ADVDIFF) {
          J[0] = stencil_advdiff<CJ>(kk, to_cj(ee[0][v], CJ()), to_cj(ww[0][v], CJ()), to_cj(nn[0][v], CJ()),
                                     to_cj(so[0][v], CJ()), to_cj(cc[0][v], CJ()));
        } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
          CJ g1 = to_cj(g1v[v], CJ());
          CJ g2 = to_cj(g2v[v], CJ());
          if (!prescaled) {
            g1 = ga * g1;
            g2 = ga * g2;
          }
          stencil_gs_a<CJ>(kk, to_cj(ee[0][v], CJ()), to_cj(ww[0][v], CJ()), to_cj(nn[0][v], CJ()),
                           to_cj(so[0][v], CJ()), to_cj(cc[0][v], CJ()), to_cj(ee[NC - 1][v], CJ()),
                           to_cj(ww[NC - 1][v], CJ()), to_cj(nn[NC - 1][v], CJ()), to_cj(so[NC - 1][v], CJ()),
                           to_cj(cc[NC - 1][v], CJ()), g1, g2, J[0], J[NC - 1]);
        } else {
          const S* srow = ss + (r + 1) * BWS + HXS + c2 + v;
          CJ Uc = to_cj(cv(srow[0]), CJ());
          CJ Ue = to_cj(cv(srow[1]), CJ());
          CJ Uw = to_cj(cv(srow[-1]), CJ());
          CJ Un = to_cj(cv(srow[BWS]), CJ());
          CJ Us = to_cj(cv(srow[-BWS]), CJ());
          J[0] = stencil_burgers<CJ>(kk, ga, to_cj(ee[0][v], CJ()), to_cj(ww[0][v], CJ()), to_cj(nn[0][v], CJ()),
                                     to_cj(so[0][v], CJ()), to_cj(cc[0][v], CJ()), Ue, Uw, Un, Us, Uc);
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          if constexpr (FOLD)
            out[q][v] = from_cj(J[q], C());
          else
            out[q][v] = from_cj(J[q], C()) + beta * cc[q][v];
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        st2(yout + q * plane + g, out[q][0], out[q][1]);
        acc_sq(acc[0], out[q][0]);
        acc_sq(acc[0], out[q][1]);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
          if (k < K) {
            const C p0 = mad(dk[k], out[q][0], pv[q][k][0]);
            const C p1 = mad(dk[k], out[q][1], pv[q][k][1]);
            st2(static_cast<T*>(a.p[k]) + q * plane + g, p0, p1);
            acc_sq(acc[1 + k], p0);
            acc_sq(acc[1 + k], p1);
          }
        }
      }
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0 && issued < nt) {
      issue(issued);
      ++issued;
    }
  }

  if (s_abort) {
    // leave no copy in flight into shared memory: wait (bounded) for the
    // stages still expected, then mark the chain
    if (tid == 0) {
      for (int jj = j; jj < issued; ++jj) (void)mbar_wait(&full[jj % nst], (unsigned)(jj / nst) & 1u);
      ctl->status = PHIX_ETIMEOUT;
      ctl->iters = m;
      ctl->done = 1;
      __threadfence();
      if (a.use_cond) cudaGraphSetConditional(a.cond, 0);
    }
    return;
  }

  if (tma_partials_and_last<Acc, KMAX + 1>(acc, a.partials, &ctl->count, sw)) {
    if constexpr (!std::is_same<Acc, double>::value) {
      // double-float totals and stop test, (d_k[m]/tol)^2 read before the partials
      float2 qk[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        qk[k] = (tid == 0 && k < K) ? q_f_of(a.ptab, M)[k * M + m] : make_float2(0.f, 0.f);
      df tot[KMAX + 1];
      tma_reduce_df<KMAX + 1>(a.partials, tot, K + 1, sw);
      if (tid == 0) {
        leja_test_df(ctl, m, K, pp->m_min, pp->m_max, qk, tot);
        ctl->m = m + 1;
        ctl->count = 0;
        if (ctl->done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
      }
      return;
    }
    // the stop test's coefficients, read before the partials
    double dkd[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) dkd[k] = (tid == 0 && k < K) ? dk_d_of(a.ptab, M)[k * M + m] : 0.0;
    double tot[KMAX + 1];
    tma_reduce<KMAX + 1>(a.partials, tot, sw);
    if (tid == 0) {
      leja_test(ctl, m, K, pp->m_min, pp->m_max, pp->tol, dkd, tot);
      ctl->m = m + 1;
      ctl->count = 0;
      // no fence: the next launch, the loop condition and the host's copy all
      // follow the kernel's completion
      if (ctl->done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
    }
  }
}

template <int P>
void* tma_kernel_p(int op) {
  switch (op) {
    case PHIX_OP_ADVDIFF:
      return (void*)k_iter_tma<P, PHIX_OP_ADVDIFF>;
    case PHIX_OP_GRAYSCOTT:
      return (void*)k_iter_tma<P, PHIX_OP_GRAYSCOTT>;
    case PHIX_OP_BURGERS:
      return (void*)k_iter_tma<P, PHIX_OP_BURGERS>;
  }
  return nullptr;
}
void* tma_kernel(int prec, int op) {
  switch (prec) {
    case P_FP64:
      return tma_kernel_p<P_FP64>(op);
    case P_DF64:
      return tma_kernel_p<P_DF64>(op);
    case P_FP32JV:
      return tma_kernel_p<P_FP32JV>(op);
    case P_FP32:
      return tma_kernel_p<P_FP32>(op);
  }
  return nullptr;
}

// element sizes of the iterate/accumulator storage and of the state
void tma_sizes(int prec, int* et, int* es) {
  *et = prec == P_FP32 ? 4 : 8;
  *es = (prec == P_FP64 || prec == P_DF64) ? 8 : 4;
}

unsigned round128(unsigned b) { return (b + 127u) & ~127u; }

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// 3-D map of planes [nz][ny][nx] of `esize`-byte elements with box bx x by x bz
bool encode3(CUtensorMap* m, const void* base, int esize, int nx, int ny, int nz, int bx, int by, int bz) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Stage layout of a spec: y box | state box | K accumulator boxes
struct Layout {
  unsigned off_s, off_p, p_box, stage, tx;
  int stages;
};
Layout tma_layout(const ChainSpec& s) {
  int et, es;
  tma_sizes(s.prec, &et, &es);
  const int nc = s.op == PHIX_OP_GRAYSCOTT ? 2 : 1;
  const unsigned ybox = (unsigned)(nc * (TR + 2) * (TW + 2 * (16 / et)) * et);
  unsigned sbox = 0;
  if (s.op == PHIX_OP_GRAYSCOTT) sbox = (unsigned)(2 * TR * TW * es);
  if (s.op == PHIX_OP_BURGERS) sbox = (unsigned)((TR + 2) * (TW + 2 * (16 / es)) * es);
  const unsigned pbox = (unsigned)(nc * TR * TW * et);
  Layout L;
  L.off_s = round128(ybox);
  L.off_p = L.off_s + round128(sbox);
  L.p_box = round128(pbox);
  L.stage = L.off_p + (unsigned)s.K * L.p_box;
  L.tx = ybox + sbox + (unsigned)s.K * pbox;
  L.stages = (int)std::min<unsigned>(STAGES_MAX, SMEM_BUDGET / L.stage);
  return L;
}

}  // namespace

bool tma_eligible(const ChainSpec& s) {
  if (s.mode != MODE_NEWTON || s.K < 1 || s.K > KMAX) return false;
  int et, es;
  tma_sizes(s.prec, &et, &es);
  const int align = 16 / std::min(et, es);  // row strides and box x coordinates: 16 bytes
  if (s.nx % align != 0 || s.nx < 2) return false;
  if (!encoder()) return false;
  return tma_layout(s).stages >= 2;
}

int tma_grid(const ChainSpec& s, int nsm) {
  const int ntiles = ((s.nx + TW - 1) / TW) * ((s.ny + TR - 1) / TR);
  return std::max(1, std::min(ntiles, CTAS_PER_SM * nsm));
}

cudaError_t tma_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage, size_t arg_bytes) {
  if (arg_bytes < sizeof(TmaDev) || (reinterpret_cast<uintptr_t>(arg_storage) & 63)) return cudaErrorInvalidValue;
  int et, es;
  tma_sizes(s.prec, &et, &es);
  const int nc = s.op == PHIX_OP_GRAYSCOTT ? 2 : 1;
  const Layout L = tma_layout(s);
  TmaDev* a = new (arg_storage) TmaDev();
  const int hx = 16 / et, hxs = 16 / es;
  for (int i = 0; i < 2; ++i)
    if (!encode3(&a->my[i], s.y[i], et, s.nx, s.ny, nc, TW + 2 * hx, TR + 2, nc)) return cudaErrorInvalidValue;
  for (int k = 0; k < s.K; ++k)
    if (!encode3(&a->mp[k], s.p[k], et, s.nx, s.ny, nc, TW, TR, nc)) return cudaErrorInvalidValue;
  if (s.op == PHIX_OP_GRAYSCOTT && !encode3(&a->ms, s.st, es, s.nx, s.ny, 2, TW, TR, 2))
    return cudaErrorInvalidValue;
  if (s.op == PHIX_OP_BURGERS && !encode3(&a->ms, s.st, es, s.nx, s.ny, 1, TW + 2 * hxs, TR + 2, 1))
    return cudaErrorInvalidValue;
  a->y[0] = s.y[0];
  a->y[1] = s.y[1];
  for (int k = 0; k < KMAX; ++k) a->p[k] = s.p[k];
  a->st = s.st;
  a->ctl = s.ctl;
  a->partials = s.partials;
  a->ptab = static_cast<const unsigned char*>(s.ptab);
  a->nx = s.nx;
  a->ny = s.ny;
  a->tiles_x = (s.nx + TW - 1) / TW;
  a->ntiles = a->tiles_x * ((s.ny + TR - 1) / TR);
  a->stages = L.stages;
  a->K = s.K;
  a->off_s = L.off_s;
  a->off_p = L.off_p;
  a->p_box = L.p_box;
  a->stage_bytes = L.stage;
  a->tx_bytes = L.tx;
  a->use_cond = s.use_cond;
  a->cond = s.cond;
  void* fn = tma_kernel(s.prec, s.op);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = (size_t)L.stages * L.stage;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  std::memset(np, 0, sizeof *np);
  np->func = fn;
  np->gridDim = dim3(s.grid);
  np->blockDim = dim3(TT);
  np->sharedMemBytes = (unsigned)smem;
  static thread_local void* argp[1];
  argp[0] = arg_storage;
  np->kernelParams = argp;
  return cudaSuccess;
}

size_t tma_arg_bytes() { return sizeof(TmaDev); }

}  // namespace phix
