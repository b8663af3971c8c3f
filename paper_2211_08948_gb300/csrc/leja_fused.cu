// Two Newton-Leja iterations per launch (Sec. 2.2's recurrence, blocked in
// time).  A launch that starts at iteration m (odd) computes
//
//   y_m     = ((J - c)/gamma - xi_{m-1}) y_{m-1}   on its tile and a one-point ring
//   y_{m+1} = ((J - c)/gamma - xi_m)     y_m       on its tile
//   p_m     = p_{m-1} + d_k[m] y_m,   p_{m+1} = p_m + d_k[m+1] y_{m+1}
//
// from y_{m-1} staged in shared memory with a two-point ring (and the state
// planes), so that y_m never goes to memory.  It stores y_{m+1} and p_m, not
// p_{m+1}: the term d_k[m+1] y_{m+1} is added by the next launch (which reads
// y_{m+1} anyway) or, when the chain stops at m + 1, by the output
// conversion.  Each p_k is thus read and written once per two iterations, and
// a stop at m finds p_m stored.  The norms of both iterations go into two
// halves of the partials; the last block tests m, then m + 1.
//
// Every accumulator update is the same fused multiply-add, in the same
// order, as in the one-iteration kernel, and every y value the same stencil
// expression, so the results are bitwise those of one iteration per launch
// for the same stop iteration (the norms are summed in another order).
//
// Per unknown and per two iterations the launch moves 16 bytes of y (8-byte
// elements), 16 K of accumulators and the state: half of two one-iteration
// launches.  Tiles of 64 x 16 points (the ring adds 16 % to the first
// iteration's stencils); grids whose sides are multiples of the tile.
//
// On GB300 the halved traffic does not turn into time: in double-float the
// two iterations' arithmetic, latency-bound at 16 warps per SM, takes as long
// as the memory traffic it saves (Gray-Scott 2048^2: 417 MB of DRAM traffic
// per two-iteration launch, 35 % of DRAM peak, 56 % issue), so the library
// runs it on request (PHIX_KERNEL_FUSED2) only.
#include <cstring>
#include <type_traits>

#include "iter_common.cuh"

namespace phix {

namespace {

constexpr int FW = 64, FH = 16;          // interior tile: 32 thread columns x 2 points, 8 thread rows x 2
constexpr int SW = FW + 4, SH = FH + 4;  // staged tile: a two-point ring

struct Fused2Dev {
  const void* y[2];  // launch L (first iteration m = 2L + 1) reads y[L & 1], writes y[(L + 1) & 1]
  void* p[KMAX];
  const void* st;
  LejaCtl* ctl;
  double* partials;  // two halves of gridDim.x * (KMAX + 1)
  const unsigned char* ptab;
  int nx, ny, tiles_x, ntiles;
  int use_cond;
  cudaGraphConditionalHandle cond;
};

template <int OP>
__host__ __device__ constexpr int state_planes() {
  return OP == PHIX_OP_GRAYSCOTT ? 2 : OP == PHIX_OP_BURGERS ? 1 : 0;
}
template <int OP>
__host__ __device__ constexpr int species() {
  return OP == PHIX_OP_GRAYSCOTT ? 2 : 1;
}

template <int P, int OP>
constexpr size_t fused2_smem_t() {
  using T = typename Tr<P>::T;
  using S = typename Tr<P>::S;
  return 2 * (size_t)species<OP>() * SH * SW * sizeof(T) + (size_t)state_planes<OP>() * SH * SW * sizeof(S);
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One point of y = ((J - c)/gamma - xi) y_prev from a staged tile (row stride
// SW): the stencil of the one-iteration kernel, the same operand order.
template <int P, int OP>
__device__ __forceinline__ void newton_point(const typename Tr<P>::CJ (&kk)[8], typename Tr<P>::C beta,
                                             typename Tr<P>::CJ ga, bool prescaled,
                                             const typename Tr<P>::T* __restrict__ sy,
                                             const typename Tr<P>::S* __restrict__ ss, int o,
                                             typename Tr<P>::C (&out)[species<OP>()]) {
  using C = typename Tr<P>::C;
  using CJ = typename Tr<P>::CJ;
  constexpr int NC = species<OP>();
  constexpr bool FOLD = std::is_same<C, CJ>::value;
  constexpr int PL = SH * SW;
  C c[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) c[q] = cv(sy[q * PL + o]);
  CJ J[NC];
  if constexpr (OP == PHIX_OP_ADVDIFF) {
    J[0] = stencil_advdiff<CJ>(kk, to_cj(cv(sy[o + 1]), CJ()), to_cj(cv(sy[o - 1]), CJ()),
                               to_cj(cv(sy[o + SW]), CJ()), to_cj(cv(sy[o - SW]), CJ()), to_cj(c[0], CJ()));
  } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
    CJ g1 = to_cj(cv(ss[o]), CJ());
    CJ g2 = to_cj(cv(ss[PL + o]), CJ());
    if (!prescaled) {
      g1 = ga * g1;
      g2 = ga * g2;
    }
    const typename Tr<P>::T* sv = sy + PL;
    stencil_gs_a<CJ>(kk, to_cj(cv(sy[o + 1]), CJ()), to_cj(cv(sy[o - 1]), CJ()), to_cj(cv(sy[o + SW]), CJ()),
                     to_cj(cv(sy[o - SW]), CJ()), to_cj(c[0], CJ()), to_cj(cv(sv[o + 1]), CJ()),
                     to_cj(cv(sv[o - 1]), CJ()), to_cj(cv(sv[o + SW]), CJ()), to_cj(cv(sv[o - SW]), CJ()),
                     to_cj(c[1], CJ()), g1, g2, J[0], J[1]);
  } else {
    const CJ Uc = to_cj(cv(ss[o]), CJ()), Ue = to_cj(cv(ss[o + 1]), CJ()), Uw = to_cj(cv(ss[o - 1]), CJ());
    const CJ Un = to_cj(cv(ss[o + SW]), CJ()), Us = to_cj(cv(ss[o - SW]), CJ());
    J[0] = stencil_burgers<CJ>(kk, ga, to_cj(cv(sy[o + 1]), CJ()), to_cj(cv(sy[o - 1]), CJ()),
                               to_cj(cv(sy[o + SW]), CJ()), to_cj(cv(sy[o - SW]), CJ()), to_cj(c[0], CJ()), Ue,
                               Uw, Un, Us, Uc);
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    if constexpr (FOLD)
      out[q] = from_cj(J[q], C());
    else
      out[q] = from_cj(J[q], C()) + beta * c[q];
  }
}

template <int P, int OP>
__global__ void __launch_bounds__(THREADS, 2) k_iter2(Fused2Dev a) {
  using T = typename Tr<P>::T;
  using T2 = typename Tr<P>::T2;
  using C = typename Tr<P>::C;
  using CJ = typename Tr<P>::CJ;
  using S = typename Tr<P>::S;
  using S2 = typename Tr<P>::S2;
  using Acc = typename Tr<P>::AccN;
  constexpr int NC = species<OP>();
  constexpr int NS = state_planes<OP>();
  constexpr bool FOLD = std::is_same<C, CJ>::value;
  constexpr int PL = SH * SW;
  extern __shared__ __align__(16) unsigned char f2_smem[];
  T* s0 = reinterpret_cast<T*>(f2_smem);            // y_{m-1}, [NC][SH][SW]
  T* s1 = s0 + NC * PL;                             // y_m on the ring and the tile
  S* ss = reinterpret_cast<S*>(s1 + NC * PL);       // state planes, [NS][SH][SW]

  if (__ldcg(&a.ctl->done)) {  // the chain already stopped
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0 && a.use_cond)
      cudaGraphSetConditional(a.cond, 0);
    return;
  }
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int m = __ldcg(&a.ctl->m);
  const PassParams* pp = pp_of(a.ptab);
  const int M = pp->M, K = pp->K;
  const bool two = m + 1 <= pp->m_max;  // the pair's second iteration exists in the table
  const bool deferred = m >= 3;         // the previous launch left d_k[m-1] y_{m-1} to add
  const CJ ga = coef<CJ>(pp->gad, pp->gaf);
  const bool prescaled = pp->prescaled;
  CJ kk0[8], kk1[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) kk0[j] = kk1[j] = coef<CJ>(pp->kd[j], pp->kf[j]);
  const C beta0 = coef<C>(beta_d_of(a.ptab, M)[m], beta_f_of(a.ptab, M)[m]);
  const C beta1 = two ? coef<C>(beta_d_of(a.ptab, M)[m + 1], beta_f_of(a.ptab, M)[m + 1]) : C{};
  C dkp[KMAX], dk0[KMAX], dk1[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const double* dd = dk_d_of(a.ptab, M) + k * M;
    const float2* df2 = dk_f_of(a.ptab, M) + k * M;
    dk0[k] = k < K ? coef<C>(dd[m], df2[m]) : C{};
    dk1[k] = (k < K && two) ? coef<C>(dd[m + 1], df2[m + 1]) : C{};
    dkp[k] = (k < K && deferred) ? coef<C>(dd[m - 1], df2[m - 1]) : C{};
  }
  if constexpr (FOLD) {
    kk0[Centre<OP>::a] = kk0[Centre<OP>::a] + from_cj(beta0, CJ());
    kk1[Centre<OP>::a] = kk1[Centre<OP>::a] + from_cj(beta1, CJ());
    if constexpr (Centre<OP>::b >= 0) {
      kk0[Centre<OP>::b] = kk0[Centre<OP>::b] + from_cj(beta0, CJ());
      kk1[Centre<OP>::b] = kk1[Centre<OP>::b] + from_cj(beta1, CJ());
    }
  }

  const int L = (m - 1) >> 1;
  const T* __restrict__ yin = static_cast<const T*>((L & 1) ? a.y[1] : a.y[0]);
  T* __restrict__ yout = static_cast<T*>(const_cast<void*>((L & 1) ? a.y[0] : a.y[1]));
  const S* __restrict__ st = static_cast<const S*>(a.st);
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;

  Acc acc0[KMAX + 1], acc1[KMAX + 1];  // norms of iterations m and m + 1
#pragma unroll
  for (int j = 0; j <= KMAX; ++j) acc0[j] = acc1[j] = acc_zero<Acc>();

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int x0 = (tile % a.tiles_x) * FW, y0 = (tile / a.tiles_x) * FH;
    __syncthreads();  // the previous tile's shared data fully read
    // stage y_{m-1} and the state with the two-point ring: pairs of elements
    // (x0 - 2 is even, so pairs stay 2-element aligned across the periodic wrap)
    for (int i = tid; i < SH * (SW / 2); i += THREADS) {
      const int r = i / (SW / 2), j2 = 2 * (i % (SW / 2));
      const size_t g = (size_t)wrap(y0 - 2 + r, ny) * nx + wrap(x0 - 2 + j2, nx);
#pragma unroll
      for (int q = 0; q < NC; ++q)
        *reinterpret_cast<T2*>(s0 + q * PL + r * SW + j2) = __ldg(reinterpret_cast<const T2*>(yin + q * plane + g));
#pragma unroll
      for (int q = 0; q < NS; ++q)
        *reinterpret_cast<S2*>(ss + q * PL + r * SW + j2) = __ldg(reinterpret_cast<const S2*>(st + q * plane + g));
    }
    __syncthreads();
    // y_m on the tile and its one-point ring (rows and columns 1 .. 18 / 1 .. 66)
    for (int i = tid; i < (FH + 2) * (FW + 2); i += THREADS) {
      const int o = (1 + i / (FW + 2)) * SW + 1 + i % (FW + 2);
      C y[NC];
      newton_point<P, OP>(kk0, beta0, ga, prescaled, s0, ss, o, y);
#pragma unroll
      for (int q = 0; q < NC; ++q) st1(s1 + q * PL + o, y[q]);
    }
    __syncthreads();
    // the tile: accumulators, y_{m+1}, norms; two rows per thread
#pragma unroll 1
    for (int rp = 0; rp < 2; ++rp) {
      const int ly = threadIdx.y + 8 * rp;
      const int o = (2 + ly) * SW + 2 + 2 * threadIdx.x;
      const size_t g = (size_t)(y0 + ly) * nx + x0 + 2 * threadIdx.x;
      C pv[NC][KMAX][2];
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
          if (k < K) ldw2(static_cast<const T*>(a.p[k]) + q * plane + g, pv[q][k][0], pv[q][k][1]);
      C y1[NC][2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (two) {
          C yy[NC];
          newton_point<P, OP>(kk1, beta1, ga, prescaled, s1, ss, o + v, yy);
#pragma unroll
          for (int q = 0; q < NC; ++q) y1[q][v] = yy[q];
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          const C ym = cv(s1[q * PL + o + v]);
          acc_sq(acc0[0], ym);
          if (two) acc_sq(acc1[0], y1[q][v]);
          const C yp = deferred ? cv(s0[q * PL + o + v]) : C{};
#pragma unroll
          for (int k = 0; k < KMAX; ++k) {
            if (k < K) {
              C p = pv[q][k][v];
              if (deferred) p = mad(dkp[k], yp, p);  // the previous launch's deferred term
              p = mad(dk0[k], ym, p);                 // p_m
              pv[q][k][v] = p;
              acc_sq(acc0[1 + k], p);
              if (two) acc_sq(acc1[1 + k], mad(dk1[k], y1[q][v], p));  // p_{m+1}, not stored
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
          if (k < K) st2(static_cast<T*>(a.p[k]) + q * plane + g, pv[q][k][0], pv[q][k][1]);
        if (two) st2(yout + q * plane + g, y1[q][0], y1[q][1]);
      }
    }
  }

  // norms: iteration m into the first half of the partials, m + 1 into the
  // second; the last block tests m, then m + 1
  block_partials_only<Acc, KMAX + 1>(acc0, a.partials);
  if (block_partials_and_last<Acc, KMAX + 1>(acc1, a.partials + (size_t)gridDim.x * (KMAX + 1), &a.ctl->count)) {
    for (int h = 0; h < (two ? 2 : 1); ++h) {
      const int mm = m + h;
      const double* part = a.partials + (size_t)h * gridDim.x * (KMAX + 1);
      bool done = false;
      if constexpr (PartialsDF<Acc>::value) {
        float2 qk[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
          qk[k] = (tid == 0 && k < K) ? q_f_of(a.ptab, M)[k * M + mm] : make_float2(0.f, 0.f);
        df tot[KMAX + 1];
        reduce_partials_df<Acc, KMAX + 1>(part, tot, K + 1);
        if (tid == 0) leja_test_df(a.ctl, mm, K, pp->m_min, pp->m_max, qk, tot);
      } else {
        double dkd[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) dkd[k] = (tid == 0 && k < K) ? dk_d_of(a.ptab, M)[k * M + mm] : 0.0;
        double tot[KMAX + 1];
        reduce_partials<Acc, KMAX + 1>(part, tot, NoHook{}, K + 1);
        if (tid == 0) leja_test(a.ctl, mm, K, pp->m_min, pp->m_max, pp->tol, dkd, tot);
      }
      __shared__ int s_done;
      if (tid == 0) s_done = a.ctl->done;
      __syncthreads();
      done = s_done != 0;
      __syncthreads();
      if (done) break;
    }
    if (tid == 0) {
      LejaCtl* ctl = a.ctl;
      ctl->m = m + (two ? 2 : 1);
      ctl->count = 0;
      if (ctl->done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
    }
  }
}

template <int P, int OP>
void* fused2_fn() {
  return reinterpret_cast<void*>(k_iter2<P, OP>);
}
template <int P>
void* fused2_fn_op(int op) {
  switch (op) {
    case PHIX_OP_ADVDIFF:
      return fused2_fn<P, PHIX_OP_ADVDIFF>();
    case PHIX_OP_GRAYSCOTT:
      return fused2_fn<P, PHIX_OP_GRAYSCOTT>();
    case PHIX_OP_BURGERS:
      return fused2_fn<P, PHIX_OP_BURGERS>();
  }
  return nullptr;
}
void* fused2_kernel(int prec, int op) {
  switch (prec) {
    case P_FP64:
      return fused2_fn_op<P_FP64>(op);
    case P_DF64:
      return fused2_fn_op<P_DF64>(op);
    case P_FP32JV:
      return fused2_fn_op<P_FP32JV>(op);
    case P_FP32:
      return fused2_fn_op<P_FP32>(op);
  }
  return nullptr;
}
template <int P>
size_t fused2_smem_op(int op) {
  switch (op) {
    case PHIX_OP_ADVDIFF:
      return fused2_smem_t<P, PHIX_OP_ADVDIFF>();
    case PHIX_OP_GRAYSCOTT:
      return fused2_smem_t<P, PHIX_OP_GRAYSCOTT>();
    case PHIX_OP_BURGERS:
      return fused2_smem_t<P, PHIX_OP_BURGERS>();
  }
  return 0;
}
size_t fused2_smem(int prec, int op) {
  switch (prec) {
    case P_FP64:
      return fused2_smem_op<P_FP64>(op);
    case P_DF64:
      return fused2_smem_op<P_DF64>(op);
    case P_FP32JV:
      return fused2_smem_op<P_FP32JV>(op);
    case P_FP32:
      return fused2_smem_op<P_FP32>(op);
  }
  return 0;
}

}  // namespace

bool fused2_eligible(const ChainSpec& s) {
  if (s.mode != MODE_NEWTON || s.K < 1 || s.K > KMAX) return false;
  if (s.op != PHIX_OP_ADVDIFF && s.op != PHIX_OP_GRAYSCOTT && s.op != PHIX_OP_BURGERS) return false;
  return s.nx % FW == 0 && s.ny % FH == 0 && fused2_kernel(s.prec, s.op) != nullptr;
}

int fused2_tiles(const ChainSpec& s) { return (s.nx / FW) * (s.ny / FH); }

int fused2_blocks_per_sm(const ChainSpec& s) {
  void* fn = fused2_kernel(s.prec, s.op);
  const size_t smem = fused2_smem(s.prec, s.op);
  int nb = 0;
  if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, THREADS, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 1;
  }
  return nb < 1 ? 1 : nb;
}

cudaError_t fused2_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage, size_t arg_bytes) {
  if (arg_bytes < sizeof(Fused2Dev)) return cudaErrorInvalidValue;
  void* fn = fused2_kernel(s.prec, s.op);
  if (!fn) return cudaErrorInvalidValue;
  Fused2Dev a{};
  a.y[0] = s.y[0];
  a.y[1] = s.y[1];
  for (int k = 0; k < KMAX; ++k) a.p[k] = s.p[k];
  a.st = s.st;
  a.ctl = s.ctl;
  a.partials = s.partials;
  a.ptab = static_cast<const unsigned char*>(s.ptab);
  a.nx = s.nx;
  a.ny = s.ny;
  a.tiles_x = s.nx / FW;
  a.ntiles = fused2_tiles(s);
  a.use_cond = s.use_cond;
  a.cond = s.cond;
  std::memcpy(arg_storage, &a, sizeof a);
  const size_t smem = fused2_smem(s.prec, s.op);
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  std::memset(np, 0, sizeof *np);
  np->func = fn;
  np->gridDim = dim3(s.grid < a.ntiles ? s.grid : a.ntiles);
  np->blockDim = dim3(32, TILE_Y);
  np->sharedMemBytes = (unsigned)smem;
  static thread_local void* argp[1];
  argp[0] = arg_storage;
  np->kernelParams = argp;
  np->extra = nullptr;
  return cudaSuccess;
}

}  // namespace phix
