// Batched phi-actions: thousands of independent advection-diffusion problems
// of different sizes and stiffness in ONE persistent launch.
//
// Every CTA pops whole problems from an atomic queue (the host orders it
// largest-first) and runs the complete real-Leja computation of Sec. 2.2 for
// each: divided-difference tables on the device (float64), then either one
// vertical Newton pass for all outputs (Sec. 4) or, when the interval needs
// substeps, the ODE-identity substeps per output.  A CTA owns its problem, so
// every reduction and stop test is block-level: there is no grid-wide
// synchronisation and no waiting on other CTAs.  Iteration arithmetic in
// float64, double-float, or float32 stencil with double-float update
// (PHIX_FP32_JV).
#include <cstring>

#include "iter_common.cuh"

namespace phix {

namespace {

constexpr int MAXWARP = 32;  // block sizes 256, 512, 1024 (tuned per batch shape)
constexpr int BM = 501;      // longest divided-difference table (m_max <= 500)

__device__ double phi_dev(int l, double z) {
  if (l == 0) return exp(z);
  if (fabs(z) < l + 1.0) {
    double inv_fact = 1.0;
    for (int j = 2; j <= l; ++j) inv_fact /= j;
    double term = inv_fact, sum = 0.0;
    for (int k = 0; k < 80; ++k) {
      sum += term;
      term *= z / (k + l + 1);
      if (fabs(term) < 1e-18 * fabs(sum)) {
        sum += term;
        break;
      }
    }
    return sum;
  }
  double p = exp(z);
  double inv_fact = 1.0;
  for (int j = 0; j < l; ++j) {
    p = (p - inv_fact) / z;
    inv_fact /= (j + 1);
  }
  return p;
}

__device__ __forceinline__ float2 split_d(double v) {
  float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

struct Shared {
  double dd[3][BM];   // divided differences of the current pass
  float2 ddf[3][BM];  // their double-float forms
  double tmp[BM];
  double beta[BM];    // shifts beta_m = -(c/gamma + xi_{m-1})
  float2 betaf[BM];
  double red[MAXWARP][4];
  float2 redf[MAXWARP][4];
  double tot[4];
  int flag;  // stop decision of the iteration, from thread 0
};

struct Prob {
  int nx, ny;
  double D, ax, ay, h;
  double rho_re, rho_hi, rho_im;
  const double* v;
  double* out[3];
  unsigned long long ws;  // element offset of this problem's workspace
  int status, iters, substeps, pad;
};

struct BArgs {
  Prob* probs;
  const int* order;
  int nprob;
  unsigned int* queue;
  void* ws;
  const double* xi;
  int m_max, m_min;
  double tol, gamma_cap, iota_cap;
  int nout;
  int l[3];
  unsigned int smem_bytes;  // dynamic shared memory: a vertical pass whose basis pair and
                            // accumulators fit runs on shared memory instead of the arena
};

// d = divided differences of xi -> phi_l(a + b xi), i < M (block-wide, float64)
__device__ void dd_block(int l, double a, double b, const double* xi, int M, double* d, float2* df2, double* tmp,
                         int tid) {
  const int nthr = blockDim.x;
  for (int i = tid; i < M; i += nthr) d[i] = phi_dev(l, a + b * xi[i]);
  __syncthreads();
  for (int j = 1; j < M; ++j) {
    for (int i = j + tid; i < M; i += nthr) tmp[i] = (d[i] - d[i - 1]) / (xi[i] - xi[i - j]);
    __syncthreads();
    for (int i = j + tid; i < M; i += nthr) d[i] = tmp[i];
    __syncthreads();
  }
  for (int i = tid; i < M; i += nthr) df2[i] = split_d(d[i]);
  __syncthreads();
}

// Block totals of the first nv accumulators, valid in thread 0 (float64).
// Float and double-float accumulators are reduced as double-float on float32
// shuffles, float64 ones on float64 shuffles; the float64 totals are formed by
// one thread only (float64 issues at 1/64 of the float32 rate, so a per-thread
// float64 tail per iteration outweighs the stencil work of a small problem).
template <typename Acc>
__device__ void block_tot(const Acc (&ac)[4], int nv, Shared& sh, int tid, double (&tot)[4]) {
  const int lane = tid & 31, warp = tid >> 5;
  const int NWARP = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) tot[j] = 0.0;
  if constexpr (std::is_same<Acc, double>::value) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < nv) {
        double x = ac[j];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh.red[warp][j] = x;
      }
    }
    __syncthreads();
    if (tid == 0)
      for (int j = 0; j < nv; ++j) {
        double t = 0.0;
        for (int w = 0; w < NWARP; ++w) t += sh.red[w][j];
        tot[j] = t;
      }
  } else {
    df s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = acc_to_df(ac[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh.redf[warp][j] = make_float2(s[j].hi, s[j].lo);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j] = lane < NWARP ? cv(sh.redf[lane][j]) : df_make(0.f, 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < nv) s[j] = df_add(s[j], shfl_down(s[j], o));
      if (lane == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < nv) tot[j] = (double)s[j].hi + (double)s[j].lo;
    }
  }
}

// J y at (r, c) of the periodic advection-diffusion stencil, coefficients k = {E, W, N, S, C}
template <typename T, typename CJ>
__device__ __forceinline__ CJ jv_point(const T* y, int nx, int ny, int r, int c, const CJ (&k)[5]) {
  const int cm = c == 0 ? nx - 1 : c - 1, cp = c == nx - 1 ? 0 : c + 1;
  const int rm = r == 0 ? ny - 1 : r - 1, rp = r == ny - 1 ? 0 : r + 1;
  const CJ yc = to_cj(cv(y[(size_t)r * nx + c]), CJ());
  const CJ ye = to_cj(cv(y[(size_t)r * nx + cp]), CJ());
  const CJ yw = to_cj(cv(y[(size_t)r * nx + cm]), CJ());
  const CJ yn = to_cj(cv(y[(size_t)rp * nx + c]), CJ());
  const CJ ys = to_cj(cv(y[(size_t)rm * nx + c]), CJ());
  return k[0] * ye + k[1] * yw + k[2] * yn + k[3] * ys + k[4] * yc;
}

// One Newton-Leja pass (Sec. 2.2) of a CTA-owned problem: p_k = sum_m d_k[m] y_m,
// y_0 = x, y_{m+1} = ((J - c)/gamma - xi_m) y_m, stop at |d_k[m]| ||y_m|| <= tol ||p_k||
// (m >= m_min); tables in sh.  Returns the status; *iters = stopping m.
template <int P>
__device__ int block_pass(const BArgs& a, int nx, int ny, const typename Tr<P>::T* x, typename Tr<P>::T* y0,
                          typename Tr<P>::T* y1, typename Tr<P>::T* const* p, int K, const double* kJ, double gamma,
                          Shared& sh, int tid, int* iters) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  using CJ = typename Tr<P>::CJ;
  using Acc = typename Tr<P>::AccN;
  constexpr bool FOLD = std::is_same<C, CJ>::value;
  const int lane = tid & 31, warp = tid >> 5;
  const int NWARP = blockDim.x >> 5;
  const double al = 1.0 / gamma;
  CJ k0[5];
  for (int j = 0; j < 5; ++j) k0[j] = coef<CJ>(al * kJ[j], split_d(al * kJ[j]));
  // m = 0
  {
    Acc ac[4] = {acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>()};
    C d0[3];
    for (int k = 0; k < K; ++k) d0[k] = coef<C>(sh.dd[k][0], sh.ddf[k][0]);
    for (int r = warp; r < ny; r += NWARP)
      for (int c = lane; c < nx; c += 32) {
        const size_t i = (size_t)r * nx + c;
        const C xv = cv(x[i]);
        st1(y0 + i, xv);
        acc_sq(ac[0], xv);
        for (int k = 0; k < K; ++k) {
          const C pv = d0[k] * xv;
          st1(p[k] + i, pv);
          acc_sq(ac[1 + k], pv);
        }
      }
    __syncthreads();  // y_0 and p_k written before the first iteration reads them
  }
  const int m_max = a.m_max;
  for (int m = 1; m <= m_max; ++m) {
    const T* yin = (m & 1) ? y0 : y1;
    T* yout = (m & 1) ? y1 : y0;
    CJ kk[5];
    for (int j = 0; j < 5; ++j) kk[j] = k0[j];
    const C beta = coef<C>(sh.beta[m], sh.betaf[m]);
    if constexpr (FOLD) kk[4] = kk[4] + from_cj(beta, CJ());
    C dk[3];
    for (int k = 0; k < K; ++k) dk[k] = coef<C>(sh.dd[k][m], sh.ddf[k][m]);
    Acc ac[4] = {acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>(), acc_zero<Acc>()};
    for (int r = warp; r < ny; r += NWARP)
      for (int c = lane; c < nx; c += 32) {
        const size_t i = (size_t)r * nx + c;
        const CJ J = jv_point<T, CJ>(yin, nx, ny, r, c, kk);
        C out;
        if constexpr (FOLD)
          out = from_cj(J, C());
        else
          out = from_cj(J, C()) + beta * cv(yin[i]);
        st1(yout + i, out);
        acc_sq(ac[0], out);
        for (int k = 0; k < K; ++k) {
          C pv = ldw1(p[k] + i);
          pv = pv + dk[k] * out;
          st1(p[k] + i, pv);
          acc_sq(ac[1 + k], pv);
        }
      }
    double t[4];
    block_tot<Acc>(ac, K + 1, sh, tid, t);  // its barrier orders this iteration's writes before the next reads
    // stop test (Sec. 2.2) |d_k[m]| ||y_m|| <= tol ||p_k|| on the squares, in thread 0
    if (tid == 0) {
      const double ny2 = t[0], tol2 = a.tol * a.tol;
      bool finite = isfinite(ny2), conv = (m >= a.m_min);
      for (int k = 0; k < K; ++k) {
        const double np2 = t[1 + k], d = sh.dd[k][m];
        finite = finite && isfinite(np2);
        conv = conv && (d * d * ny2 <= tol2 * np2);
      }
      sh.flag = !finite ? 2 : (conv ? 1 : 0);
    }
    __syncthreads();  // also: warp 0 has read the shared partials before they are rewritten
    // every thread reads the flag before the next iteration's reduction barrier,
    // after which thread 0 rewrites it
    const int flag = sh.flag;
    if (flag == 2) {
      *iters = m;
      return PHIX_ENAN;
    }
    if (flag == 1) {
      *iters = m;
      return PHIX_OK;
    }
  }
  *iters = m_max;
  return PHIX_ENOTCONV;
}

template <int P, int BT>
__global__ void __launch_bounds__(BT) k_batched(BArgs a) {
  using T = typename Tr<P>::T;
  using C = typename Tr<P>::C;
  constexpr int BTHREADS = BT, NWARP = BT / 32;
  __shared__ Shared sh;
  __shared__ int slot_s;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int tid = threadIdx.x;
  const int M = a.m_max + 1;
  for (;;) {
    if (tid == 0) slot_s = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int slot = slot_s;
    __syncthreads();
    if (slot >= a.nprob) break;
    Prob& pr = a.probs[a.order[slot]];
    const int nx = pr.nx, ny = pr.ny;
    const size_t N = (size_t)nx * ny;
    T* W = static_cast<T*>(a.ws) + pr.ws;
    T* Y0 = W;
    T* Y1 = W + N;
    T* PP[3] = {W + 2 * N, W + 3 * N, W + 4 * N};
    T* VV = W + 5 * N;
    T* U = W + 6 * N;
    T* WW[3] = {U, W + 7 * N, W + 8 * N};
    T* TMP = W + 9 * N;
    // J coefficients (float64): {E, W, N, S, C}
    const double ix2 = (double)nx * nx, iy2 = (double)ny * ny;
    double kJ[5] = {pr.D * ix2 + 0.5 * pr.ax * nx, pr.D * ix2 - 0.5 * pr.ax * nx, pr.D * iy2 + 0.5 * pr.ay * ny,
                    pr.D * iy2 - 0.5 * pr.ay * ny, -2.0 * pr.D * (ix2 + iy2)};
    const double alpha_i = -pr.rho_re, beta_i = pr.rho_hi;
    // half-width covering twice the imaginary extent (complex spectra), the
    // interval anchored at its right end beta
    const double gamma = fmax(0.25 * (beta_i - alpha_i), 2.0 * fmax(0.0, pr.rho_im));
    const double cc = beta_i - 2.0 * gamma;
    const double h = pr.h;
    // input in the iteration precision
    for (size_t i = tid; i < N; i += BTHREADS) {
      C x;
      if constexpr (P == P_FP64)
        x = pr.v[i];
      else if constexpr (P == P_FP32)
        x = (float)pr.v[i];
      else
        x = df_split_pow2(pr.v[i], 0);
      st1(VV + i, x);
    }
    __syncthreads();
    int status = PHIX_OK, iters = 0, subs = 0;
    if (gamma == 0.0) {
      for (int k = 0; k < a.nout; ++k) {
        double f = 1.0;
        for (int j = 2; j <= a.l[k]; ++j) f *= j;
        for (size_t i = tid; i < N; i += BTHREADS) pr.out[k][i] = pr.v[i] / f;
      }
    } else {
      for (int m = tid; m < M; m += BTHREADS) {
        const double b = m >= 1 ? -(cc / gamma + a.xi[m - 1]) : 0.0;
        sh.beta[m] = b;
        sh.betaf[m] = split_d(b);
      }
      int s = 1;
      if (a.gamma_cap > 0) s = max(s, (int)ceil(h * gamma / a.gamma_cap - 1e-12));
      if (a.iota_cap > 0 && pr.rho_im > 0) s = max(s, (int)ceil(h * pr.rho_im / a.iota_cap - 1e-12));
      __syncthreads();
      if (s == 1) {
        for (int k = 0; k < a.nout; ++k)
          dd_block(a.l[k], h * cc, h * gamma, a.xi, M, sh.dd[k], sh.ddf[k], sh.tmp, tid);
        int it = 0;
        T* y0 = Y0;
        T* y1 = Y1;
        T* pp[3] = {PP[0], PP[1], PP[2]};
        if ((size_t)(2 + a.nout) * N * sizeof(T) <= a.smem_bytes) {
          // small problem: the whole pass on shared memory (generic addressing)
          T* sm = reinterpret_cast<T*>(dyn_smem);
          y0 = sm;
          y1 = sm + N;
          for (int k = 0; k < a.nout; ++k) pp[k] = sm + (2 + k) * N;
        }
        status = block_pass<P>(a, nx, ny, VV, y0, y1, pp, a.nout, kJ, gamma, sh, tid, &it);
        iters = it;
        subs = 1;
        for (int k = 0; k < a.nout; ++k)
          for (size_t i = tid; i < N; i += BTHREADS) {
            const C pv = cv(pp[k][i]);
            double d;
            if constexpr (P == P_FP64)
              d = pv;
            else if constexpr (P == P_FP32)
              d = (double)pv;
            else
              d = df_to_double_pow2(pv, 0);
            pr.out[k][i] = d;
          }
      } else {
        // ODE-identity substeps per output:
        //   u(t+tau) = sum_{j<l} tau^j/j! w_j + tau^l phi_l(tau B) w_l,
        //   w_0 = u(t), w_j = B w_{j-1} + v t^(l-j)/(l-j)!,  B = h J
        const double tau = 1.0 / s;
        using CJ = typename Tr<P>::CJ;
        CJ kb[5];
        for (int j = 0; j < 5; ++j) kb[j] = coef<CJ>(h * kJ[j], split_d(h * kJ[j]));
        for (int k = 0; k < a.nout; ++k) {
          const int L = a.l[k];
          dd_block(L, tau * h * cc, tau * h * gamma, a.xi, M, sh.dd[0], sh.ddf[0], sh.tmp, tid);
          for (size_t i = tid; i < N; i += BTHREADS) st1(U + i, L == 0 ? cv(VV[i]) : C{});
          __syncthreads();
          for (int sub = 0; sub < s; ++sub) {
            const double t = sub * tau;
            for (int j = 1; j <= L; ++j) {
              double cf = 1.0;
              for (int q = 0; q < L - j; ++q) cf *= t;
              for (int q = 2; q <= L - j; ++q) cf /= q;
              const C cfc = coef<C>(cf, split_d(cf));
              for (int r = tid >> 5; r < ny; r += NWARP)
                for (int c = tid & 31; c < nx; c += 32) {
                  const size_t i = (size_t)r * nx + c;
                  const C jv = from_cj(jv_point<T, CJ>(WW[j - 1], nx, ny, r, c, kb), C());
                  st1(WW[j] + i, jv + cfc * cv(VV[i]));
                }
              __syncthreads();
            }
            T* outp[1] = {TMP};
            int it = 0;
            const int st = block_pass<P>(a, nx, ny, WW[L], Y0, Y1, outp, 1, kJ, gamma, sh, tid, &it);
            iters += it;
            if (st != PHIX_OK) status = st;
            // u = tau^l tmp + sum_{j<l} tau^j / j! w_j
            double cw[3] = {1.0, tau, 0.5 * tau * tau};
            const double tl = L == 0 ? 1.0 : (L == 1 ? tau : tau * tau * (L == 2 ? 1.0 : tau));
            const C ctl = coef<C>(tl, split_d(tl));
            C cwc[3];
            for (int j = 0; j < 3; ++j) cwc[j] = coef<C>(cw[j], split_d(cw[j]));
            for (size_t i = tid; i < N; i += BTHREADS) {
              C un = ctl * cv(TMP[i]);
              for (int j = 0; j < L; ++j) un = un + cwc[j] * cv(WW[j][i]);
              st1(U + i, un);
            }
            __syncthreads();
          }
          subs += s;
          for (size_t i = tid; i < N; i += BTHREADS) {
            const C uv = cv(U[i]);
            double d;
            if constexpr (P == P_FP64)
              d = uv;
            else if constexpr (P == P_FP32)
              d = (double)uv;
            else
              d = df_to_double_pow2(uv, 0);
            pr.out[k][i] = d;
          }
          __syncthreads();
        }
      }
    }
    if (tid == 0) {
      pr.status = status;
      pr.iters = iters;
      pr.substeps = subs;
    }
    __syncthreads();
  }
}

}  // namespace

size_t batched_prob_bytes() { return sizeof(Prob); }

template <int P>
static void* batched_fn(int bt) {
  switch (bt) {
    case 256:
      return (void*)k_batched<P, 256>;
    case 512:
      return (void*)k_batched<P, 512>;
    case 1024:
      return (void*)k_batched<P, 1024>;
  }
  return nullptr;
}
static void* batched_kernel(int prec, int bt) {
  switch (prec) {
    case P_FP64:
      return batched_fn<P_FP64>(bt);
    case P_DF64:
      return batched_fn<P_DF64>(bt);
    case P_FP32JV:
      return batched_fn<P_FP32JV>(bt);
  }
  return nullptr;
}

int batched_blocks_per_sm(int prec, int bt, unsigned int smem_bytes) {
  void* fn = batched_kernel(prec, bt);
  if (!fn) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, bt, smem_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return nb;
}

// probs: device array of nprob Prob records (host-built with batched_fill_prob)
cudaError_t launch_batched(int prec, void* probs, const int* order, int nprob, unsigned int* queue, void* ws,
                           const double* xi, int m_max, int m_min, double tol, double gamma_cap, double iota_cap,
                           int nout, const int* l, int grid, int bt, unsigned int smem_bytes, cudaStream_t st) {
  if (m_max + 1 > BM || nout < 1 || nout > 3) return cudaErrorInvalidValue;
  BArgs a{};
  a.probs = static_cast<Prob*>(probs);
  a.order = order;
  a.nprob = nprob;
  a.queue = queue;
  a.ws = ws;
  a.xi = xi;
  a.m_max = m_max;
  a.m_min = m_min;
  a.tol = tol;
  a.gamma_cap = gamma_cap;
  a.iota_cap = iota_cap;
  a.nout = nout;
  for (int k = 0; k < nout; ++k) a.l[k] = l[k];
  a.smem_bytes = smem_bytes;
  void* fn = batched_kernel(prec, bt);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  void* args[1] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(bt), args, smem_bytes, st);
}

void batched_fill_prob(void* dst, int nx, int ny, double D, double ax, double ay, double h, double rho_re,
                       double rho_hi, double rho_im, const double* v, double* const* out, int nout,
                       unsigned long long ws_off) {
  Prob p{};
  p.nx = nx;
  p.ny = ny;
  p.D = D;
  p.ax = ax;
  p.ay = ay;
  p.h = h;
  p.rho_re = rho_re;
  p.rho_hi = rho_hi;
  p.rho_im = rho_im;
  p.v = v;
  for (int k = 0; k < nout && k < 3; ++k) p.out[k] = out[k];
  p.ws = ws_off;
  std::memcpy(dst, &p, sizeof p);
}

void batched_read_prob(const void* src, int* status, int* iters, int* substeps) {
  Prob p;
  std::memcpy(&p, src, sizeof p);
  *status = p.status;
  *iters = p.iters;
  *substeps = p.substeps;
}

}  // namespace phix
