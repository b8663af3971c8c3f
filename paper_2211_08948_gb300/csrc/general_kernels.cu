// The general Newton-Leja / power-iteration step, float64: every operator
// (the periodic ones and the paper's no-flow problems of Sec. 3), the
// Jacobian action analytic or by finite differences of f (Sec. 4, the
// "numerical Jacobian"), and the source terms of the augmented-matrix form
// (Appendix A).  One launch = one iteration; the last block reduces the
// partial norms in block order and takes the stop decision of Sec. 2.2, as
// the fast single-step kernel does.  This path serves what the fast
// double-float kernels do not cover; it runs one point per thread.
//
//   Newton: y_{m+1} = a J y_m + beta_m y_m + sum_j w_{m,j} src_j   (a = 1/gamma)
//           p_k   += d_k[m+1] y_{m+1}; stop on the norms plus the host-known
//           parts of an augmented vector (its p-dimensional tail)
//   power:  y_k = alpha J y_{k-1}, alpha = 1 / ||y_{k-1}||, rho_k = ||y_k||
//   init:   y_0 = v, p_k = d_k[0] y_0
#include "iter_common.cuh"
#include "op_points.cuh"

namespace phix {

namespace {

constexpr int GT = 256;

struct GenArgs {
  int kind, nx, ny, K, mode, fd, nsrc;
  const double* v;                // init: the input
  double* y[2];                   // ping-pong (launch m reads y[(m-1)&1], writes y[m&1])
  double* p[KMAX];                // accumulators (the caller's outputs)
  const double* st;               // state planes (nonlinear operators), NULL otherwise
  const double* fu;               // f(state) (finite differences)
  double fd_scale;                // sqrt(2^-52) (1 + ||state||)
  double prm[8];
  const double* src[KIOPS_PMAX];  // augmented-form sources b_j
  LejaCtl* ctl;
  double* partials;
  const double* tab;              // GenTable
};

}  // namespace

// Host-built table of one general pass (float64):
//   [0] K, [1] m_min, [2] m_max, [3] M, [4] tol, [5] rel, [6] a, [7] nsrc,
//   then beta[M], dk[KMAX][M], w[M][KIOPS_PMAX], ytail2[M], ptail2[KMAX][M].
size_t gen_table_doubles(int M) { return 8 + (size_t)M * (2 + KIOPS_PMAX + 2 * KMAX); }

namespace {

__device__ __forceinline__ const double* g_beta(const double* t) { return t + 8; }
__device__ __forceinline__ const double* g_dk(const double* t, int M) { return t + 8 + M; }
__device__ __forceinline__ const double* g_w(const double* t, int M) { return t + 8 + M + KMAX * M; }
__device__ __forceinline__ const double* g_yt(const double* t, int M) { return t + 8 + M + KMAX * M + KIOPS_PMAX * M; }
__device__ __forceinline__ const double* g_pt(const double* t, int M) {
  return t + 8 + 2 * M + KMAX * M + KIOPS_PMAX * M;
}

enum { G_NEWTON = 0, G_POWER = 1, G_INIT = 2 };

__global__ void __launch_bounds__(GT) k_general(GenArgs a) {
  if (a.mode != G_INIT && __ldcg(&a.ctl->done)) return;
  const double* t = a.tab;
  const int K = a.mode == G_POWER ? 0 : (int)t[0];
  const int M = (int)t[3];
  const int m = a.mode == G_INIT ? 0 : __ldcg(&a.ctl->m);
  const Geo g = make_geo(a.kind, a.nx, a.ny);
  const size_t plane = (size_t)a.nx * a.ny;
  const int nc = op_ncomp(a.kind);
  double coefA = 0.0, coefB = 0.0, eps = 0.0;
  double dk[KMAX] = {0, 0, 0, 0}, w[KIOPS_PMAX] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (a.mode == G_NEWTON) {
    coefA = t[6];
    coefB = g_beta(t)[m];
    for (int k = 0; k < K; ++k) dk[k] = g_dk(t, M)[k * M + m];
    // sources of y_m from the tail of y_{m-1}
    for (int j = 0; j < a.nsrc; ++j) w[j] = g_w(t, M)[(m - 1) * KIOPS_PMAX + j];
    if (a.fd) eps = a.fd_scale / sqrt(__ldcg(&a.ctl->ysq));
  } else if (a.mode == G_POWER) {
    coefA = __ldcg(&a.ctl->alpha);
    if (a.fd) eps = a.fd_scale * coefA;  // ||y_{k-1}|| = 1 / alpha
  } else {
    for (int k = 0; k < K; ++k) dk[k] = g_dk(t, M)[k * M];
  }
  const double* yin = a.mode == G_INIT ? a.v : a.y[(m - 1) & 1];
  double* yout = a.y[m & 1];
  const Nbr zero{0, 0, 0, 0, 0};
  double acc[KMAX + 1] = {0, 0, 0, 0, 0};
  for (size_t i = (size_t)blockIdx.x * GT + threadIdx.x; i < plane; i += (size_t)gridDim.x * GT) {
    const int ix = (int)(i % (size_t)a.nx), iy = (int)(i / (size_t)a.nx);
    double out[2];
    if (a.mode == G_INIT) {
      for (int q = 0; q < nc; ++q) out[q] = yin[q * plane + i];
    } else {
      const Nbr xa = load_nbr(yin, g, ix, iy);
      const Nbr xb = nc == 2 ? load_nbr(yin + plane, g, ix, iy) : xa;
      const Nbr sa = a.st ? load_nbr(a.st, g, ix, iy) : zero;
      const Nbr sb = (a.st && nc == 2) ? load_nbr(a.st + plane, g, ix, iy) : sa;
      double J[2];
      if (a.fd) {
        // (f(u + eps y) - f(u)) / eps
        double fw[2];
        rhs_nbr(a.kind, a.prm, g, axpy_nbr(sa, eps, xa), axpy_nbr(sb, eps, xb), fw);
        for (int q = 0; q < nc; ++q) J[q] = (fw[q] - a.fu[q * plane + i]) / eps;
      } else {
        jv_nbr(a.kind, a.prm, g, xa, xb, sa, sb, J);
      }
      const double yc[2] = {xa.c, xb.c};
      for (int q = 0; q < nc; ++q) {
        double o = coefA * J[q] + coefB * yc[q];
        for (int j = 0; j < a.nsrc; ++j) o += w[j] * a.src[j][q * plane + i];
        out[q] = o;
      }
    }
    for (int q = 0; q < nc; ++q) {
      yout[q * plane + i] = out[q];
      acc[0] += out[q] * out[q];
      for (int k = 0; k < K; ++k) {
        double* pk = a.p[k] + q * plane + i;
        const double pv = a.mode == G_INIT ? dk[k] * out[q] : *pk + dk[k] * out[q];
        *pk = pv;
        acc[1 + k] += pv * pv;
      }
    }
  }
  if (block_partials_and_last<double, KMAX + 1>(acc, a.partials, &a.ctl->count)) {
    double tot[KMAX + 1];
    reduce_partials<double, KMAX + 1>(a.partials, tot, NoHook{}, K + 1);
    if (threadIdx.x == 0) {
      LejaCtl* ctl = a.ctl;
      if (a.mode == G_POWER) {
        const double rho = sqrt(tot[0]);
        const double prev = ctl->rho;
        ctl->rho_prev = prev;
        ctl->rho = rho;
        ctl->iters = m;
        if (!isfinite(rho)) {
          ctl->status = PHIX_ENAN;
          ctl->done = 1;
        } else if (rho == 0.0) {
          ctl->status = PHIX_OK;
          ctl->done = 1;
        } else if ((m >= 2 && fabs(rho - prev) <= t[5] * rho) || m >= (int)t[2]) {
          ctl->status = PHIX_OK;
          ctl->done = 1;
        }
        ctl->alpha = 1.0 / rho;
      } else {
        double dkd[KMAX], tt[KMAX + 1];
        tt[0] = tot[0] + g_yt(t, M)[m];
        for (int k = 0; k < K; ++k) {
          dkd[k] = g_dk(t, M)[k * M + m];
          tt[1 + k] = tot[1 + k] + g_pt(t, M)[k * M + m];
        }
        leja_test(ctl, m, K, (int)t[1], (int)t[2], t[4], dkd, tt);
      }
      ctl->m = m + 1;
      ctl->count = 0;
    }
  }
}

}  // namespace

cudaError_t launch_general(int mode, int kind, int nx, int ny, int K, const double* v, double* const* y,
                           double* const* p, const double* st, const double* fu, double fd_scale, int fd,
                           const double* prm, const double* const* src, int nsrc, LejaCtl* ctl, double* partials,
                           const double* tab, int grid, cudaStream_t s) {
  GenArgs a{};
  a.kind = kind;
  a.nx = nx;
  a.ny = ny;
  a.K = K;
  a.mode = mode;
  a.fd = fd;
  a.nsrc = nsrc;
  a.v = v;
  a.y[0] = y[0];
  a.y[1] = y[1];
  for (int k = 0; k < KMAX; ++k) a.p[k] = k < K ? p[k] : nullptr;
  a.st = st;
  a.fu = fu;
  a.fd_scale = fd_scale;
  for (int j = 0; j < 8; ++j) a.prm[j] = prm[j];
  for (int j = 0; j < KIOPS_PMAX; ++j) a.src[j] = j < nsrc ? src[j] : nullptr;
  a.ctl = ctl;
  a.partials = partials;
  a.tab = tab;
  const size_t plane = (size_t)nx * ny;
  const int g = (int)std::max<size_t>(1, std::min<size_t>((size_t)grid, (plane + GT - 1) / GT));
  k_general<<<g, GT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace phix
