// Float64 kernels of the integrator stages: right-hand sides f(u), the
// nonlinear remainder R(a) = f(a) - f(u) - J(u)(a - u) (Sec. 1), Jacobian
// actions with an axpy (ODE-identity substeps), linear combinations and
// norms.  They run a handful of times per time step, against hundreds of
// Newton-Leja iterations, so they stay in plain float64.
#include "op_points.cuh"

namespace phix {

namespace {

__global__ void k_rhs(OpDesc op, const double* __restrict__ u, double* __restrict__ f) {
  const Geo g = make_geo(op.kind, op.nx, op.ny);
  const size_t plane = (size_t)g.nx * g.ny;
  const int nc = op_ncomp(op.kind);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)((unsigned)i % (unsigned)g.nx), iy = (int)((unsigned)i / (unsigned)g.nx);  // i < 2^31
    const Nbr a = load_nbr(u, g, ix, iy);
    const Nbr b = nc == 2 ? load_nbr(u + plane, g, ix, iy) : a;
    double o[2];
    rhs_nbr(op.kind, op.p, g, a, b, o);
    for (int q = 0; q < nc; ++q) f[q * plane + i] = o[q];
  }
}

// R(a) = f(a) - f(u) - J(u)(a - u) (Sec. 1).  The linear parts of f cancel
// exactly, so R is the remainder of the nonlinear term alone, with d = a - u:
//   Gray-Scott  n(u, v) = u v^2:   n(a) - n(u) - n'(u) d = dv (a_u dv + 2 v du),
//               R_u = -that, R_v = +that (pointwise, no stencil);
//   Burgers     n(u) = -u (D_x u + D_y u):  R = -d (D_x d + D_y d);
//   advection-diffusion is linear: R = 0.
// This is the same quantity as the definition, without its cancellation
// (f(a) and f(u) carry the O(n^2) Laplacian terms; R is O(|d|^2)).
__global__ void k_remainder_gs(size_t plane, const double* __restrict__ u, const double* __restrict__ a,
                               double* __restrict__ R) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  auto body = [&](size_t i, double uu, double v, double au, double av) {
    const double du = au - uu, dv = av - v;
    const double r = dv * (au * dv + 2.0 * v * du);
    R[i] = -r;
    R[plane + i] = r;
  };
  // the thread's points in grid-stride order, their loads issued UNR at a time
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (UNR - 1) * stride < plane; i += UNR * stride) {
    double uu[UNR], v[UNR], au[UNR], av[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const size_t j = i + q * stride;
      uu[q] = u[j];
      v[q] = u[plane + j];
      au[q] = a[j];
      av[q] = a[plane + j];
    }
#pragma unroll
    for (int q = 0; q < UNR; ++q) body(i + q * stride, uu[q], v[q], au[q], av[q]);
  }
  for (; i < plane; i += stride) body(i, u[i], u[plane + i], a[i], a[plane + i]);
}

__global__ void k_remainder_burgers(OpDesc op, const double* __restrict__ u, const double* __restrict__ a,
                                    double* __restrict__ R) {
  const Geo g = make_geo(op.kind, op.nx, op.ny);
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;  // <= 2^31 points
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += gridDim.x * blockDim.x) {
    const int ix = (int)(i % (unsigned)g.nx), iy = (int)(i / (unsigned)g.nx);
    Nbr A = load_nbr(a, g, ix, iy), U = load_nbr(u, g, ix, iy);
    Nbr d{A.c - U.c, A.e - U.e, A.w - U.w, A.n - U.n, A.s - U.s};
    R[i] = -d.c * grad_sum(d, g);
  }
}

// The no-flow problems' remainders, pointwise in d = a - u (their linear parts
// cancel):  ADR  g (n(a) - n(u) - n'(u) d) with n(u) = u (1-u)(u-1/2):  g d^2 (3/2 - a - 2u);
// Allen-Cahn  -(a^3 - u^3 - 3u^2 d) = -d^2 (a + 2u);
// Brusselator  a_u^2 a_v - u^2 v - 2uv d_u - u^2 d_v = d_u (2u d_v + v d_u + d_u d_v) = R_u, R_v = -R_u.
__global__ void k_remainder_point(int kind, double gcoef, size_t plane, const double* __restrict__ u,
                                  const double* __restrict__ a, double* __restrict__ R) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const double uc = u[i], ac = a[i], d = ac - uc;
    if (kind == PHIX_OP_ADR) {
      R[i] = gcoef * d * d * (1.5 - ac - 2.0 * uc);
    } else if (kind == PHIX_OP_ALLEN_CAHN) {
      R[i] = -d * d * (ac + 2.0 * uc);
    } else {
      const double v = u[plane + i], dv = a[plane + i] - v;
      const double r = d * (2.0 * uc * dv + v * d + d * dv);
      R[i] = r;
      R[plane + i] = -r;
    }
  }
}

__global__ void k_jv_axpy(OpDesc op, const double* __restrict__ st, const double* __restrict__ x,
                          double alpha, const double* __restrict__ v, double beta,
                          double* __restrict__ out) {
  const Geo g = make_geo(op.kind, op.nx, op.ny);
  const size_t plane = (size_t)g.nx * g.ny;
  const int nc = op_ncomp(op.kind);
  const Nbr zero{0, 0, 0, 0, 0};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)((unsigned)i % (unsigned)g.nx), iy = (int)((unsigned)i / (unsigned)g.nx);  // i < 2^31
    const Nbr xa = load_nbr(x, g, ix, iy);
    const Nbr xb = nc == 2 ? load_nbr(x + plane, g, ix, iy) : xa;
    const Nbr sa = st ? load_nbr(st, g, ix, iy) : zero;
    const Nbr sb = (st && nc == 2) ? load_nbr(st + plane, g, ix, iy) : sa;
    double o[2];
    jv_nbr(op.kind, op.p, g, xa, xb, sa, sb, o);
    for (int q = 0; q < nc; ++q) {
      double r = alpha * o[q];
      if (v) r += beta * v[q * plane + i];
      out[q * plane + i] = r;
    }
  }
}

struct Comb {
  double c[6];
  const double* x[6];
};

__global__ void k_lincomb(size_t n, int nt, Comb cb, double* out) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // UNR elements per pass: each term's loads of them issued together; every
  // element's sum runs over the terms in order, as in the element loop below
  for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
    double r[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) r[q] = 0.0;
    for (int t = 0; t < nt; ++t) {
      double x[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) x[q] = cb.x[t][i + q * stride];
#pragma unroll
      for (int q = 0; q < UNR; ++q) r[q] += cb.c[t] * x[q];
    }
#pragma unroll
    for (int q = 0; q < UNR; ++q) out[i + q * stride] = r[q];
  }
  for (; i < n; i += stride) {
    double r = 0.0;
    for (int t = 0; t < nt; ++t) r += cb.c[t] * cb.x[t][i];
    out[i] = r;
  }
}

__global__ void k_norm2(size_t n, const double* __restrict__ x, const double* __restrict__ y,
                        double* partials, unsigned int* counter, double* result) {
  __shared__ double sw[32];
  __shared__ bool last;
  double s = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (UNR - 1) * stride < n; i += UNR * stride) {
    double d[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) d[q] = y ? x[i + q * stride] - y[i + q * stride] : x[i + q * stride];
#pragma unroll
    for (int q = 0; q < UNR; ++q) s = fma(d[q], d[q], s);
  }
  for (; i < n; i += stride) {
    double d = y ? x[i] - y[i] : x[i];
    s = fma(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sw[w];
    partials[blockIdx.x] = b;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    // fixed-order parallel sum of the block partials
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + b);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sw[w];
      *result = tot;
      *counter = 0;
      __threadfence();
    }
  }
}

}  // namespace

static inline int clamp_grid(size_t work, int grid) {
  size_t need = (work + 255) / 256;
  if (need < 1) need = 1;
  return (int)(need < (size_t)grid ? need : (size_t)grid);
}

cudaError_t launch_rhs(const OpDesc& op, const double* u, double* f, int grid, cudaStream_t s) {
  size_t plane = (size_t)op.nx * op.ny;
  k_rhs<<<clamp_grid(plane, grid), 256, 0, s>>>(op, u, f);
  return cudaGetLastError();
}

cudaError_t launch_remainder(const OpDesc& op, const double* u, const double* a, double* R, int grid,
                             cudaStream_t s) {
  const size_t plane = (size_t)op.nx * op.ny;
  if (op.kind == PHIX_OP_GRAYSCOTT) {
    k_remainder_gs<<<clamp_grid(plane, grid), 256, 0, s>>>(plane, u, a, R);
  } else if (op.kind == PHIX_OP_BURGERS) {
    k_remainder_burgers<<<clamp_grid(plane, grid), 256, 0, s>>>(op, u, a, R);
  } else if (op.kind >= PHIX_OP_ADR) {
    k_remainder_point<<<clamp_grid(plane, grid), 256, 0, s>>>(op.kind, op.p[2], plane, u, a, R);
  } else {
    return cudaMemsetAsync(R, 0, plane * sizeof(double), s);
  }
  return cudaGetLastError();
}

cudaError_t launch_jv_axpy(const OpDesc& op, const double* state, const double* x, double alpha,
                           const double* v, double beta, double* out, int grid, cudaStream_t s) {
  size_t plane = (size_t)op.nx * op.ny;
  k_jv_axpy<<<clamp_grid(plane, grid), 256, 0, s>>>(op, state, x, alpha, v, beta, out);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(size_t n, int nterms, const double* c, const double* const* x,
                           double* out, int grid, cudaStream_t s) {
  if (nterms < 1 || nterms > 6) return cudaErrorInvalidValue;
  Comb cb{};
  for (int t = 0; t < nterms; ++t) {
    cb.c[t] = c[t];
    cb.x[t] = x[t];
  }
  k_lincomb<<<clamp_grid(n, grid), 256, 0, s>>>(n, nterms, cb, out);
  return cudaGetLastError();
}

cudaError_t launch_norm2(size_t n, const double* x, const double* y, double* partials,
                         unsigned int* counter, double* result, int grid, cudaStream_t s) {
  k_norm2<<<clamp_grid(n, grid), 256, 0, s>>>(n, x, y, partials, counter, result);
  return cudaGetLastError();
}

}  // namespace phix
