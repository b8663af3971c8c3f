// Point evaluations of the right-hand sides f(u) and Jacobian actions J(u)x of
// every operator (Sec. 3: second-order centred differences), float64, for the
// stage kernels and the general Newton-Leja kernel.  Periodic operators live
// on the unit square with nodes x_j = j / n; the paper's no-flow problems
// (ADR, Allen-Cahn, Brusselator) on cell-centred grids of [0, 1]^2 (Allen-Cahn:
// [-1, 1]^2) whose Neumann ghost cells repeat the boundary cell.
#pragma once
#include "phix_internal.h"

namespace phix {

// operators with no-flow (Neumann) boundaries
__host__ __device__ __forceinline__ bool op_neumann(int kind) { return kind >= PHIX_OP_ADR; }
__host__ __device__ __forceinline__ int op_ncomp(int kind) {
  return (kind == PHIX_OP_GRAYSCOTT || kind == PHIX_OP_BRUSSELATOR) ? 2 : 1;
}
__host__ __device__ __forceinline__ double op_length(int kind) { return kind == PHIX_OP_ALLEN_CAHN ? 2.0 : 1.0; }

struct Nbr {
  double c, e, w, n, s;
};

struct Geo {
  int nx, ny;
  bool neumann;
  double idx2, idy2, i2dx, i2dy;
};

__device__ __forceinline__ Geo make_geo(int kind, int nx, int ny) {
  Geo g;
  g.nx = nx;
  g.ny = ny;
  g.neumann = op_neumann(kind);
  const double L = op_length(kind);
  const double dx = L / nx, dy = L / ny;
  g.idx2 = 1.0 / (dx * dx);
  g.idy2 = 1.0 / (dy * dy);
  g.i2dx = 0.5 / dx;
  g.i2dy = 0.5 / dy;
  return g;
}

__device__ __forceinline__ Nbr load_nbr(const double* __restrict__ x, const Geo& g, int ix, int iy) {
  int ixm, ixp, iym, iyp;
  if (g.neumann) {  // ghost = boundary cell
    ixm = ix == 0 ? 0 : ix - 1;
    ixp = ix == g.nx - 1 ? ix : ix + 1;
    iym = iy == 0 ? 0 : iy - 1;
    iyp = iy == g.ny - 1 ? iy : iy + 1;
  } else {
    ixm = ix == 0 ? g.nx - 1 : ix - 1;
    ixp = ix == g.nx - 1 ? 0 : ix + 1;
    iym = iy == 0 ? g.ny - 1 : iy - 1;
    iyp = iy == g.ny - 1 ? 0 : iy + 1;
  }
  Nbr r;
  r.c = x[(size_t)iy * g.nx + ix];
  r.e = x[(size_t)iy * g.nx + ixp];
  r.w = x[(size_t)iy * g.nx + ixm];
  r.n = x[(size_t)iyp * g.nx + ix];
  r.s = x[(size_t)iym * g.nx + ix];
  return r;
}

__device__ __forceinline__ double lap(const Nbr& a, const Geo& g) {
  return (a.e + a.w - 2.0 * a.c) * g.idx2 + (a.n + a.s - 2.0 * a.c) * g.idy2;
}
__device__ __forceinline__ double grad_sum(const Nbr& a, const Geo& g) {  // a_x + a_y
  return (a.e - a.w) * g.i2dx + (a.n - a.s) * g.i2dy;
}
__device__ __forceinline__ Nbr axpy_nbr(const Nbr& u, double e, const Nbr& y) {
  return Nbr{u.c + e * y.c, u.e + e * y.e, u.w + e * y.w, u.n + e * y.n, u.s + e * y.s};
}

// f at a point from the neighbourhoods of its species (b: second species).
__device__ __forceinline__ void rhs_nbr(int kind, const double* p, const Geo& g, const Nbr& a, const Nbr& b,
                                        double* out) {
  switch (kind) {
    case PHIX_OP_ADVDIFF:
      out[0] = p[0] * lap(a, g) + p[1] * (a.e - a.w) * g.i2dx + p[2] * (a.n - a.s) * g.i2dy;
      break;
    case PHIX_OP_GRAYSCOTT: {
      const double uvv = a.c * b.c * b.c;
      out[0] = p[0] * lap(a, g) - uvv + p[2] * (1.0 - a.c);
      out[1] = p[1] * lap(b, g) + uvv - (p[2] + p[3]) * b.c;
      break;
    }
    case PHIX_OP_BURGERS:
      out[0] = p[0] * lap(a, g) - a.c * grad_sum(a, g);
      break;
    case PHIX_OP_ADR:  // a lap u + b (u_x + u_y) + g u (1 - u) (u - 1/2)
      out[0] = p[0] * lap(a, g) + p[1] * grad_sum(a, g) + p[2] * a.c * (1.0 - a.c) * (a.c - 0.5);
      break;
    case PHIX_OP_ALLEN_CAHN:  // a lap u + u - u^3
      out[0] = p[0] * lap(a, g) + a.c - a.c * a.c * a.c;
      break;
    default: {  // Brusselator: a lap u + 1 + u^2 v - 4u,  a lap v + 3u - u^2 v
      const double uuv = a.c * a.c * b.c;
      out[0] = p[0] * lap(a, g) + 1.0 + uuv - 4.0 * a.c;
      out[1] = p[0] * lap(b, g) + 3.0 * a.c - uuv;
    }
  }
}

// J(state) x at a point: x neighbourhoods (xa, xb), state neighbourhoods (sa, sb).
__device__ __forceinline__ void jv_nbr(int kind, const double* p, const Geo& g, const Nbr& xa, const Nbr& xb,
                                       const Nbr& sa, const Nbr& sb, double* out) {
  switch (kind) {
    case PHIX_OP_ADVDIFF:
      out[0] = p[0] * lap(xa, g) + p[1] * (xa.e - xa.w) * g.i2dx + p[2] * (xa.n - xa.s) * g.i2dy;
      break;
    case PHIX_OP_GRAYSCOTT: {
      const double U = sa.c, V = sb.c;
      out[0] = p[0] * lap(xa, g) - (V * V + p[2]) * xa.c - 2.0 * U * V * xb.c;
      out[1] = p[1] * lap(xb, g) + V * V * xa.c + (2.0 * U * V - (p[2] + p[3])) * xb.c;
      break;
    }
    case PHIX_OP_BURGERS:
      out[0] = p[0] * lap(xa, g) - grad_sum(sa, g) * xa.c - sa.c * grad_sum(xa, g);
      break;
    case PHIX_OP_ADR: {
      const double U = sa.c;
      out[0] = p[0] * lap(xa, g) + p[1] * grad_sum(xa, g) + p[2] * (-3.0 * U * U + 3.0 * U - 0.5) * xa.c;
      break;
    }
    case PHIX_OP_ALLEN_CAHN: {
      const double U = sa.c;
      out[0] = p[0] * lap(xa, g) + (1.0 - 3.0 * U * U) * xa.c;
      break;
    }
    default: {
      const double U = sa.c, V = sb.c;
      out[0] = p[0] * lap(xa, g) + (2.0 * U * V - 4.0) * xa.c + U * U * xb.c;
      out[1] = p[0] * lap(xb, g) + (3.0 - 2.0 * U * V) * xa.c - U * U * xb.c;
    }
  }
}

}  // namespace phix
