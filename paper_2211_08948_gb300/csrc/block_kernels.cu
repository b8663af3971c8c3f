// Kernels of the domain-decomposed Newton-Leja pass (Sec. 2.2; the paper's
// case for Leja over Krylov is its small number of inner products, Sec. 1 and
// Sec. 2.1): a rank owns rectangular blocks of the global periodic grid, each
// stored with a one-cell halo ring, and one Newton iteration on a block needs
// only its halo (exchanged by the caller) and one reduction of squared norms.
//
// Block layout: per species a padded (bx + 2) x (by + 2) plane, row-major, the
// interior at rows 1..by, columns 1..bx; accumulators p_k are unpadded bx x by
// planes.  Face buffers (pack / unpack): [S | N | W | E], each face holding
// all species contiguously (ncomp * bx for S and N, ncomp * by for W and E):
// pack reads the interior faces (row 1, row by, column 1, column bx), unpack
// writes the halo faces (row 0, row by + 1, column 0, column bx + 1).
// Arithmetic: float64.
#include <cmath>
#include <cstring>

#include "iter_common.cuh"

namespace phix {

namespace {

constexpr int BT = 256;

struct BlockArgs {
  int bx, by, ncomp, K, init;
  const double* yin;   // padded
  double* yout;        // padded (unused when init)
  double* p[KMAX];     // unpadded
  const double* st;    // padded state (Gray-Scott: u, v planes; Burgers: U), may be NULL
  double k[8];         // uniform J coefficients (unscaled)
  double dk[KMAX];
  double a, b;         // y' = a J y + b y
  double* partials;    // gridDim.x * (KMAX + 1)
  unsigned int* counter;
  double* norms;       // K + 1 totals
};

// Sum of (KMAX + 1) values over the block into partials[blockIdx], the last
// block to finish adds the partials in block order (deterministic).
__device__ void block_reduce_store(double (&acc)[KMAX + 1], const BlockArgs& a) {
  __shared__ double sh[KMAX + 1][BT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j <= KMAX; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[j][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j <= KMAX; ++j) {
      double s = 0.0;
      for (int q = 0; q < BT / 32; ++q) s += sh[j][q];
      a.partials[blockIdx.x * (KMAX + 1) + j] = s;
    }
    __threadfence();
    last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x <= KMAX) {
    __threadfence();
    double s = 0.0;
    for (unsigned q = 0; q < gridDim.x; ++q) s += __ldcg(&a.partials[q * (KMAX + 1) + threadIdx.x]);
    if ((int)threadIdx.x <= a.K) a.norms[threadIdx.x] = s;
  }
  if (last && threadIdx.x == 0) *a.counter = 0;
}

template <int OP>
__global__ void __launch_bounds__(BT) k_block_newton(BlockArgs a) {
  constexpr int NC = OP == PHIX_OP_GRAYSCOTT ? 2 : 1;
  const int px = a.bx + 2;
  const size_t pplane = (size_t)px * (a.by + 2), plane = (size_t)a.bx * a.by;
  double acc[KMAX + 1] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double k8[8] = {a.k[0], a.k[1], a.k[2], a.k[3], a.k[4], a.k[5], a.k[6], a.k[7]};
  for (size_t i = (size_t)blockIdx.x * BT + threadIdx.x; i < plane; i += (size_t)gridDim.x * BT) {
    const int x = (int)(i % a.bx), y = (int)(i / a.bx);
    const size_t c = (size_t)(y + 1) * px + (x + 1);
    double yc[NC], out[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) yc[q] = a.yin[q * pplane + c];
    if (a.init) {
#pragma unroll
      for (int q = 0; q < NC; ++q) out[q] = yc[q];
    } else {
      double J[NC];
      if constexpr (OP == PHIX_OP_ADVDIFF) {
        const double* Y = a.yin;
        J[0] = stencil_advdiff<double>(k8, Y[c + 1], Y[c - 1], Y[c + px], Y[c - px], Y[c]);
      } else if constexpr (OP == PHIX_OP_GRAYSCOTT) {
        const double* U = a.yin;
        const double* V = a.yin + pplane;
        const double su = a.st[c], sv = a.st[pplane + c];
        stencil_gs<double>(k8, 1.0, U[c + 1], U[c - 1], U[c + px], U[c - px], U[c], V[c + 1], V[c - 1],
                           V[c + px], V[c - px], V[c], sv * sv, 2.0 * su * sv, J[0], J[1]);
      } else {
        const double* Y = a.yin;
        const double* S = a.st;
        J[0] = stencil_burgers<double>(k8, 1.0, Y[c + 1], Y[c - 1], Y[c + px], Y[c - px], Y[c], S[c + 1],
                                       S[c - 1], S[c + px], S[c - px], S[c]);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        out[q] = a.a * J[q] + a.b * yc[q];
        a.yout[q * pplane + c] = out[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      acc[0] += out[q] * out[q];
#pragma unroll
      for (int kq = 0; kq < KMAX; ++kq) {
        if (kq < a.K) {
          double* pk = a.p[kq] + q * plane + i;
          const double pv = a.init ? a.dk[kq] * out[q] : *pk + a.dk[kq] * out[q];
          *pk = pv;
          acc[1 + kq] += pv * pv;
        }
      }
    }
  }
  block_reduce_store(acc, a);
}

// Faces: pack (dir = 0) interior faces into buf; unpack (dir = 1) halo faces from buf.
__global__ void k_block_faces(int bx, int by, int ncomp, int dir, double* ypad, double* buf) {
  const int px = bx + 2;
  const size_t pplane = (size_t)px * (by + 2);
  const int per = 2 * bx + 2 * by;  // one species' four faces
  const int total = ncomp * per;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    // buffer index i -> (face, species, position): faces S, N hold ncomp * bx each, W, E ncomp * by
    int f, q, t, off;
    if (i < 2 * ncomp * bx) {
      f = i / (ncomp * bx);
      off = i - f * ncomp * bx;
      q = off / bx;
      t = off - q * bx;
    } else {
      const int j = i - 2 * ncomp * bx;
      f = 2 + j / (ncomp * by);
      off = j - (f - 2) * ncomp * by;
      q = off / by;
      t = off - q * by;
    }
    int row, col;
    if (f == 0) {        // S
      row = dir ? 0 : 1;
      col = t + 1;
    } else if (f == 1) { // N
      row = dir ? by + 1 : by;
      col = t + 1;
    } else if (f == 2) { // W
      row = t + 1;
      col = dir ? 0 : 1;
    } else {             // E
      row = t + 1;
      col = dir ? bx + 1 : bx;
    }
    double* cell = ypad + q * pplane + (size_t)row * px + col;
    if (dir)
      *cell = buf[i];
    else
      buf[i] = *cell;
  }
}

// Interior of a padded block from the SplitMix64 stream by GLOBAL index
// (species-major, then row, then column of the global gnx x gny grid), the
// power iteration's start vector restricted to the block.
__global__ void k_block_splitmix(int bx, int by, int ncomp, int gnx, int gny, int x0, int y0, uint64_t seed,
                                 double* ypad) {
  const int px = bx + 2;
  const size_t pplane = (size_t)px * (by + 2), plane = (size_t)bx * by;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane * ncomp;
       i += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / plane);
    const size_t r = i - (size_t)q * plane;
    const int x = (int)(r % bx), y = (int)(r / bx);
    const uint64_t g = (uint64_t)q * gnx * gny + (uint64_t)(y0 + y) * gnx + (uint64_t)(x0 + x);
    ypad[q * pplane + (size_t)(y + 1) * px + (x + 1)] = splitmix_uniform(seed, g);
  }
}

}  // namespace

cudaError_t launch_block_newton(int kind, int bx, int by, int ncomp, int K, const double* yin, double* yout,
                                double* const* p, const double* st, const double* k8, const double* dk,
                                double a, double b, double* partials, unsigned int* counter, double* norms,
                                int grid, cudaStream_t s) {
  BlockArgs A{};
  A.bx = bx;
  A.by = by;
  A.ncomp = ncomp;
  A.K = K;
  A.init = yout == nullptr;
  A.yin = yin;
  A.yout = yout;
  for (int k = 0; k < KMAX; ++k) {
    A.p[k] = k < K ? p[k] : nullptr;
    A.dk[k] = k < K ? dk[k] : 0.0;
  }
  A.st = st;
  for (int j = 0; j < 8; ++j) A.k[j] = k8[j];
  A.a = a;
  A.b = b;
  A.partials = partials;
  A.counter = counter;
  A.norms = norms;
  const size_t plane = (size_t)bx * by;
  const int g = (int)std::max<size_t>(1, std::min<size_t>((size_t)grid, (plane + BT - 1) / BT));
  if (kind == PHIX_OP_ADVDIFF)
    k_block_newton<PHIX_OP_ADVDIFF><<<g, BT, 0, s>>>(A);
  else if (kind == PHIX_OP_GRAYSCOTT)
    k_block_newton<PHIX_OP_GRAYSCOTT><<<g, BT, 0, s>>>(A);
  else
    k_block_newton<PHIX_OP_BURGERS><<<g, BT, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_block_faces(int bx, int by, int ncomp, int dir, double* ypad, double* buf, cudaStream_t s) {
  const int total = ncomp * (2 * bx + 2 * by);
  const int g = std::max(1, std::min(1024, (total + 255) / 256));
  k_block_faces<<<g, 256, 0, s>>>(bx, by, ncomp, dir, ypad, buf);
  return cudaGetLastError();
}

cudaError_t launch_block_splitmix(int bx, int by, int ncomp, int gnx, int gny, int x0, int y0, uint64_t seed,
                                  double* ypad, int grid, cudaStream_t s) {
  const size_t n = (size_t)bx * by * ncomp;
  const int g = (int)std::max<size_t>(1, std::min<size_t>((size_t)grid, (n + 255) / 256));
  k_block_splitmix<<<g, 256, 0, s>>>(bx, by, ncomp, gnx, gny, x0, y0, seed, ypad);
  return cudaGetLastError();
}

}  // namespace phix
