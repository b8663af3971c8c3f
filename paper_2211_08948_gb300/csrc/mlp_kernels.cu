// Learned spectral interval: state features and the MLP 16 -> 64 -> 64 -> 3
// (GELU), bfloat16 weights with float32 accumulation, trained with Adam on
// float32 master weights.  Hand-written CUDA-core kernels: the network has
// 5443 parameters and ~5.3k FMAs per sample, far too small for tensor cores.
//
// Parameter layout (float32): W1[64x16] b1[64] W2[64x64] b2[64] W3[3x64] b3[3].
// Loss per sample: sum_j w_j (y_j - t_j)^2, w_0 = 4 when y_0 < t_0 (an
// under-estimated spectral radius is the dangerous side), batch mean.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "iter_common.cuh"

namespace phix {

namespace {

constexpr int H1 = 64, H2 = 64, NI = 16, NO = 3;
constexpr int OW1 = 0, OB1 = OW1 + H1 * NI, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1, OW3 = OB2 + H2,
              OB3 = OW3 + NO * H2, NP = OB3 + NO;  // 5443

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// weights rounded to bfloat16 (kept as bf16 in shared memory, indexed by
// parameter offset; bias slots unused), biases float32 in b[]
constexpr int NB = H1 + H2 + NO;
__host__ __device__ constexpr int bias_slot(int off) {
  return off < OW2 ? off - OB1 : (off < OW3 ? H1 + off - OB2 : H1 + H2 + off - OB3);
}
struct Net {
  __nv_bfloat16 w[OB3];
  float b[NB];
};

__device__ void load_net(const float* __restrict__ p, Net& n, int tid, int nthr) {
  for (int i = tid; i < NP; i += nthr) {
    const bool is_b = (i >= OB1 && i < OW2) || (i >= OB2 && i < OW3) || i >= OB3;
    if (is_b)
      n.b[bias_slot(i)] = p[i];
    else
      n.w[i] = __float2bfloat16_rn(p[i]);
  }
  __syncthreads();
}

__device__ __forceinline__ float wv(const Net& n, int i) { return __bfloat162float(n.w[i]); }
__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// one sample: x[16] -> y[3]; activations kept for the backward pass
__device__ void mlp_sample(const Net& n, const float* x, float* z1, float* a1, float* z2, float* a2, float* y) {
  for (int j = 0; j < H1; ++j) {
    float s = n.b[j];
#pragma unroll
    for (int i = 0; i < NI; ++i) s = fmaf(wv(n, OW1 + j * NI + i), x[i], s);
    z1[j] = s;
    a1[j] = gelu(s);
  }
  for (int j = 0; j < H2; ++j) {
    float s = n.b[H1 + j];
    for (int i = 0; i < H1; ++i) s = fmaf(wv(n, OW2 + j * H1 + i), a1[i], s);
    z2[j] = s;
    a2[j] = gelu(s);
  }
  for (int j = 0; j < NO; ++j) {
    float s = n.b[H1 + H2 + j];
    for (int i = 0; i < H2; ++i) s = fmaf(wv(n, OW3 + j * H2 + i), a2[i], s);
    y[j] = s;
  }
}

__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ p, const float* __restrict__ X, int n,
                                                 float* __restrict__ Y) {
  __shared__ Net net;
  load_net(p, net, threadIdx.x, blockDim.x);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[NI], z1[H1], a1[H1], z2[H2], a2[H2], y[NO];
  for (int i = 0; i < NI; ++i) x[i] = X[(size_t)s * NI + i];
  mlp_sample(net, x, z1, a1, z2, a2, y);
  for (int j = 0; j < NO; ++j) Y[(size_t)s * NO + j] = y[j];
}

// Inference of a few samples (the learned phi-action evaluates one): one CTA
// of 64 threads per sample, thread j owning hidden unit j of each layer and
// the activations in shared memory; weights read from global memory and
// rounded to bfloat16 as they are used.  Every unit's sum is the same fmaf
// chain as in mlp_sample (inputs in ascending order), so the outputs equal
// k_mlp_fwd's bit for bit.
__global__ void __launch_bounds__(64) k_mlp_fwd_unit(const float* __restrict__ p, const float* __restrict__ X,
                                                     float* __restrict__ Y) {
  __shared__ float x[NI], a1[H1], a2[H2];
  const int j = threadIdx.x, s = blockIdx.x;
  if (j < NI) x[j] = X[(size_t)s * NI + j];
  __syncthreads();
  float z = p[OB1 + j];
#pragma unroll
  for (int i = 0; i < NI; ++i) z = fmaf(bf16r(p[OW1 + j * NI + i]), x[i], z);
  a1[j] = gelu(z);
  __syncthreads();
  z = p[OB2 + j];
#pragma unroll 16
  for (int i = 0; i < H1; ++i) z = fmaf(bf16r(p[OW2 + j * H1 + i]), a1[i], z);
  a2[j] = gelu(z);
  __syncthreads();
  if (j < NO) {
    z = p[OB3 + j];
#pragma unroll 16
    for (int i = 0; i < H2; ++i) z = fmaf(bf16r(p[OW3 + j * H2 + i]), a2[i], z);
    Y[(size_t)s * NO + j] = z;
  }
}

// Gradient of the batch-mean loss over samples [0, n) of (X, T): one CTA of
// 256 threads, the batch in chunks of GC samples held in shared memory as
// row-major activation tiles (rows padded to 65 floats: a warp reading 32
// consecutive samples of one unit hits 32 banks).  Each layer is a small
// dense product done with warp-broadcast weights; each thread owns a fixed
// set of weight-gradient entries and accumulates them in registers over the
// whole batch (no atomics), so the sums run in one fixed order.
constexpr int GC = 64;            // samples per chunk
constexpr int LD = 65;            // padded row length of the activation tiles
constexpr int GT = 256;           // threads
struct GradSmem {
  float w1[H1 * NI];              // bf16-rounded weights as float32, natural layout W[j][i]
  float w2[H2 * H1];
  float w3[NO * H2];
  float b[NB];
  float x[GC * NI];
  float z1[GC * LD], a1[GC * LD], z2[GC * LD], a2[GC * LD];
  float dy[GC * 4];
  float red[GT / 32][NO + 1];
};

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__global__ void __launch_bounds__(GT) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                 const float* __restrict__ T, int n, float* __restrict__ G,
                                                 float* loss_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < H1 * NI; i += GT) S.w1[i] = bf(p[OW1 + i]);
  for (int i = tid; i < H2 * H1; i += GT) S.w2[i] = bf(p[OW2 + i]);
  for (int i = tid; i < NO * H2; i += GT) S.w3[i] = bf(p[OW3 + i]);
  for (int i = tid; i < H1; i += GT) S.b[i] = p[OB1 + i];
  for (int i = tid; i < H2; i += GT) S.b[H1 + i] = p[OB2 + i];
  if (tid < NO) S.b[H1 + H2 + tid] = p[OB3 + tid];
  // register accumulators: W2 entries e = tid + 256 q (16), W1 entries tid + 256 q (4),
  // W3 entry tid (tid < 192), b1 / b2 entry in gb (tid < 64 / 64 <= tid < 128), b3 in gb3 (tid < 3)
  float gw2[16], gw1[4], gw3 = 0.f, gb = 0.f, gb3 = 0.f, lacc = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) gw2[q] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) gw1[q] = 0.f;
  const float inv_n = 1.f / n;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += GC) {
    const int cn = min(GC, n - c0);
    for (int i = tid; i < GC * NI; i += GT) S.x[i] = (i / NI) < cn ? X[(size_t)c0 * NI + i] : 0.f;
    __syncthreads();
    // layer 1: thread -> sample s = lane + 32 (warp & 1), units j = (warp >> 1) + 4 r
    const int s = lane + 32 * (warp & 1);
    for (int r = 0; r < H1 / 4; ++r) {
      const int j = (warp >> 1) + 4 * r;
      float z = S.b[j];
#pragma unroll
      for (int i = 0; i < NI; ++i) z = fmaf(S.w1[j * NI + i], S.x[s * NI + i], z);
      S.z1[s * LD + j] = z;
      S.a1[s * LD + j] = gelu(z);
    }
    __syncthreads();
    for (int r = 0; r < H2 / 4; ++r) {
      const int j = (warp >> 1) + 4 * r;
      float z = S.b[H1 + j];
#pragma unroll 16
      for (int i = 0; i < H1; ++i) z = fmaf(S.w2[j * H1 + i], S.a1[s * LD + i], z);
      S.z2[s * LD + j] = z;
      S.a2[s * LD + j] = gelu(z);
    }
    __syncthreads();
    // outputs, loss and dL/dy (threads 0..GC-1, one sample each)
    if (tid < GC) {
      float l = 0.f;
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float y = S.b[H1 + H2 + j];
        for (int i = 0; i < H2; ++i) y = fmaf(S.w3[j * H2 + i], S.a2[tid * LD + i], y);
        float d = 0.f;
        if (tid < cn) {
          const float t = T[(size_t)(c0 + tid) * NO + j];
          const float e = y - t;
          const float w = (j == 0 && y < t) ? 4.f : 1.f;
          l += w * e * e;
          d = 2.f * w * e * inv_n;
        }
        S.dy[tid * 4 + j] = d;
      }
      lacc += l * inv_n;
    }
    __syncthreads();
    // dW3, db3
    if (tid < NO * H2) {
      const int j = tid / H2, i = tid % H2;
      for (int q = 0; q < GC; ++q) gw3 = fmaf(S.dy[q * 4 + j], S.a2[q * LD + i], gw3);
    }
    if (tid < NO)
      for (int q = 0; q < GC; ++q) gb3 += S.dy[q * 4 + tid];
    // dZ2 = (dY W3) * gelu'(Z2), in place of Z2
    for (int r = 0; r < H2 / 4; ++r) {
      const int j = (warp >> 1) + 4 * r;
      float d = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o) d = fmaf(S.dy[s * 4 + o], S.w3[o * H2 + j], d);
      S.z2[s * LD + j] = d * gelu_d(S.z2[s * LD + j]);
    }
    __syncthreads();
    // dW2[j][i] += sum_s dZ2[s][j] A1[s][i]  (entries e = tid + 256 q: j = e / 64, i = e % 64)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + GT * q, j = e / H1, i = e % H1;
      float acc = gw2[q];
      for (int t = 0; t < GC; ++t) acc = fmaf(S.z2[t * LD + j], S.a1[t * LD + i], acc);
      gw2[q] = acc;
    }
    if (tid >= H1 && tid < H1 + H2)
      for (int t = 0; t < GC; ++t) gb += S.z2[t * LD + tid - H1];
    __syncthreads();
    // dZ1 = (dZ2 W2) * gelu'(Z1), into the A1 tile (A1 is no longer needed)
    for (int r = 0; r < H1 / 4; ++r) {
      const int i = (warp >> 1) + 4 * r;
      float d = 0.f;
#pragma unroll 16
      for (int j = 0; j < H2; ++j) d = fmaf(S.z2[s * LD + j], S.w2[j * H1 + i], d);
      S.a1[s * LD + i] = d * gelu_d(S.z1[s * LD + i]);
    }
    __syncthreads();
    // dW1[j][i] += sum_s dZ1[s][j] X[s][i] (entries e = tid + 256 q: j = e / 16, i = e % 16), db1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + GT * q, j = e / NI, i = e % NI;
      float acc = gw1[q];
      for (int t = 0; t < GC; ++t) acc = fmaf(S.a1[t * LD + j], S.x[t * NI + i], acc);
      gw1[q] = acc;
    }
    if (tid < H1)
      for (int t = 0; t < GC; ++t) gb += S.a1[t * LD + tid];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) G[OW2 + tid + GT * q] = gw2[q];
#pragma unroll
  for (int q = 0; q < 4; ++q) G[OW1 + tid + GT * q] = gw1[q];
  if (tid < NO * H2) G[OW3 + tid] = gw3;
  if (tid < H1) G[OB1 + tid] = gb;
  if (tid >= H1 && tid < H1 + H2) G[OB2 + tid - H1] = gb;
  if (tid < NO) G[OB3 + tid] = gb3;
  // batch loss: threads 0..GC-1 hold their samples' terms
  for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
  if (lane == 0) S.red[warp][0] = lacc;
  __syncthreads();
  if (tid == 0 && loss_out) {
    float l = 0.f;
    for (int w = 0; w < GT / 32; ++w) l += S.red[w][0];
    *loss_out = l;
  }
}

// Adam (Kingma & Ba 2015) on the float32 master weights; step counts from 1
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int step, float lr) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---- state features (grid reduction) --------------------------------------
// partial slots: 0 max|s1| 1 max|s2| 2 sum|s1| 3 max g 4 sum g 5 max V^2 6 max 2UV
//                7 max|div U| (Burgers)
constexpr int NF = 8;
// Reduce a[NF] over the block (slots 2 and 4 summed, the rest by max); the
// result is left in sr[0][0..NF).
__device__ void feat_block_reduce(const double* a, double (*sr)[NF]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < NF; ++j) {
    double x = a[j];
    const bool is_sum = (j == 2 || j == 4);
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = is_sum ? x + y : fmax(x, y);
    }
    if (lane == 0) sr[warp][j] = x;
  }
  __syncthreads();
  if (tid < NF) {
    const bool is_sum = (tid == 2 || tid == 4);
    double x = sr[0][tid];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = is_sum ? x + sr[w][tid] : fmax(x, sr[w][tid]);
    sr[0][tid] = x;
  }
  __syncthreads();
}

// the operator and step features, computed on the host in float64
struct FConst {
  float f[16];
};

__global__ void __launch_bounds__(256) k_features(int kind, int nx, int ny, float rho_diff, FConst fconst,
                                                  const double* __restrict__ st, double* partials,
                                                  unsigned int* counter, float* feats) {
  __shared__ double sr[8][NF];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const size_t N = (size_t)nx * ny;
  // per point: the centred differences in float64 (differences of close
  // values), then float32 (the features are float32; rounding is monotone,
  // so the maximum of the rounded values is the rounded maximum); the sums
  // of the two means in float32 per thread (a few points each), float64
  // across threads and blocks
  float mx[NF];
  float sm2 = 0.f, sm4 = 0.f;
  for (int j = 0; j < NF; ++j) mx[j] = 0.f;
  for (int r = blockIdx.x; r < ny; r += gridDim.x) {
    const size_t row = (size_t)r * nx;
    const size_t rowm = (size_t)(r == 0 ? ny - 1 : r - 1) * nx, rowp = (size_t)(r == ny - 1 ? 0 : r + 1) * nx;
    for (int c = tid; c < nx; c += blockDim.x) {
      const int cm = c == 0 ? nx - 1 : c - 1, cp = c == nx - 1 ? 0 : c + 1;
      const double s1 = st[row + c];
      const double dx = st[row + cp] - st[row + cm];
      const double dy = st[rowp + c] - st[rowm + c];
      const float as1 = fabsf((float)s1);
      const float g = 0.5f * (fabsf((float)dx) + fabsf((float)dy));
      mx[0] = fmaxf(mx[0], as1);
      sm2 += as1;
      mx[3] = fmaxf(mx[3], g);
      sm4 += g;
      if (kind == PHIX_OP_GRAYSCOTT) {
        const float s2 = (float)st[N + row + c];
        const float s1f = (float)s1;
        mx[1] = fmaxf(mx[1], fabsf(s2));
        mx[5] = fmaxf(mx[5], s2 * s2);
        mx[6] = fmaxf(mx[6], 2.f * s1f * s2);
      } else {
        mx[7] = fmaxf(mx[7], fabsf((float)(0.5 * (dx * nx + dy * ny))));
      }
    }
  }
  double a[NF];
  for (int j = 0; j < NF; ++j) a[j] = mx[j];
  a[2] = sm2;
  a[4] = sm4;
  // block reduction: max slots by max, slots 2 and 4 by sum
  feat_block_reduce(a, sr);
  if (tid < NF) partials[(size_t)blockIdx.x * NF + tid] = sr[0][tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  // the last block folds the per-block partials, all its threads at once
  for (int j = 0; j < NF; ++j) a[j] = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += blockDim.x)
    for (int j = 0; j < NF; ++j) {
      const double x = __ldcg(partials + (size_t)b * NF + j);
      a[j] = (j == 2 || j == 4) ? a[j] + x : fmax(a[j], x);
    }
  __syncthreads();
  feat_block_reduce(a, sr);
  if (tid < 16) {
    // the operator and step features (host-computed) and the state's
    float f = fconst.f[tid];
    const double* t = sr[0];
    switch (tid) {
      case 5: f = (float)t[0]; break;
      case 6: f = (float)t[1]; break;
      case 7: f = (float)(t[2] / (double)N); break;
      case 8: f = (float)t[3]; break;
      case 9: f = (float)(t[4] / (double)N); break;
      case 10: f = kind == PHIX_OP_GRAYSCOTT ? (float)t[5] : (float)t[7] / rho_diff; break;
      case 11: f = kind == PHIX_OP_GRAYSCOTT ? (float)t[6] : 0.f; break;
      case 12: f = kind == PHIX_OP_GRAYSCOTT ? 0.f : (float)t[0] * (float)(nx + ny) / rho_diff; break;
      default: break;
    }
    feats[tid] = f;
  }
  if (tid == 0) {
    *counter = 0;
    __threadfence();
  }
}

// *out = max_i |x_i| (out zeroed by the caller): block maxima, then one
// atomicMax per block on the bit patterns (non-negative doubles order as
// their unsigned 64-bit patterns), independent of the block order.
__global__ void __launch_bounds__(256) k_maxabs(const double* __restrict__ x, size_t n, unsigned long long* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double sw[8];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, sw[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

}  // namespace

int mlp_nparam() { return NP; }

cudaError_t launch_mlp_forward(const float* p, const float* X, int n, float* Y, cudaStream_t st) {
  if (n <= 256)
    k_mlp_fwd_unit<<<n, H1, 0, st>>>(p, X, Y);
  else
    k_mlp_fwd<<<(n + 127) / 128, 128, 0, st>>>(p, X, n, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* p, const float* X, const float* T, int n, float* G, float* loss,
                            cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem));
  if (e != cudaSuccess) return e;
  k_mlp_grad<<<1, GT, sizeof(GradSmem), st>>>(p, X, T, n, G, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int step, float lr, cudaStream_t st) {
  k_adam<<<(NP + 255) / 256, 256, 0, st>>>(p, m, v, g, step, lr);
  return cudaGetLastError();
}

cudaError_t launch_maxabs(const double* x, size_t n, double* out, int grid, cudaStream_t st) {
  k_maxabs<<<grid, 256, 0, st>>>(x, n, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

cudaError_t launch_features(int kind, int nx, int ny, const double* prm, double h, const double* state,
                            double* partials, unsigned int* counter, float* feats, int grid, cudaStream_t st) {
  // features that depend on the operator and the step only, computed here in
  // float64 and passed in the kernel's argument block
  FConst fc{};
  const double Dmax = kind == PHIX_OP_GRAYSCOTT ? std::max(prm[0], prm[1]) : prm[0];
  const double rho_diff = 4.0 * Dmax * ((double)nx * nx + (double)ny * ny);
  fc.f[0] = kind == PHIX_OP_GRAYSCOTT ? 1.f : 0.f;
  fc.f[1] = (float)(std::log((double)nx * ny) / 10.0);
  fc.f[2] = (float)(std::log(Dmax) / 10.0);
  fc.f[3] = (float)(std::log(h) / 10.0);
  fc.f[4] = (float)(std::log(h * rho_diff) / 5.0);
  if (kind == PHIX_OP_GRAYSCOTT) {
    fc.f[13] = (float)prm[2];
    fc.f[14] = (float)prm[3];
  }
  fc.f[15] = 1.f;
  k_features<<<grid, 256, 0, st>>>(kind, nx, ny, (float)rho_diff, fc, state, partials, counter, feats);
  return cudaGetLastError();
}

}  // namespace phix
