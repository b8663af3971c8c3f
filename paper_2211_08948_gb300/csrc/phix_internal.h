// Internal declarations shared by the host driver and the kernel files.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "df64.cuh"
#include "phix.h"

#include <vector>

namespace phix {

constexpr int KMAX = 4;       // accumulators of one vertical Newton pass
constexpr int TILE_Y = 8;     // rows per tile (one warp per row)
constexpr int THREADS = 256;  // 32 x 8
constexpr int UNR = 4;        // elements per thread whose loads a streaming kernel issues together

enum Prec { P_FP64 = 0, P_DF64 = 1, P_FP32JV = 2, P_FP32 = 3 };
enum Mode { MODE_NEWTON = 0, MODE_POWER = 1 };

// Device-resident control block of one chain of iteration launches.  The
// last block of each launch reduces the per-block partial sums in a fixed
// order, takes the stop decision and sets `done`; later launches of the
// chain read `done` and return at once, so the host may enqueue more
// launches than needed without reading anything back.
struct LejaCtl {
  unsigned int count;  // arrival counter of the last-block reduction (reset by the last block)
  int done;            // 1: converged or failed
  int iters;           // iteration index m at which the chain stopped
  int status;          // phix_status
  int m;               // index of the next iteration of the chain (advanced by the last block)
  int sigma_e;         // sigma = 2^sigma_e
  double ysq;          // ||y_m||^2 (scaled units) of the last completed launch
  double psq[KMAX];    // ||p_m^(k)||^2
  double sigma;        // input scale, a power of two
  double inv_sigma;
  double rho;          // power iteration: ||J v_k||
  double rho_prev;
  double alpha;        // power iteration: 1/||y_k|| for the next launch
  float alpha_hi, alpha_lo;
  unsigned int bar_count, bar_gen;  // grid barrier of a persistent chain (zero at its start)
};

// Parameters of one chain of iteration launches, in device memory, written by
// the host before the chain.  Every launch of a chain then has the same
// arguments (so a chain can be replayed as a CUDA graph): the kernel reads its
// iteration index m from the control block and its shift beta_m and
// coefficients d_k[m] from the tables that follow this header:
//   PassParams | beta_d[M] | beta_f[M] | dk_d[KMAX][M] | dk_f[KMAX][M]
// (float64 forms and double-float (hi, lo) forms; float32 kernels use .x).
// Uniform J coefficients k:
//   ADVDIFF:   {E, W, N, S, C}
//   GRAYSCOTT: {xu, yu, Cu, xv, yv, Cv}, per-point terms g1 = V^2, g2 = 2UV
//   BURGERS:   {x, y, C, bx, by},        per-point state U
// In MODE_NEWTON the host folds alpha = 1/gamma into k and ga; beta_m =
// -(c/gamma + xi_{m-1}) shifts the centre value.
struct PassParams {
  int K, m_min, m_max, M;
  int prescaled, pad;  // 1: the state planes already carry the factor ga (Gray-Scott Newton passes)
  double tol, rel;
  double kd[8], gad;
  float2 kf[8], gaf;
};
// Bytes of a parameter block with tables of M entries (the layout above plus
// the stop-test table q_k[m] = (d_k[m]/tol)^2 as double-float pairs).
constexpr size_t ptab_bytes(int M) {
  return sizeof(PassParams) + 16 * (size_t)M + 24 * (size_t)KMAX * (size_t)M;
}
// Fill a host copy of a parameter block.  beta and dk may be NULL (power iteration).
void ptab_fill(void* host, int K, int m_min, int m_max, double tol, double rel, const double* k8,
               double ga, const double* beta, const double* const* dk, int prescaled = 0);

// ---- launchers (leja_kernels.cu) -----------------------------------------
struct ChainSpec {
  int prec, op, mode, nx, ny;
  void* y[2];         // Newton basis / power iterate ping-pong: launch m reads y[(m-1)&1]
  void* p[KMAX];
  const void* st;     // per-point state planes (precision's state type)
  LejaCtl* ctl;
  double* partials;   // grid * (KMAX + 1)
  const void* ptab;   // parameter block (device)
  int grid;           // blocks (<= partials capacity)
  int K;              // MODE_NEWTON: accumulators
  int tma;            // MODE_NEWTON: 1 = the TMA-staged kernel (leja_tma.cu)
  int fused2;         // MODE_NEWTON: 1 = two iterations per launch (leja_fused.cu)
  int use_cond;       // launched as the body of a conditional WHILE graph node:
  unsigned long long cond;  // its handle; the kernel clears it once the chain stopped
  int prefix;         // graph chains: launches queued ahead of the WHILE node (no condition
                      // evaluations; a launch after the stop returns at once and clears the condition)
};
// One iteration launch.
cudaError_t launch_iter(const ChainSpec& s, cudaStream_t st);
// Kernel node of one iteration launch, for graph building.
cudaError_t iter_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage,
                             size_t arg_bytes);
// Blocks per SM the iteration kernel of this spec can keep resident.
int iter_blocks_per_sm(const ChainSpec& s);
// TMA-staged Newton step (leja_tma.cu): applicable when the rows are 16-byte
// multiples and the staging fits; persistent CTAs, four per SM
bool tma_eligible(const ChainSpec& s);
int tma_grid(const ChainSpec& s, int nsm);
cudaError_t tma_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage, size_t arg_bytes);
size_t tma_arg_bytes();
int iter_tiles(const ChainSpec& s);  // tiles of one launch (work units of the grid loop)
// Two Newton iterations per launch (leja_fused.cu): grids whose sides are
// multiples of 64 x 16; the launch starting at iteration m stores y_{m+1}
// and p_m and leaves d_k[m+1] y_{m+1} to the next launch or to the output
// conversion (launch_finalize with a FusedOut); partials: two halves of
// grid * (KMAX + 1).
bool fused2_eligible(const ChainSpec& s);
int fused2_tiles(const ChainSpec& s);
int fused2_blocks_per_sm(const ChainSpec& s);
cudaError_t fused2_node_params(const ChainSpec& s, cudaKernelNodeParams* np, void* arg_storage, size_t arg_bytes);
// Persistent chain (MODE_NEWTON, single-step kernel): every iteration of the
// pass in one cooperative launch of chain_grid() blocks (all resident), one
// grid barrier per iteration; s.partials must hold 2 * grid * (KMAX + 1).
int chain_grid(const ChainSpec& s, int nsm);  // 0 if the kernel cannot be resident
cudaError_t launch_chain(const ChainSpec& s, cudaStream_t st);

// y0 = v / sigma (stored in the precision's format), p_k = d_k[0] y0, norms, ctl->m = 1.
struct InitLaunch {
  int prec, ncomp, nx, ny;
  const double* v;
  void* y0;
  void* p[KMAX];
  LejaCtl* ctl;
  double* partials;
  const void* ptab;
  int grid;
};
cudaError_t launch_init(const InitLaunch& L, cudaStream_t s);

// ctl->sigma = 2^round(log2(rms(v))), ctl cleared.
cudaError_t launch_scale(const double* v, size_t n, LejaCtl* ctl, double* partials, int grid,
                         cudaStream_t s);

struct PtrPack {
  const void* p[KMAX];
  double* o[KMAX];
};
// A chain of two-iteration launches that stopped at an even iteration m >= 2
// left d_k[m] y_m out of the accumulators: y_m is in y[(m/2) & 1], d_k[m] in
// the pass's parameter block.
struct FusedOut {
  const void* y[2];
  const void* ptab;
};
// out_k = sigma * p_k (float64); p and out are HOST arrays of K device
// pointers; fo (NULL: none) adds the term a two-iteration chain deferred
cudaError_t launch_finalize(int prec, size_t n, int K, void* const* p, double* const* out,
                            const LejaCtl* ctl, int grid, cudaStream_t s, const FusedOut* fo = nullptr);

// power iteration start: y0[i] = splitmix64_uniform(seed, i) in the precision's format,
// ctl->alpha = 1/||y0||, ctl->m = 1.
cudaError_t launch_power_start(int prec, size_t n, uint64_t seed, void* y0, LejaCtl* ctl,
                               double* partials, int grid, cudaStream_t s);

// Per-point state arrays of the Jacobian in the precision's format:
// GRAYSCOTT: st = [V^2 plane, 2UV plane]; BURGERS: st = [U plane].
cudaError_t launch_prep_state(int prec, int op, int nx, int ny, const double* state, void* st,
                              int grid, cudaStream_t s, double scale = 1.0);

// ---- KIOPS-style Krylov kernels (kiops_kernels.cu) -----------------------
constexpr int KIOPS_MMAX = 128;  // largest Krylov dimension
constexpr int KIOPS_PMAX = 8;    // largest p (augmented tail length)

// Device control block of one KIOPS run.  The basis is kept unnormalised:
// V_i = s[i] * Zhat_i (N part in the iteration precision, tail in float64).
// The last block of each Arnoldi pass does the scalar work and prepares the
// coefficients of the next launch, so the host only reads `omega` & co.
struct KiopsCtl {
  // --- read back by the host after each small exponential --------------------
  int stop;        // happy breakdown or NaN: later Arnoldi launches return at once
  int happy_m;     // basis size at a happy breakdown (0: none)
  int status;      // phix_status
  unsigned int count;
  double omega, err, beta;
  // --- device-side state -----------------------------------------------------
  double eta;
  double s[KIOPS_MMAX + 2];
  float2 sf[KIOPS_MMAX + 2];
  double hd[KIOPS_MMAX + 2];   // h_{j,j}
  double hu[KIOPS_MMAX + 2];   // h_{j-1,j}
  double hl[KIOPS_MMAX + 2];   // h_{j+1,j}
  double z0[KIOPS_MMAX + 2];   // ||A~ V_j|| before orthogonalisation
  double tail[(KIOPS_MMAX + 2) * KIOPS_PMAX];
  double F[KIOPS_MMAX + 2];
  double coef[KIOPS_MMAX + 2];  // beta * F_i * s_i
  float2 coeff[KIOPS_MMAX + 2];
  // coefficients of the next pass-1 launch: k (x h s_j), ga, b-column weights
  double kd[8], gad, bd[KIOPS_PMAX];
  float2 kf[8], gaf, bf[KIOPS_PMAX];
  // coefficients of the next pass-2 launch: z' = z - c1 Zhat_j - c0 Zhat_{j-1}
  double c1d, c0d;
  float2 c1f, c0f;
  // fused steps: Zhat_{j+1} = ws W - c1 Zhat_j - c0 Zhat_{j-1}, then
  // u = A~ [Zhat_{j+1}; tail_{j+1}] unscaled (k h, ga = h, b-column weights eta tail_{j+1})
  double wsd;
  float2 wsf;
  double kud[8], gud, bud[KIOPS_PMAX];
  float2 kuf[8], guf, buf[KIOPS_PMAX];
};
constexpr size_t KIOPS_HOST_BYTES = 40;  // leading fields the host reads back
// Host-mapped (zero-copy) mailbox of the substep decision: the small
// exponential's kernel copies the header fields there, then publishes `seq`
// (system-scope fence in between); the host polls `seq` instead of a copy
// and a stream synchronisation.
struct KiopsMailbox {
  unsigned char header[KIOPS_HOST_BYTES];
  volatile unsigned int seq;
};

struct KiopsSpec {
  int prec, op, nx, ny, p;
  int nb;                       // nonzero b_j, j >= 1 (converted copies in bz[])
  int bslot[KIOPS_PMAX];        // tail index t of each nonzero b (b_{p-t})
  const void* bz[KIOPS_PMAX];   // their copies in the iteration precision
  void* const* Z;               // device array of basis slot pointers (host copy in Zh)
  void* Zh[KIOPS_MMAX + 2];
  const void* st;               // Jacobian state planes
  KiopsCtl* kc;
  double* partials;
  double h;                     // A = h J
  double kJ[8];                 // unscaled uniform J coefficients
  double prm[8];                // operator parameters (general operators: the no-flow problems,
                                // float64 only, st = the raw state)
  int nscaled;
  int grid;                     // streaming kernels (combine, start)
  int nsm;                      // SMs (the Arnoldi kernels size their grids by occupancy)
  void* W[2];                   // fused steps: scratch vectors (pass-1 results)
};
// w_0 = c [b_0; e_p / eta] (c a power of two): Zhat_0 = c b_0 (or 0), tail_0 = c e_p / eta,
// s_0 = 1/||w_0||, next pass-1 coefficients.
cudaError_t kiops_start(const KiopsSpec& s, const double* b0, double eta, double cscale, cudaStream_t st);
// Convert b (float64) into the iteration precision (out may be NULL: norm only); its 1-norm -> *norm1.
cudaError_t kiops_convert(int prec, size_t n, const double* b, void* out, double* partials,
                          unsigned int* counter, double* norm1, int grid, cudaStream_t st);
// Arnoldi step j: pass 1 (z = A~ V_j, dots) and pass 2 (orthogonalise, norm).
cudaError_t kiops_arnoldi(const KiopsSpec& s, int j, cudaStream_t st);
// Fused Arnoldi steps on tile-aligned grids: kiops_fused_first(s) runs pass 1 of
// step 0 into the scratch vector W0; kiops_fused_step(s, j) completes step j
// (Zhat_{j+1} from W, its norm) and runs pass 1 of step j + 1 (u = A~ Zhat_{j+1}
// into the other scratch vector, its dot products).  W0/W1 alternate.
bool kiops_fused_ok(const KiopsSpec& s);
cudaError_t kiops_fused_first(const KiopsSpec& s, cudaStream_t st);
cudaError_t kiops_fused_step(const KiopsSpec& s, int j, cudaStream_t st);
// F = exp(tau Hbar) e_1 (n = m+1, or m after a happy breakdown), err, omega.
// mbox (device address of a host-mapped KiopsMailbox, or NULL): receives the
// header and then seq
cudaError_t kiops_smallexp(KiopsCtl* kc, int m, double tau, double tau_end, double tol, KiopsMailbox* mbox,
                           unsigned int seq, cudaStream_t st);
// out = exp(tau T) e_1 for a tridiagonal T (device arrays d[n], u[n-1], l[n-1]); mode: 0 Chebyshev, 1 Taylor
cudaError_t small_expm_e1(int n, const double* d, const double* u, const double* l, double tau, double* out,
                          int* mode, cudaStream_t st);
// w = sum_{i<n} coef_i Zhat_i into slot 0, s_0 = 1/||w||; out (float64, may be NULL) = scale * w_N.
cudaError_t kiops_combine(const KiopsSpec& s, int n, double* out, double scale, cudaStream_t st);

// ---- batched persistent kernel (batched_kernels.cu) -------------------------
size_t batched_prob_bytes();
void batched_fill_prob(void* dst, int nx, int ny, double D, double ax, double ay, double h, double rho_re,
                       double rho_hi, double rho_im, const double* v, double* const* out, int nout,
                       unsigned long long ws_off);
void batched_read_prob(const void* src, int* status, int* iters, int* substeps);
// bt: threads per CTA (256, 512 or 1024); smem_bytes: dynamic shared memory per CTA (a
// vertical pass whose basis pair and accumulators fit in it runs there)
cudaError_t launch_batched(int prec, void* probs, const int* order, int nprob, unsigned int* queue, void* ws,
                           const double* xi, int m_max, int m_min, double tol, double gamma_cap, double iota_cap,
                           int nout, const int* l, int grid, int bt, unsigned int smem_bytes, cudaStream_t st);
int batched_blocks_per_sm(int prec, int bt, unsigned int smem_bytes);  // 0: not launchable

// ---- learned spectral interval (mlp_kernels.cu) ---------------------------
int mlp_nparam();
cudaError_t launch_mlp_forward(const float* p, const float* X, int n, float* Y, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* p, const float* X, const float* T, int n, float* G, float* loss,
                            cudaStream_t st);
cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int step, float lr, cudaStream_t st);
// *out = max |x_i| (*out zeroed by the caller; device pointers)
cudaError_t launch_maxabs(const double* x, size_t n, double* out, int grid, cudaStream_t st);
cudaError_t launch_features(int kind, int nx, int ny, const double* prm, double h, const double* state,
                            double* partials, unsigned int* counter, float* feats, int grid, cudaStream_t st);

// ---- float64 stage kernels (stage_kernels.cu) -----------------------------
struct OpDesc {
  int kind, nx, ny;
  double p[8];
};
// f = f(u)
cudaError_t launch_rhs(const OpDesc& op, const double* u, double* f, int grid, cudaStream_t s);
// R = f(a) - fu - J(u)(a - u)
cudaError_t launch_remainder(const OpDesc& op, const double* u, const double* a, double* R, int grid,
                             cudaStream_t s);
// out = alpha * J(state) x + beta * v   (v may be NULL)
cudaError_t launch_jv_axpy(const OpDesc& op, const double* state, const double* x, double alpha,
                           const double* v, double beta, double* out, int grid, cudaStream_t s);
// out = sum_i c[i] * x[i], i < nterms <= 6 (x[i] may alias out)
cudaError_t launch_lincomb(size_t n, int nterms, const double* c, const double* const* x,
                           double* out, int grid, cudaStream_t s);
// result[0] = ||x - y||_2^2 (y may be NULL) -> device double via last-block reduction
cudaError_t launch_norm2(size_t n, const double* x, const double* y, double* partials,
                         unsigned int* counter, double* result, int grid, cudaStream_t s);

// ---- domain-decomposed Newton-Leja pass (block_kernels.cu) ----------------
// padded block (bx + 2) x (by + 2) per species; yout == NULL: p_k = dk[k] yin
// (interior) and norms of yin; else yout = a J yin + b yin, p_k += dk[k] yout.
// norms[0..K] = ||y||^2, ||p_k||^2 over the block interior (device).
cudaError_t launch_block_newton(int kind, int bx, int by, int ncomp, int K, const double* yin, double* yout,
                                double* const* p, const double* st, const double* k8, const double* dk,
                                double a, double b, double* partials, unsigned int* counter, double* norms,
                                int grid, cudaStream_t s);
// dir 0: interior faces -> buf; dir 1: buf -> halo faces ([S | N | W | E], species contiguous per face)
cudaError_t launch_block_faces(int bx, int by, int ncomp, int dir, double* ypad, double* buf, cudaStream_t s);
// interior of a padded block <- SplitMix64 stream by global index
cudaError_t launch_block_splitmix(int bx, int by, int ncomp, int gnx, int gny, int x0, int y0, uint64_t seed,
                                  double* ypad, int grid, cudaStream_t s);

// ---- general float64 Newton / power step (general_kernels.cu) -------------
// mode 0 Newton, 1 power, 2 init; tab: gen_table_doubles(M) doubles (device)
size_t gen_table_doubles(int M);
cudaError_t launch_general(int mode, int kind, int nx, int ny, int K, const double* v, double* const* y,
                           double* const* p, const double* st, const double* fu, double fd_scale, int fd,
                           const double* prm, const double* const* src, int nsrc, LejaCtl* ctl, double* partials,
                           const double* tab, int grid, cudaStream_t s);

// ---- host math (host_math.cpp) --------------------------------------------
double phi_host(int l, double z);
int leja_points_host(double* xi, int m);                 // 0 on success
const double* leja_table(int m);                         // cached, thread-safe
void divided_differences_host(const double* x, double* f, int n);

// Newton divided differences d_i = f[x_0, ..., x_i] of f(x) = phi_l(a + b x)
// on the Leja points, built one point at a time (O(n) per point): appending
// x_n forms f[x_{n-k}, ..., x_n] for k = 1..n from the previous point's
// diagonal.  Every entry comes from the same two operands and the same
// formula as in the column-by-column recursion, so a table grown to n points
// equals, bit for bit, the first n entries of any longer table.
struct DDTable {
  int l = 0;
  double a = 0.0, b = 0.0;
  std::vector<double> d;     // d[i] = f[x_0, ..., x_i]
  std::vector<double> diag;  // diag[k] = f[x_{n-1-k}, ..., x_{n-1}], n = d.size()
  void grow(int n);          // extend to n points (n <= 4096)
};
}  // namespace phix
