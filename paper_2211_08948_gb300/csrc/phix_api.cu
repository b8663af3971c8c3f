// Host driver and C-ABI entry points of libphix (declared in include/phix.h).
//
// A phi-action call: validate -> Jacobian state arrays -> spectral interval
// (caller value or power iteration, Sec. 2.2) -> divided-difference tables
// (host, float64) -> chains of Newton-Leja launches that stop themselves on
// the device (a conditional WHILE graph node per chain; the host reads the
// chains' control blocks once per call) -> outputs scaled back to float64.  EXPRB43 / EPIRK4s3 steps chain these actions with
// float64 stage kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <string>
#include <vector>

#include "phix_internal.h"

using namespace phix;

namespace {

enum Slot {
  S_Y0 = 0, S_Y1, S_P0, S_P1, S_P2, S_P3, S_ST,                 // Newton pass
  S_F, S_A, S_B, S_RA, S_RB, S_T0, S_Q, S_T3, S_T4, S_O1, S_O2, S_O3,  // stages
  S_SUB_U, S_SUB_TMP, S_SUB_W0,                                  // substeps (W0..W0+8)
  S_KBASIS = S_SUB_W0 + 9, S_KB, S_KPTR, S_KCTL, S_KMODE, S_KW,                 // KIOPS basis, b copies, slot table, control, scratch
  S_ST2,                                                         // Gray-Scott state planes scaled for Newton passes
  S_BPROB, S_BORDER, S_BWS, S_BQ, S_XI,                          // batched problems, order, arena, queue, Leja points
  S_MFEAT, S_MY, S_MG, S_MCNT,                                   // learned interval: features, outputs, gradient
  S_FH, S_O4, S_O5, S_O6, S_UH, S_UB,                            // stages: f h, more outputs, host-state copy, step backup
  S_GTAB, S_GCTL, S_GFU, S_GZ,                                   // general pass: table, control, f(u), zero state
  S_NSLOT
};

}  // namespace

static constexpr int NSLOT = 16;  // passes queued between synchronisations

struct phix_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 1;
  int grid_iter = 1;
  int grid_stream = 1;
  double l2_bytes = 0.0;
  std::string err;
  void* buf[S_NSLOT] = {};
  size_t cap[S_NSLOT] = {};
  LejaCtl* ctl = nullptr;        // device, one control block per slot
  LejaCtl* ctl_h = nullptr;      // pinned host mirror
  double* partials = nullptr;    // device, grid_iter * (KMAX+1)
  double* scal = nullptr;        // device scalars (norms)
  double* scal_h = nullptr;      // pinned
  unsigned int* counter = nullptr;
  long launches = 0;
  std::vector<cudaEvent_t> ev;   // profiling: one event pair per slot
  unsigned char* ptab_d = nullptr;  // chain parameter blocks, one per slot (device)
  unsigned char* ptab_h = nullptr;  // their pinned staging
  size_t ptab_slot = 0;             // bytes per slot
  struct Pending {
    int slot;
    phix_stats* stats;    // where the outcome goes (null: read by the caller)
    bool profile;
    double bytes_per_launch;
    int m_table;          // last iteration the pass's table covers
    int m_limit;          // the caller's m_max
    bool persistent;      // one cooperative launch ran the whole chain
    bool fused2;          // two iterations per launch
    int prefix;           // graph chain: launches ahead of its WHILE node
  };
  std::vector<Pending> pend;     // queued passes since the last flush
  int nslot = 0;                 // slots in use
  // divided-difference tables: truncated to about twice the predicted chain
  // length; a chain that reaches the end of its table without converging
  // sets ran_out, and the call is run again once with full tables
  bool full_tables = false;
  bool ran_out = false;
  // state planes scaled by the Newton factor: valid for one preparation of the
  // planes (prep_gen) and one factor
  unsigned long prep_gen = 0, st2_gen = ~0ul;
  double st2_alpha = 0.0;
  std::list<DDTable> dd_cache;   // recent tables (pure functions of l, a, b); references stay valid
  struct Graph {
    ChainSpec spec;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;     // cached chain graphs (WHILE loops of iteration launches)
  KiopsCtl* kc_h = nullptr;      // pinned mirror of the KIOPS control header
  KiopsMailbox* kmb_h = nullptr; // host-mapped decision mailbox (host address)
  KiopsMailbox* kmb_d = nullptr; // its device address
  unsigned int kmb_seq = 0;
  struct BatchGraph {
    unsigned long long key;
    int grid;
    cudaGraphExec_t exec;
  };
  std::vector<BatchGraph> bgraphs;  // batched launch graphs
  struct BatchCfg {
    int bt = 512;            // threads per CTA
    unsigned int smem = 0;   // dynamic shared memory per CTA (small passes run there)
    int per_sm = 2;          // CTAs per SM
  };
  std::vector<std::pair<unsigned long long, BatchCfg>> btune;  // tuned launch per batch shape
  BatchCfg blast;                   // the configuration of the last batched call
};

static constexpr int GRAPH_ITERS = 8;  // iteration launches per body of a chain's WHILE loop

namespace {

struct Fail {
  phix_status st;
};
struct Rerun {};  // a pass ran past its truncated table: repeat the call with full tables

void set_err(phix_ctx* c, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  c->err = b;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_err(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      throw Fail{PHIX_ECUDA};                                                     \
    }                                                                             \
  } while (0)

#define KL(call)          \
  do {                    \
    ctx->launches++;      \
    CK(call);             \
  } while (0)

[[noreturn]] void fail(phix_ctx* ctx, phix_status st, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  ctx->err = b;
  throw Fail{st};
}

void* ws(phix_ctx* ctx, int slot, size_t bytes) {
  if (ctx->cap[slot] < bytes) {
    if (ctx->buf[slot]) {
      CK(cudaStreamSynchronize(ctx->stream));
      CK(cudaFree(ctx->buf[slot]));
      ctx->buf[slot] = nullptr;
      ctx->cap[slot] = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->buf[slot], bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      fail(ctx, PHIX_ENOMEM, "workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->cap[slot] = bytes;
  }
  return ctx->buf[slot];
}
double* wsd(phix_ctx* ctx, int slot, size_t n) { return static_cast<double*>(ws(ctx, slot, n * sizeof(double))); }

int ncomp_of(int kind) { return (kind == PHIX_OP_GRAYSCOTT || kind == PHIX_OP_BRUSSELATOR) ? 2 : 1; }
// operators served by the general float64 kernel only (the no-flow problems)
bool general_kind(int kind) { return kind >= PHIX_OP_ADR; }

size_t elem_bytes(int prec) { return prec == P_FP32 ? 4 : 8; }

// Validated operator + its per-point state arrays in the iteration precision.
struct OpState {
  OpDesc d;
  int ncomp;
  size_t plane, N;
  const double* state;  // float64 state (caller memory)
  const void* st;       // prepared state arrays (workspace)
  double kJ[8];         // unscaled uniform J coefficients
};

void check_op(phix_ctx* ctx, const phix_jop* op, bool need_state) {
  if (!op) fail(ctx, PHIX_EINVAL, "op is NULL");
  if (op->kind < 0 || op->kind > PHIX_OP_BRUSSELATOR) fail(ctx, PHIX_EINVAL, "unknown operator kind %d", op->kind);
  if (op->nx < 3 || op->ny < 3) fail(ctx, PHIX_EINVAL, "grid %dx%d too small (>= 3 required)", op->nx, op->ny);
  if ((size_t)op->nx * op->ny > ((size_t)1 << 31)) fail(ctx, PHIX_EINVAL, "grid too large");
  if (need_state && op->kind != PHIX_OP_ADVDIFF && !op->state)
    fail(ctx, PHIX_EINVAL, "operator kind %d needs a state vector", op->kind);
}

// Uniform coefficients of the Jacobian's stencil on an nx x ny periodic grid
// of the unit square (dx = 1/nx, dy = 1/ny), Sec. 3 centred differences.
void uniform_coeffs(int kind, int nx, int ny, const double* p, double (&k)[8]) {
  const double idx2 = (double)nx * nx, idy2 = (double)ny * ny;
  for (double& x : k) x = 0.0;
  if (kind == PHIX_OP_ADVDIFF) {
    k[0] = p[0] * idx2 + 0.5 * p[1] * nx;  // E
    k[1] = p[0] * idx2 - 0.5 * p[1] * nx;  // W
    k[2] = p[0] * idy2 + 0.5 * p[2] * ny;  // N (y + 1)
    k[3] = p[0] * idy2 - 0.5 * p[2] * ny;  // S
    k[4] = -2.0 * p[0] * (idx2 + idy2);    // C
  } else if (kind == PHIX_OP_GRAYSCOTT) {
    k[0] = p[0] * idx2;
    k[1] = p[0] * idy2;
    k[2] = -2.0 * p[0] * (idx2 + idy2) - p[2];
    k[3] = p[1] * idx2;
    k[4] = p[1] * idy2;
    k[5] = -2.0 * p[1] * (idx2 + idy2) - (p[2] + p[3]);
  } else {
    k[0] = p[0] * idx2;
    k[1] = p[0] * idy2;
    k[2] = -2.0 * p[0] * (idx2 + idy2);
    k[3] = 0.5 * nx;
    k[4] = 0.5 * ny;
  }
}

OpState make_opstate(phix_ctx* ctx, const phix_jop* op, const double* state, int prec) {
  OpState s{};
  s.d.kind = op->kind;
  s.d.nx = op->nx;
  s.d.ny = op->ny;
  for (int i = 0; i < 8; ++i) s.d.p[i] = op->param[i];
  s.ncomp = ncomp_of(op->kind);
  s.plane = (size_t)op->nx * op->ny;
  s.N = s.plane * s.ncomp;
  s.state = state;
  uniform_coeffs(op->kind, op->nx, op->ny, op->param, s.kJ);
  s.st = nullptr;
  if (op->kind != PHIX_OP_ADVDIFF && !general_kind(op->kind)) {
    size_t nplanes = op->kind == PHIX_OP_GRAYSCOTT ? 2 : 1;
    size_t sb = prec == P_FP64 || prec == P_DF64 ? 8 : 4;
    void* st = ws(ctx, S_ST, nplanes * s.plane * sb);
    KL(launch_prep_state(prec, op->kind, op->nx, op->ny, state, st, ctx->grid_stream, ctx->stream));
    s.st = st;
    ++ctx->prep_gen;
  }
  return s;
}

// number of scalar uniform coefficients that alpha scales
int n_scaled(int kind) { return kind == PHIX_OP_ADVDIFF ? 5 : (kind == PHIX_OP_GRAYSCOTT ? 6 : 3); }

// ---------------------------------------------------------------------------
// Deferred chains.  Each pass (a Newton-Leja chain or a power iteration) gets
// a slot: its own control block, parameter block (device + pinned staging)
// and event pair.  The chain is one CUDA graph whose conditional WHILE node
// repeats GRAPH_ITERS iterations until the kernel clears the
// condition (the chain converged, hit m_max, or met a non-finite norm; m_max
// bounds the loop).  The host does not wait for a chain: it reads every
// pending slot at the next flush (one copy, one synchronisation), at the end
// of each API call or where it needs a value (the power-iteration estimate).
// ---------------------------------------------------------------------------
void flush(phix_ctx* ctx) {
  if (ctx->nslot == 0) return;
  CK(cudaMemcpyAsync(ctx->ctl_h, ctx->ctl, sizeof(LejaCtl) * ctx->nslot, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (const phix_ctx::Pending& q : ctx->pend) {
    const LejaCtl& c = ctx->ctl_h[q.slot];
    // the prefix launches, then the WHILE loop until the body holding the
    // launch that stopped the chain (none when it stopped inside the prefix;
    // one body when a chain without prefix stopped before its first
    // iteration); a persistent chain is one launch
    const int work_launches = q.fused2 ? (c.iters + 1) / 2 : c.iters;
    const int rest = work_launches - q.prefix;
    const long bodies = rest > 0 ? (rest + GRAPH_ITERS - 1) / GRAPH_ITERS : (q.prefix == 0 ? 1 : 0);
    ctx->launches += q.persistent ? 1 : q.prefix + (long)GRAPH_ITERS * bodies;
    if (!q.stats) continue;
    const int status = c.done ? c.status : PHIX_ENOTCONV;
    if (status == PHIX_ENOTCONV && c.iters == q.m_table && q.m_table < q.m_limit) {
      ctx->ran_out = true;  // the table was too short: the call runs again with full tables
      continue;
    }
    phix_stats& s = *q.stats;
    s.iters += c.iters;
    s.jv += c.iters;
    if (status != PHIX_OK) s.status = status;
    if (q.profile) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ctx->ev[2 * q.slot], ctx->ev[2 * q.slot + 1]));
      s.iter_ms += t;
      s.iter_bytes += q.bytes_per_launch * c.iters;
      s.iter_launches += c.iters;
    }
  }
  ctx->pend.clear();
  ctx->nslot = 0;
}

// A free slot whose parameter block holds `ptab_need` bytes (flushes when
// every slot is taken or the blocks must grow).
int acquire_slot(phix_ctx* ctx, size_t ptab_need) {
  if (ctx->nslot == NSLOT || ptab_need > ctx->ptab_slot) flush(ctx);
  if (ptab_need > ctx->ptab_slot) {
    const size_t sz = (std::max(ptab_need, (size_t)(64 << 10)) + 255) & ~(size_t)255;
    if (ctx->ptab_d) CK(cudaFree(ctx->ptab_d));
    if (ctx->ptab_h) CK(cudaFreeHost(ctx->ptab_h));
    ctx->ptab_d = nullptr;
    ctx->ptab_h = nullptr;
    ctx->ptab_slot = 0;
    cudaError_t e = cudaMalloc(&ctx->ptab_d, sz * NSLOT);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      fail(ctx, PHIX_ENOMEM, "parameter blocks of %zu bytes: %s", sz * NSLOT, cudaGetErrorString(e));
    }
    CK(cudaMallocHost(&ctx->ptab_h, sz * NSLOT));
    ctx->ptab_slot = sz;
  }
  const int s = ctx->nslot++;
  CK(cudaMemsetAsync(ctx->ctl + s, 0, sizeof(LejaCtl), ctx->stream));
  return s;
}

// Fill slot s's parameter block and queue its upload.
const void* upload_ptab(phix_ctx* ctx, int s, int K, int m_min, int m_max, double tol, double rel, const double* k8,
                        double ga, const double* beta, const double* const* dk, int prescaled = 0) {
  const size_t bytes = ptab_bytes(m_max + 1);
  unsigned char* h = ctx->ptab_h + (size_t)s * ctx->ptab_slot;
  unsigned char* d = ctx->ptab_d + (size_t)s * ctx->ptab_slot;
  ptab_fill(h, K, m_min, m_max, tol, rel, k8, ga, beta, dk, prescaled);
  CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return d;
}

// A cached CUDA graph: one conditional WHILE node whose body is GRAPH_ITERS
// iteration launches of `spec`; the key is the spec without the handle.
cudaGraphExec_t chain_graph(phix_ctx* ctx, const ChainSpec& key) {
  for (auto& g : ctx->graphs)
    if (std::memcmp(&g.spec, &key, sizeof key) == 0) return g.exec;
  if (ctx->graphs.size() >= 256) {
    CK(cudaGraphExecDestroy(ctx->graphs.front().exec));
    ctx->graphs.erase(ctx->graphs.begin());
  }
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) break;
    ChainSpec spec = key;
    spec.use_cond = 1;
    spec.cond = h;
    alignas(64) unsigned char argbuf[2048];  // kernel arguments (tensor maps are 64-byte aligned)
    // the prefix: launches in sequence ahead of the loop, clearing the same
    // condition when the chain has stopped
    cudaGraphNode_t last = nullptr;
    for (int i = 0; i < key.prefix && e == cudaSuccess; ++i) {
      cudaKernelNodeParams np;
      e = iter_node_params(spec, &np, argbuf, sizeof argbuf);
      if (e != cudaSuccess) break;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, g, last ? &last : nullptr, last ? 1 : 0, &np);
      last = node;
    }
    if (e != cudaSuccess) break;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};  // the rest zero
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    e = cudaGraphAddNode(&cn, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &cp);
    if (e != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < GRAPH_ITERS && e == cudaSuccess; ++i) {
      cudaKernelNodeParams np;
      e = iter_node_params(spec, &np, argbuf, sizeof argbuf);
      if (e != cudaSuccess) break;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &np);
      prev = node;
    }
    if (e != cudaSuccess) break;
    e = cudaGraphInstantiate(&exec, g, 0);
  } while (false);
  cudaGraphDestroy(g);
  CK(e);
  phix_ctx::Graph gg;
  gg.spec = key;
  gg.exec = exec;
  ctx->graphs.push_back(gg);
  return exec;
}

// Queue a chain in slot s (bracketed by the slot's events when profiling).
// direct: launch the iteration kernels one by one, GRAPH_ITERS at a time,
// reading the slot's control block in between (for per-kernel profilers,
// which do not see into conditional graphs); the device stops the chain by
// m_max, so at most m_max + GRAPH_ITERS launches are made.
void queue_chain(phix_ctx* ctx, int s, const ChainSpec& spec, bool profile, bool direct, int m_max) {
  ChainSpec key = spec;
  key.use_cond = 0;
  key.cond = 0;
  if (profile) CK(cudaEventRecord(ctx->ev[2 * s], ctx->stream));
  if (direct) {
    alignas(64) unsigned char argbuf[2048];
    cudaKernelNodeParams np;
    CK(iter_node_params(key, &np, argbuf, sizeof argbuf));
    LejaCtl c{};
    for (int launched = 0; launched <= m_max;) {
      for (int i = 0; i < GRAPH_ITERS; ++i, ++launched) {
        CK(cudaLaunchKernel(np.func, np.gridDim, np.blockDim, np.kernelParams, np.sharedMemBytes, ctx->stream));
        ctx->launches += 1;
      }
      CK(cudaMemcpyAsync(&c, ctx->ctl + s, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (c.done) break;
    }
    const int wl = key.fused2 ? (c.iters + 1) / 2 : c.iters;
    ctx->launches -= (long)GRAPH_ITERS * std::max(1, (wl + GRAPH_ITERS - 1) / GRAPH_ITERS);  // counted at the flush
  } else {
    CK(cudaGraphLaunch(chain_graph(ctx, key), ctx->stream));  // its kernel launches are counted at the flush
  }
  if (profile) CK(cudaEventRecord(ctx->ev[2 * s + 1], ctx->stream));
}

// ---------------------------------------------------------------------------
// The general float64 path (general_kernels.cu): the no-flow problems, the
// finite-difference Jacobian and the augmented-matrix form.  One launch per
// iteration, GRAPH_ITERS at a time, the host reading the control block in
// between (the device stops the chain itself; at most m_max + GRAPH_ITERS
// launches).
// ---------------------------------------------------------------------------
struct GenAug {                 // augmented-matrix form (Appendix A)
  std::vector<const double*> src;  // b_j, j = 1..p (index j - 1; NULL = zero)
  double hgamma = 1.0;             // h gamma of the interval (source weights 1 / (h gamma))
  double hc = 0.0;
};

struct GenOp {                  // operator data of the general kernel
  const double* st = nullptr;   // state (nonlinear operators)
  const double* fu = nullptr;   // f(state) (finite differences)
  double fd_scale = 0.0;
  int fd = 0;
};

GenOp general_op(phix_ctx* ctx, const OpState& os, const phix_opts& o) {
  GenOp g;
  g.fd = o.jv == PHIX_JV_FD;
  g.st = os.state;
  if (g.fd) {
    if (!g.st) {  // a linear operator has no state: linearise at zero
      double* z = wsd(ctx, S_GZ, os.N);
      CK(cudaMemsetAsync(z, 0, os.N * sizeof(double), ctx->stream));
      g.st = z;
    }
    double* fu = wsd(ctx, S_GFU, os.N);
    KL(launch_rhs(os.d, g.st, fu, ctx->grid_stream, ctx->stream));
    KL(launch_norm2(os.N, g.st, nullptr, ctx->partials, ctx->counter, ctx->scal, ctx->grid_stream, ctx->stream));
    CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    g.fu = fu;
    g.fd_scale = std::sqrt(std::ldexp(1.0, -52)) * (1.0 + std::sqrt(ctx->scal_h[0]));
  }
  return g;
}

// Run a general chain (init or power start already queued) to its end; returns the control block.
LejaCtl general_chain(phix_ctx* ctx, int mode, const OpState& os, int K, double* const* y, double* const* p,
                      const GenOp& go, const GenAug* aug, LejaCtl* ctl, const double* tab, int m_max) {
  std::vector<const double*> src;
  if (aug) src = aug->src;
  LejaCtl c{};
  for (int launched = 0; launched <= m_max;) {
    for (int i = 0; i < GRAPH_ITERS; ++i, ++launched)
      KL(launch_general(mode, os.d.kind, os.d.nx, os.d.ny, K, nullptr, y, p, go.st, go.fu, go.fd_scale, go.fd, os.d.p,
                        src.data(), (int)src.size(), ctl, ctx->partials, tab, ctx->grid_stream, ctx->stream));
    CK(cudaMemcpyAsync(&c, ctl, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (c.done) break;
  }
  return c;
}

// One vertical Newton-Leja pass on the general kernel: out[k] = sum_m d_k[m] y_m
// (the outputs accumulate in place, float64, no input scaling).
void general_pass(phix_ctx* ctx, const OpState& os, const double* v, int K,
                  const std::vector<const std::vector<double>*>& d, double c, double gamma, double tol,
                  const phix_opts& o, double* const* out, phix_stats& stats, const GenAug* aug = nullptr) {
  flush(ctx);
  const int M = (int)d[0]->size();
  const int m_max = M - 1;
  const double* xi = leja_table(M);
  std::vector<double> tab(gen_table_doubles(M), 0.0);
  const int nsrc = aug ? (int)aug->src.size() : 0;
  tab[0] = K;
  tab[1] = o.m_min;
  tab[2] = m_max;
  tab[3] = M;
  tab[4] = tol;
  tab[5] = 0.0;
  tab[6] = 1.0 / gamma;
  tab[7] = nsrc;
  double* beta = &tab[8];
  double* dk = beta + M;
  double* w = dk + (size_t)KMAX * M;
  double* yt = w + (size_t)KIOPS_PMAX * M;
  double* pt = yt + M;
  for (int m = 1; m < M; ++m) beta[m] = -(c / gamma + xi[m - 1]);
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < M; ++m) dk[(size_t)k * M + m] = (*d[k])[m];
  if (aug && nsrc > 0) {
    // the tail y_T of the augmented vector [b_0; e_p] evolves alone:
    // y_T,m+1 = ((K - hc)/(h gamma) - xi_m) y_T,m (K: the upward shift); its
    // source weights B y_T / (h gamma) and its share of the norms are known here
    const int pn = nsrc;
    std::vector<double> yT(pn, 0.0), pT(pn, 0.0), nxt(pn);
    yT[pn - 1] = 1.0;
    for (int m = 0; m < M; ++m) {
      double y2 = 0.0, p2 = 0.0;
      for (int i = 0; i < pn; ++i) {
        pT[i] += (*d[0])[m] * yT[i];
        y2 += yT[i] * yT[i];
        p2 += pT[i] * pT[i];
      }
      yt[m] = y2;
      pt[m] = p2;  // K == 1 in the augmented form
      for (int j = 1; j <= pn; ++j) w[(size_t)m * KIOPS_PMAX + (j - 1)] = yT[pn - j] / aug->hgamma;
      for (int i = 0; i < pn; ++i) {
        const double ky = i + 1 < pn ? yT[i + 1] : 0.0;
        nxt[i] = (ky - aug->hc * yT[i]) / aug->hgamma - (m < M - 1 ? xi[m] : 0.0) * yT[i];
      }
      yT = nxt;
    }
  }
  double* dtab = wsd(ctx, S_GTAB, tab.size());
  CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LejaCtl* ctl = static_cast<LejaCtl*>(ws(ctx, S_GCTL, sizeof(LejaCtl)));
  CK(cudaMemsetAsync(ctl, 0, sizeof(LejaCtl), ctx->stream));
  double* y[2] = {wsd(ctx, S_Y0, os.N), wsd(ctx, S_Y1, os.N)};
  const GenOp go = general_op(ctx, os, o);
  std::vector<const double*> src;
  if (aug) src = aug->src;
  KL(launch_general(2, os.d.kind, os.d.nx, os.d.ny, K, v, y, out, go.st, go.fu, go.fd_scale, go.fd, os.d.p,
                    src.data(), nsrc, ctl, ctx->partials, dtab, ctx->grid_stream, ctx->stream));
  const LejaCtl cb = general_chain(ctx, 0, os, K, y, out, go, aug, ctl, dtab, m_max);
  const int status = cb.done ? cb.status : PHIX_ENOTCONV;
  if (status == PHIX_ENOTCONV && cb.iters == m_max && m_max < o.m_max) {
    ctx->ran_out = true;  // the table was too short: the call runs again with full tables
    throw Rerun{};
  }
  stats.iters += cb.iters;
  stats.jv += cb.iters;
  stats.passes += 1;
  if (status != PHIX_OK) stats.status = status;
}

// Power iteration on the general kernel (the no-flow problems, or the
// finite-difference Jacobian).
double general_power(phix_ctx* ctx, const OpState& os, const phix_opts& o, int* mv) {
  flush(ctx);
  std::vector<double> tab(gen_table_doubles(1), 0.0);
  tab[2] = o.power_max_it;
  tab[3] = 1;
  tab[5] = o.power_rel;
  double* dtab = wsd(ctx, S_GTAB, tab.size());
  CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  LejaCtl* ctl = static_cast<LejaCtl*>(ws(ctx, S_GCTL, sizeof(LejaCtl)));
  CK(cudaMemsetAsync(ctl, 0, sizeof(LejaCtl), ctx->stream));
  double* y[2] = {wsd(ctx, S_Y0, os.N), wsd(ctx, S_Y1, os.N)};
  const GenOp go = general_op(ctx, os, o);
  KL(launch_power_start(P_FP64, os.N, o.power_seed, y[0], ctl, ctx->partials, ctx->grid_iter, ctx->stream));
  const LejaCtl c = general_chain(ctx, 1, os, 0, y, nullptr, go, nullptr, ctl, dtab, o.power_max_it);
  if (c.status == PHIX_ENAN) fail(ctx, PHIX_ENAN, "power iteration produced a non-finite norm");
  *mv = c.iters;
  return c.rho;
}

// One Newton-Leja pass (Sec. 2.2): queued; its outcome reaches `stats` at the
// next flush.
void leja_pass(phix_ctx* ctx, const OpState& os, int prec, const double* v, int K,
               const std::vector<const std::vector<double>*>& d, double c, double gamma, double tol,
               const phix_opts& o, double* const* out, phix_stats& stats, const void* st_newton,
               int prescaled) {
  if (general_kind(os.d.kind) || o.jv == PHIX_JV_FD) {
    general_pass(ctx, os, v, K, d, c, gamma, tol, o, out, stats);
    return;
  }
  const int M = (int)d[0]->size();  // table length: at most o.m_max + 1
  const int m_max = M - 1;
  const double* xi = leja_table(M);
  const size_t eb = elem_bytes(prec);
  void* y[2] = {ws(ctx, S_Y0, os.N * eb), ws(ctx, S_Y1, os.N * eb)};
  void* p[KMAX] = {};
  for (int k = 0; k < K; ++k) p[k] = ws(ctx, S_P0 + k, os.N * eb);

  const int s = acquire_slot(ctx, ptab_bytes(M));
  LejaCtl* ctl = ctx->ctl + s;
  const double alpha = 1.0 / gamma;
  const int ns = n_scaled(os.d.kind);
  double k8[8];
  for (int j = 0; j < 8; ++j) k8[j] = j < ns ? alpha * os.kJ[j] : os.kJ[j];
  std::vector<double> beta(M, 0.0);
  for (int m = 1; m < M; ++m) beta[m] = -(c / gamma + xi[m - 1]);
  const double* dk[KMAX] = {};
  for (int k = 0; k < K; ++k) dk[k] = d[k]->data();
  const void* ptab = upload_ptab(ctx, s, K, o.m_min, m_max, tol, 0.0, k8, alpha, beta.data(), dk, prescaled);

  KL(launch_scale(v, os.N, ctl, ctx->partials, ctx->grid_iter, ctx->stream));
  InitLaunch IL{};
  IL.prec = prec;
  IL.ncomp = os.ncomp;
  IL.nx = os.d.nx;
  IL.ny = os.d.ny;
  IL.v = v;
  IL.y0 = y[0];
  for (int k = 0; k < K; ++k) IL.p[k] = p[k];
  IL.ctl = ctl;
  IL.partials = ctx->partials;
  IL.ptab = ptab;
  IL.grid = ctx->grid_iter;
  KL(launch_init(IL, ctx->stream));

  ChainSpec cs{};
  cs.prec = prec;
  cs.op = os.d.kind;
  cs.mode = MODE_NEWTON;
  cs.nx = os.d.nx;
  cs.ny = os.d.ny;
  cs.y[0] = y[0];
  cs.y[1] = y[1];
  for (int k = 0; k < K; ++k) cs.p[k] = p[k];
  cs.st = st_newton;
  cs.ctl = ctl;
  cs.partials = ctx->partials;
  cs.ptab = ptab;
  cs.K = K;
  const double st_b = os.d.kind == PHIX_OP_GRAYSCOTT ? 2.0 * os.plane * eb
                     : os.d.kind == PHIX_OP_BURGERS ? 1.0 * os.plane * eb : 0.0;
  {
    // TMA staging pays once an iteration's operands no longer stay in L2
    // (read y, write y', read and write each p_k, read the state).  Two
    // iterations per launch on request only: measured on GB300 it is no faster
    // (1024^2 Gray-Scott double-float 21.5-22.4 us per iteration against 18.6-18.7
    // single-step; 2048^2 69.9-72.2 against 73.0-73.3 TMA-staged; Burgers 2048^2
    // float64 179 against 163, float32 26.2 against 24.5)
    const double work = (double)os.N * eb * (2.0 + 2.0 * K) + st_b;
    cs.fused2 = o.kernel == PHIX_KERNEL_FUSED2 && o.chain != PHIX_CHAIN_PERSISTENT && fused2_eligible(cs) ? 1 : 0;
    const bool want = o.kernel == PHIX_KERNEL_TMA || (o.kernel == PHIX_KERNEL_AUTO && work > ctx->l2_bytes);
    cs.tma = !cs.fused2 && want && tma_eligible(cs) ? 1 : 0;
  }
  bool persistent = false;
  if (cs.tma) {
    cs.grid = tma_grid(cs, ctx->nsm);
  } else if (cs.fused2) {
    // the partials hold two halves of grid x (KMAX + 1)
    const int gmax = std::min(ctx->grid_iter / 2, ctx->nsm * std::min(8, fused2_blocks_per_sm(cs)));
    const int ntiles = fused2_tiles(cs);
    const int per = (ntiles + gmax - 1) / gmax;  // tiles per block, balanced
    cs.grid = (ntiles + per - 1) / per;
  } else {
    if (o.chain == PHIX_CHAIN_PERSISTENT) {
      // the whole pass in one cooperative launch: every block resident, its
      // partials double-buffered (2 x grid x (KMAX + 1) doubles)
      const int g = chain_grid(cs, ctx->nsm);
      persistent = g >= 1 && 2 * g <= ctx->grid_iter;
      if (persistent) cs.grid = g;
    }
    if (!persistent) {
      const int gmax = ctx->nsm * std::min(8, iter_blocks_per_sm(cs));
      const int ntiles = iter_tiles(cs);
      const int per = (ntiles + gmax - 1) / gmax;  // tiles per block, balanced
      cs.grid = (ntiles + per - 1) / per;
    }
  }
  const bool profile = o.profile != 0;
  // graph chains: the predicted chain length (the table was truncated to
  // twice the prediction plus 24; chains measured 1.2-1.9x the prediction),
  // in whole bodies, runs ahead of the WHILE node without condition evaluations
  if (!persistent && o.profile != 2 && m_max < o.m_max) {
    const int m_pred = (M - 24) / 2;
    const int pl = cs.fused2 ? m_pred / 2 : m_pred;
    cs.prefix = std::max(0, pl / GRAPH_ITERS * GRAPH_ITERS);
  }
  if (persistent) {
    if (profile) CK(cudaEventRecord(ctx->ev[2 * s], ctx->stream));
    CK(launch_chain(cs, ctx->stream));
    if (profile) CK(cudaEventRecord(ctx->ev[2 * s + 1], ctx->stream));
  } else {
    queue_chain(ctx, s, cs, profile, o.profile == 2, m_max);
  }
  stats.tma_passes += cs.tma;
  FusedOut fo{};
  fo.y[0] = y[0];
  fo.y[1] = y[1];
  fo.ptab = ptab;
  KL(launch_finalize(prec, os.N, K, p, out, ctl, ctx->grid_stream, ctx->stream, cs.fused2 ? &fo : nullptr));
  phix_ctx::Pending q{};
  q.slot = s;
  q.stats = &stats;
  q.profile = profile;
  q.m_table = m_max;
  q.m_limit = o.m_max;
  q.persistent = persistent;
  q.fused2 = cs.fused2 != 0;
  q.prefix = cs.prefix;
  if (profile) {
    // algorithmic bytes of one iteration: read y, write the new iterate, read
    // and write each p_k, read the state planes; a two-iteration launch moves
    // that once for two iterations
    const size_t sb = (prec == P_FP64 || prec == P_DF64) ? 8 : 4;
    const double st_bytes = os.d.kind == PHIX_OP_GRAYSCOTT ? 2.0 * os.plane * sb
                           : os.d.kind == PHIX_OP_BURGERS ? 1.0 * os.plane * sb : 0.0;
    q.bytes_per_launch = ((double)os.N * eb * (2.0 + 2.0 * K) + st_bytes) / (cs.fused2 ? 2.0 : 1.0);
  }
  ctx->pend.push_back(q);
}

// The cached table of phi_l(a + b x), grown as needed.  At most 16 are kept,
// least recently used first; one pass looks up at most KMAX < 16 tables, so
// none of them is evicted while the pass holds references.
DDTable& dd_lookup(phix_ctx* ctx, int l, double a, double b) {
  auto& c = ctx->dd_cache;
  for (auto it = c.begin(); it != c.end(); ++it)
    if (it->l == l && it->a == a && it->b == b) {
      c.splice(c.end(), c, it);  // most recent last
      return c.back();
    }
  if (c.size() >= 16) c.pop_front();
  c.emplace_back();
  DDTable& t = c.back();
  t.l = l;
  t.a = a;
  t.b = b;
  return t;
}

// Coefficient tables of one pass (outputs l_k of phi_{l_k}(a_k + b_k x)),
// truncated to twice the predicted chain length plus 24 points: the chain is
// predicted to stop by the first m >= m_min with |d_k[m]| <= tol |d_k[0]| / 2
// for every k (the Newton terms decay like the divided differences).  Full
// length (m_max + 1) when ctx->full_tables is set.
std::vector<std::vector<double>> pass_tables(phix_ctx* ctx, int K, const int* l, const double* a, const double* b,
                                             double tol, const phix_opts& o) {
  const int M = o.m_max + 1;
  std::vector<DDTable*> t(K);
  for (int k = 0; k < K; ++k) t[k] = &dd_lookup(ctx, l[k], a[k], b[k]);
  int M1 = M;
  if (!ctx->full_tables) {
    int m_pred = -1, n = 0;
    while (m_pred < 0 && n < M) {
      const int n0 = n;
      n = std::min(M, n + 32);
      for (int k = 0; k < K; ++k) t[k]->grow(n);
      for (int m = std::max({1, o.m_min, n0}); m < n && m_pred < 0; ++m) {
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) ok = std::fabs(t[k]->d[m]) <= 0.5 * tol * std::fabs(t[k]->d[0]);
        if (ok) m_pred = m;
      }
    }
    if (m_pred >= 0) M1 = std::min(M, 2 * m_pred + 24);
  }
  std::vector<std::vector<double>> d(K);
  for (int k = 0; k < K; ++k) {
    t[k]->grow(M1);
    d[k].assign(t[k]->d.begin(), t[k]->d.begin() + M1);
  }
  return d;
}

// Power iteration (Sec. 2.2) on the device, queued: returns its slot.
int power_iteration_queue(phix_ctx* ctx, const OpState& os, int prec, const phix_opts& o) {
  const size_t eb = elem_bytes(prec);
  void* y[2] = {ws(ctx, S_Y0, os.N * eb), ws(ctx, S_Y1, os.N * eb)};
  const int s = acquire_slot(ctx, ptab_bytes(o.power_max_it + 1));
  LejaCtl* ctl = ctx->ctl + s;
  const void* ptab = upload_ptab(ctx, s, 0, 0, o.power_max_it, 0.0, o.power_rel, os.kJ, 1.0, nullptr, nullptr);
  KL(launch_power_start(prec, os.N, o.power_seed, y[0], ctl, ctx->partials, ctx->grid_iter, ctx->stream));
  ChainSpec cs{};
  cs.prec = prec;
  cs.op = os.d.kind;
  cs.mode = MODE_POWER;
  cs.nx = os.d.nx;
  cs.ny = os.d.ny;
  cs.y[0] = y[0];
  cs.y[1] = y[1];
  cs.st = os.st;
  cs.ctl = ctl;
  cs.partials = ctx->partials;
  cs.ptab = ptab;
  cs.grid = ctx->nsm * std::min(8, iter_blocks_per_sm(cs));
  queue_chain(ctx, s, cs, false, o.profile == 2, o.power_max_it);
  phix_ctx::Pending q{};
  q.slot = s;
  ctx->pend.push_back(q);
  return s;
}

double power_result(phix_ctx* ctx, int s, int* mv) {
  const LejaCtl& c = ctx->ctl_h[s];
  if (c.status == PHIX_ENAN) fail(ctx, PHIX_ENAN, "power iteration produced a non-finite norm");
  *mv = c.iters;
  return c.rho;
}

// The estimate, flushing every queued pass.
double power_iteration(phix_ctx* ctx, const OpState& os, int prec, const phix_opts& o, int* mv) {
  if (general_kind(os.d.kind) || o.jv == PHIX_JV_FD) return general_power(ctx, os, o, mv);
  const int s = power_iteration_queue(ctx, os, prec, o);
  flush(ctx);
  return power_result(ctx, s, mv);
}

// Queued with a read-back of its control block behind it (and an event after
// that): the host queues work that does not need the estimate, then waits
// for the read-back alone (power_iteration_collect) while that work runs.
int power_iteration_split(phix_ctx* ctx, const OpState& os, int prec, const phix_opts& o) {
  const int s = power_iteration_queue(ctx, os, prec, o);
  CK(cudaMemcpyAsync(ctx->ctl_h + s, ctx->ctl + s, sizeof(LejaCtl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaEventRecord(ctx->ev[2 * NSLOT + 2], ctx->stream));
  return s;
}

double power_iteration_collect(phix_ctx* ctx, int s, int* mv) {
  CK(cudaEventSynchronize(ctx->ev[2 * NSLOT + 2]));
  return power_result(ctx, s, mv);
}

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

int substeps_for(double h, double s, double gamma, double rho_im, const phix_opts& o) {
  int n = 1;
  if (o.gamma_cap > 0) n = std::max(n, (int)std::ceil(s * h * gamma / o.gamma_cap - 1e-12));
  if (o.iota_cap > 0 && rho_im > 0) n = std::max(n, (int)std::ceil(s * h * rho_im / o.iota_cap - 1e-12));
  return n;
}

void lincomb(phix_ctx* ctx, size_t n, std::vector<double> c, std::vector<const double*> x, double* out) {
  // chains of at most 6 terms; out may alias x[0]
  size_t i = 0;
  bool first = true;
  while (i < c.size()) {
    std::vector<double> cc;
    std::vector<const double*> xx;
    if (!first) {
      cc.push_back(1.0);
      xx.push_back(out);
    }
    while (i < c.size() && cc.size() < 6) {
      cc.push_back(c[i]);
      xx.push_back(x[i]);
      ++i;
    }
    KL(launch_lincomb(n, (int)cc.size(), cc.data(), xx.data(), out, ctx->grid_stream, ctx->stream));
    first = false;
  }
}

struct Interval {
  double c, gamma, rho;
};

// Real Leja actions: out[k] = phi_{l_k}(s_k h J) v (vertical when no substeps).
void leja_phi(phix_ctx* ctx, const OpState& os, int prec, double h, const double* v, int nout,
              const int* l, const double* sc, double* const* out, double tol, const phix_opts& o,
              const Interval& iv, phix_stats& stats) {
  // complex spectra: the half-width covers twice the imaginary extent (scaled
  // imaginary extent <= 1/2) and the interval stays anchored at its right end
  Interval ivc = iv;
  ivc.gamma = std::max(iv.gamma, 2.0 * std::max(0.0, o.rho_im));
  ivc.c = (iv.c + 2.0 * iv.gamma) - 2.0 * ivc.gamma;
  if (ivc.gamma == 0.0) {  // zero spectrum: phi_l(0) v = v / l!
    for (int k = 0; k < nout; ++k) lincomb(ctx, os.N, {1.0 / factorial(l[k])}, {v}, out[k]);
    return;
  }
  // Gray-Scott: the Newton passes read the state terms V^2, 2UV already
  // multiplied by the factor 1/gamma their stencil applies (one preparation
  // per state and factor, shared by every pass of the call)
  const void* st_n = os.st;
  int pre = 0;
  if (os.d.kind == PHIX_OP_GRAYSCOTT && o.jv != PHIX_JV_FD) {
    const double alpha = 1.0 / ivc.gamma;
    const size_t sb = prec == P_FP64 || prec == P_DF64 ? 8 : 4;
    void* st2 = ws(ctx, S_ST2, 2 * os.plane * sb);
    if (ctx->st2_gen != ctx->prep_gen || ctx->st2_alpha != alpha) {
      KL(launch_prep_state(prec, os.d.kind, os.d.nx, os.d.ny, os.state, st2, ctx->grid_stream, ctx->stream, alpha));
      ctx->st2_gen = ctx->prep_gen;
      ctx->st2_alpha = alpha;
    }
    st_n = st2;
    pre = 1;
  }
  int smax = 1;
  std::vector<int> subs(nout);
  for (int k = 0; k < nout; ++k) {
    subs[k] = substeps_for(h, sc[k], ivc.gamma, o.rho_im, o);
    smax = std::max(smax, subs[k]);
  }
  if (smax == 1) {
    double ta[KMAX], tb[KMAX];
    for (int k = 0; k < nout; ++k) {
      ta[k] = sc[k] * h * ivc.c;
      tb[k] = sc[k] * h * ivc.gamma;
    }
    const std::vector<std::vector<double>> d = pass_tables(ctx, nout, l, ta, tb, tol, o);
    std::vector<const std::vector<double>*> dp(nout);
    for (int k = 0; k < nout; ++k) dp[k] = &d[k];
    leja_pass(ctx, os, prec, v, nout, dp, ivc.c, ivc.gamma, tol, o, out, stats, st_n, pre);
    stats.passes += 1;
    stats.substeps += 1;
    return;
  }
  // ODE-identity substeps, one output at a time:
  //   u(t+tau) = sum_{j<l} tau^j/j! w_j + tau^l phi_l(tau B) w_l,
  //   w_0 = u(t), w_j = B w_{j-1} + v t^(l-j)/(l-j)!,  B = s h J
  double* u = wsd(ctx, S_SUB_U, os.N);
  double* tmp = wsd(ctx, S_SUB_TMP, os.N);
  for (int k = 0; k < nout; ++k) {
    const int L = l[k], ns = subs[k];
    if (L > 8) fail(ctx, PHIX_EINVAL, "substepped phi_l needs l <= 8");
    const double tau = 1.0 / ns;
    const double ta = tau * sc[k] * h * ivc.c, tb = tau * sc[k] * h * ivc.gamma;
    const std::vector<std::vector<double>> d = pass_tables(ctx, 1, &L, &ta, &tb, tol, o);
    const std::vector<const std::vector<double>*> dp(1, &d[0]);
    if (L == 0)
      CK(cudaMemcpyAsync(u, v, os.N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemsetAsync(u, 0, os.N * sizeof(double), ctx->stream));
    std::vector<double*> w(L + 1);
    w[0] = u;
    for (int j = 1; j <= L; ++j) w[j] = wsd(ctx, S_SUB_W0 + j, os.N);
    for (int i = 0; i < ns; ++i) {
      const double t = i * tau;
      for (int j = 1; j <= L; ++j) {
        double coef = std::pow(t, L - j) / factorial(L - j);
        KL(launch_jv_axpy(os.d, os.state, w[j - 1], sc[k] * h, v, coef, w[j], ctx->grid_stream, ctx->stream));
        stats.jv += 1;
      }
      double* outs[1] = {tmp};
      leja_pass(ctx, os, prec, w[L], 1, dp, ivc.c, ivc.gamma, tol, o, outs, stats, st_n, pre);
      stats.passes += 1;
      std::vector<double> cc;
      std::vector<const double*> xx;
      cc.push_back(std::pow(tau, L));
      xx.push_back(tmp);
      for (int j = 0; j < L; ++j) {
        cc.push_back(std::pow(tau, j) / factorial(j));
        xx.push_back(w[j]);
      }
      // u appears as w[0] on the right: write to tmp first, then swap roles by copying
      lincomb(ctx, os.N, cc, xx, tmp);
      CK(cudaMemcpyAsync(u, tmp, os.N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    stats.substeps += ns;
    CK(cudaMemcpyAsync(out[k], u, os.N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
}

struct Interval;
void leja_phi(phix_ctx* ctx, const OpState& os, int prec, double h, const double* v, int nout,
              const int* l, const double* sc, double* const* out, double tol, const phix_opts& o,
              const Interval& iv, phix_stats& stats);
Interval interval_for(phix_ctx* ctx, const OpState& os, int prec, const phix_opts& o, phix_stats& stats);

// out_k = phi_{l_k}(s_k h J) v by the chosen method (iv: the Leja interval,
// estimated here when NULL).
void phi_actions(phix_ctx* ctx, const OpState& os, phix_method method, int prec, double h, const double* v,
                 int nout, const int* l, const double* sc, double* const* out, double tol, const phix_opts& o,
                 const Interval* iv, phix_stats& stats);

// ---------------------------------------------------------------------------
// KIOPS-style run (Sec. 2.1): w(tau) = sum_j tau^j phi_j(tau h J) b_j at the
// sorted distinct output times; substep and Krylov-dimension control as in
// the oracle (accept omega <= 1; else grow m by m_step up to m_max, then
// shrink tau).
// ---------------------------------------------------------------------------
struct KOut {
  double* out;
  double scale;
};

int kiops_prec(int prec) { return prec == P_FP64 ? P_FP64 : P_DF64; }

void read_kc(phix_ctx* ctx, KiopsCtl* kc) {
  CK(cudaMemcpyAsync(ctx->kc_h, kc, KIOPS_HOST_BYTES, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
}

// The small exponential with its decision read from the mailbox: poll the
// sequence number (a few microseconds after the kernel's write, against the
// wake-up of a stream synchronisation); after 0.5 s without it, synchronise
// the stream, which reports a failed kernel, and read the mailbox then.
void smallexp_decision(phix_ctx* ctx, KiopsCtl* kc, int m, double tau, double tau_end, double tol) {
  const unsigned int seq = ++ctx->kmb_seq;
  KL(kiops_smallexp(kc, m, tau, tau_end, tol, ctx->kmb_d, seq, ctx->stream));
  const auto t0 = std::chrono::steady_clock::now();
  for (long spin = 0; ctx->kmb_h->seq != seq; ++spin) {
    if ((spin & 1023) == 1023 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(500)) {
      CK(cudaStreamSynchronize(ctx->stream));
      if (ctx->kmb_h->seq != seq) fail(ctx, PHIX_ECUDA, "KIOPS decision mailbox not written");
      break;
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  std::memcpy(ctx->kc_h, const_cast<const unsigned char*>(ctx->kmb_h->header), KIOPS_HOST_BYTES);
}

void kiops_run(phix_ctx* ctx, const OpState& os, int prec, double h, const double* const* b, int p,
               const std::vector<double>& times, const std::vector<std::vector<KOut>>& outs, double tol,
               const phix_opts& o, phix_stats& stats) {
  const bool general = general_kind(os.d.kind);  // the no-flow problems: float64 general pass 1
  const int kp = general ? P_FP64 : kiops_prec(prec);
  const size_t N = os.N, eb = 8;
  const int mmax = o.kiops_m_max;
  if (p > KIOPS_PMAX) fail(ctx, PHIX_EINVAL, "KIOPS supports p <= %d", KIOPS_PMAX);
  KiopsSpec ks{};
  ks.prec = kp;
  ks.op = os.d.kind;
  ks.nx = os.d.nx;
  ks.ny = os.d.ny;
  ks.p = p;
  unsigned char* base = static_cast<unsigned char*>(ws(ctx, S_KBASIS, (size_t)(mmax + 2) * N * eb));
  for (int i = 0; i < mmax + 2; ++i) ks.Zh[i] = base + (size_t)i * N * eb;
  void** Zd = static_cast<void**>(ws(ctx, S_KPTR, sizeof(void*) * (mmax + 2)));
  CK(cudaMemcpyAsync(Zd, ks.Zh, sizeof(void*) * (mmax + 2), cudaMemcpyHostToDevice, ctx->stream));
  ks.Z = Zd;
  ks.st = general ? static_cast<const void*>(os.state) : os.st;
  for (int i = 0; i < 8; ++i) ks.prm[i] = os.d.p[i];
  KiopsCtl* kc = static_cast<KiopsCtl*>(ws(ctx, S_KCTL, sizeof(KiopsCtl)));
  CK(cudaMemsetAsync(kc, 0, sizeof(KiopsCtl), ctx->stream));
  ks.kc = kc;
  ks.partials = ctx->partials;
  ks.h = h;
  for (int i = 0; i < 8; ++i) ks.kJ[i] = os.kJ[i];
  ks.nscaled = n_scaled(os.d.kind);
  ks.grid = ctx->grid_iter;
  ks.nsm = ctx->nsm;
  ks.W[0] = ks.W[1] = nullptr;
  if (o.kiops_fused) {
    ks.W[0] = ws(ctx, S_KW, 2 * N * eb);
    ks.W[1] = static_cast<unsigned char*>(ks.W[0]) + N * eb;
  }
  const bool fused = kiops_fused_ok(ks);
  // b_j (j >= 1) copies in the iteration precision and their 1-norms -> eta
  int nb = 0;
  for (int j = 1; j <= p; ++j)
    if (b[j]) ++nb;
  unsigned char* bbase = nb ? static_cast<unsigned char*>(ws(ctx, S_KB, (size_t)nb * N * eb)) : nullptr;
  // 1-norms (float64 sums) of b_1..b_p, with their copies, and of b_0 -> eta and
  // a power-of-two scale c of the whole augmented start vector [c b_0; c e_p / eta]
  // (the action is linear; c keeps the double-float squares of the basis in range)
  double eta = 1.0, cscale = 1.0;
  {
    int q = 0;
    for (int j = 1; j <= p; ++j) {
      if (!b[j]) continue;
      ks.bz[q] = bbase + (size_t)q * N * eb;
      ks.bslot[q] = p - j;  // column b_j multiplies tail entry t = p - j
      KL(kiops_convert(kp, N, b[j], const_cast<void*>(ks.bz[q]), ctx->partials, ctx->counter, ctx->scal + q,
                       ctx->grid_stream, ctx->stream));
      ++q;
    }
    ks.nb = nb;
    if (b[0])
      KL(kiops_convert(kp, N, b[0], nullptr, ctx->partials, ctx->counter, ctx->scal + nb, ctx->grid_stream,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double) * (nb + 1), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double nmax = 0.0;
    for (int q2 = 0; q2 < nb; ++q2) nmax = std::max(nmax, ctx->scal_h[q2]);
    const double n0 = b[0] ? ctx->scal_h[nb] : 0.0;
    if (!std::isfinite(nmax) || !std::isfinite(n0)) fail(ctx, PHIX_ENAN, "non-finite input vector");
    if (nmax > 0) eta = std::ldexp(1.0, -(int)std::ceil(std::log2(nmax)));
    const double ref = std::max(n0, nb ? 1.0 / eta : 0.0);
    if (ref > 0) cscale = std::ldexp(1.0, -(int)std::ceil(std::log2(ref)));
  }
  // algorithmic bytes of one Arnoldi step: the Jacobian product reads z_j, the
  // state planes and the b copies and writes w, with <w, z_{j-1}> on the way;
  // the orthogonalisation reads w, z_j, z_{j-1} and writes w back
  const size_t sbytes = os.d.kind == PHIX_OP_GRAYSCOTT ? 2 * os.plane * eb
                       : os.d.kind == PHIX_OP_BURGERS ? os.plane * eb : 0;
  // fused steps: read W, Zhat_j, Zhat_{j-1}, the state and the b copies, write
  // Zhat_{j+1} and u; the pass 1 of step 0 that starts them reads Zhat_0, the
  // state and the b copies and writes W0
  const double step_bytes = fused ? (double)N * eb * (5.0 + nb) + (double)sbytes
                                  : (double)N * eb * (7.0 + nb) + (double)sbytes;
  const double first_bytes = (double)N * eb * (2.0 + nb) + (double)sbytes;
  KL(kiops_start(ks, b[0], eta, cscale, ctx->stream));
  read_kc(ctx, kc);
  stats.passes += 1;
  if (ctx->kc_h->status == PHIX_ENAN) fail(ctx, PHIX_ENAN, "non-finite input vector");
  if (ctx->kc_h->beta == 0.0) {
    for (size_t ti = 0; ti < times.size(); ++ti)
      for (const KOut& ko : outs[ti]) CK(cudaMemsetAsync(ko.out, 0, N * sizeof(double), ctx->stream));
    return;
  }
  const double tau_end = times.back();
  double t = 0.0, tau = tau_end;
  int m = std::min(o.kiops_m_init, mmax);
  size_t ti = 0;
  int substeps = 0;
  while (ti < times.size()) {
    if (substeps >= o.kiops_max_substeps) {
      stats.status = PHIX_ENOTCONV;
      set_err(ctx, "KIOPS substep limit reached");
      break;
    }
    const double next_out = times[ti];
    tau = std::min(tau, next_out - t);
    int built = 0;
    for (;;) {
      const bool prof = o.profile != 0 && m > built;
      if (prof) CK(cudaEventRecord(ctx->ev[2 * NSLOT], ctx->stream));
      int launched = 0;
      for (int j = built; j < m; ++j) {
        if (fused) {
          if (j == 0) {
            CK(kiops_fused_first(ks, ctx->stream));
            ++launched;
          }
          CK(kiops_fused_step(ks, j, ctx->stream));
          ++launched;
        } else {
          CK(kiops_arnoldi(ks, j, ctx->stream));
          launched += 2;
        }
      }
      ctx->launches += launched;
      if (prof) CK(cudaEventRecord(ctx->ev[2 * NSLOT + 1], ctx->stream));
      smallexp_decision(ctx, kc, m, tau, tau_end, tol);
      const KiopsCtl& H = *ctx->kc_h;
      const int happy = H.happy_m;
      const int steps = (happy > 0 ? std::min(happy, m) : m) - built;
      stats.iters += steps;
      stats.jv += steps;
      if (prof) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[2 * NSLOT], ctx->ev[2 * NSLOT + 1]));
        stats.iter_ms += ms;
        stats.iter_launches += launched;
        stats.iter_bytes += steps * step_bytes + (fused && built == 0 && steps > 0 ? first_bytes : 0.0);
      }
      if (H.status == PHIX_ENAN || !std::isfinite(H.omega)) fail(ctx, PHIX_ENAN, "KIOPS produced a non-finite value");
      built = m;
      if (happy > 0) m = happy;
      const double omega = H.omega;
      if (happy > 0 || omega <= 1.0) {
        const bool landed = std::fabs(t + tau - next_out) <= 1e-13 * std::max(1.0, next_out);
        const KOut* k0 = landed ? &outs[ti][0] : nullptr;
        KL(kiops_combine(ks, happy > 0 ? m : m + 1, k0 ? k0->out : nullptr, k0 ? k0->scale / cscale : 0.0,
                         ctx->stream));
        if (landed) {
          for (size_t q = 1; q < outs[ti].size(); ++q)
            lincomb(ctx, N, {outs[ti][q].scale / k0->scale}, {k0->out}, outs[ti][q].out);
          t = next_out;
          ++ti;
        } else {
          t = t + tau;
        }
        ++substeps;
        const double g = omega == 0.0 ? 2.0 : std::min(2.0, std::max(1.0, 0.8 * std::pow(omega, -1.0 / m)));
        tau *= g;
        break;
      }
      stats.rejections += 1;
      if (m < mmax) {
        m = std::min(mmax, m + o.kiops_m_step);
      } else {
        tau *= std::min(0.9, std::max(0.1, 0.8 * std::pow(omega, -1.0 / m)));
      }
    }
  }
  stats.substeps += substeps;
}

// phi_{l_k}(s_k h J) v by KIOPS: one run per distinct l with b_l = v and the
// output times s_k; out_k = w(s_k) / s_k^l.
void kiops_phi(phix_ctx* ctx, const OpState& os, int prec, double h, const double* v, int nout,
               const int* l, const double* sc, double* const* out, double tol, const phix_opts& o,
               phix_stats& stats) {
  std::vector<int> ls(l, l + nout);
  std::sort(ls.begin(), ls.end());
  ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
  for (int L : ls) {
    std::vector<double> times;
    for (int k = 0; k < nout; ++k)
      if (l[k] == L) times.push_back(sc[k]);
    std::sort(times.begin(), times.end());
    times.erase(std::unique(times.begin(), times.end()), times.end());
    std::vector<std::vector<KOut>> outs(times.size());
    for (int k = 0; k < nout; ++k) {
      if (l[k] != L) continue;
      size_t ti = std::lower_bound(times.begin(), times.end(), sc[k]) - times.begin();
      outs[ti].push_back(KOut{out[k], 1.0 / std::pow(sc[k], L)});
    }
    std::vector<const double*> b(L + 1, nullptr);
    b[L] = v;
    kiops_run(ctx, os, prec, h, b.data(), L, times, outs, tol, o, stats);
  }
}

// The interval [-safety rho, rho_hi] from a power-iteration estimate.
Interval interval_from_estimate(double rho, int mv, const phix_opts& o, phix_stats& stats) {
  Interval iv{};
  stats.power_mv += mv;
  iv.rho = rho;
  const double alpha = -o.safety * rho, beta = o.rho_hi;
  iv.c = 0.5 * (alpha + beta);
  iv.gamma = 0.25 * (beta - alpha);
  stats.rho = iv.rho;
  return iv;
}

Interval interval_for(phix_ctx* ctx, const OpState& os, int prec, const phix_opts& o, phix_stats& stats) {
  if (o.rho_re > 0) {
    Interval iv{};
    const double alpha = -o.rho_re, beta = o.rho_hi;
    iv.rho = o.rho_re;
    iv.c = 0.5 * (alpha + beta);
    iv.gamma = 0.25 * (beta - alpha);
    stats.rho = iv.rho;
    return iv;
  }
  int mv = 0;
  const double rho = power_iteration(ctx, os, prec, o, &mv);
  return interval_from_estimate(rho, mv, o, stats);
}

void phi_actions(phix_ctx* ctx, const OpState& os, phix_method method, int prec, double h, const double* v,
                 int nout, const int* l, const double* sc, double* const* out, double tol, const phix_opts& o,
                 const Interval* iv, phix_stats& stats) {
  if (method == PHIX_KIOPS) {
    if (o.jv == PHIX_JV_FD) fail(ctx, PHIX_EINVAL, "KIOPS takes the analytic Jacobian only");
    kiops_phi(ctx, os, prec, h, v, nout, l, sc, out, tol, o, stats);
    return;
  }
  Interval own;
  if (!iv) {
    own = interval_for(ctx, os, prec, o, stats);
    iv = &own;
  }
  leja_phi(ctx, os, prec, h, v, nout, l, sc, out, tol, o, *iv, stats);
}

phix_opts resolve_opts(phix_ctx* ctx, const phix_opts* in) {
  phix_opts o;
  phix_opts_default(&o);
  if (in) o = *in;
  if (o.prec < PHIX_FP64 || o.prec > PHIX_FP32) fail(ctx, PHIX_EINVAL, "bad precision %d", (int)o.prec);
  if (o.m_max < 1 || o.m_max > 4000) fail(ctx, PHIX_EINVAL, "m_max must be in 1..4000");
  if (o.m_min < 0) fail(ctx, PHIX_EINVAL, "m_min must be >= 0");
  if (!(o.safety > 0)) fail(ctx, PHIX_EINVAL, "safety must be > 0");
  if (o.power_max_it < 1 || o.power_max_it > 4000) fail(ctx, PHIX_EINVAL, "power_max_it must be in 1..4000");
  if (o.kernel < PHIX_KERNEL_AUTO || o.kernel > PHIX_KERNEL_FUSED2) fail(ctx, PHIX_EINVAL, "unknown kernel %d", o.kernel);
  if (o.profile < 0 || o.profile > 2) fail(ctx, PHIX_EINVAL, "profile must be 0, 1 or 2");
  if (o.kiops_m_max < 2 || o.kiops_m_max > 128) fail(ctx, PHIX_EINVAL, "kiops_m_max must be in 2..128");
  if (o.kiops_fused != 0 && o.kiops_fused != 1) fail(ctx, PHIX_EINVAL, "kiops_fused must be 0 or 1");
  if (o.chain < PHIX_CHAIN_AUTO || o.chain > PHIX_CHAIN_GRAPH) fail(ctx, PHIX_EINVAL, "unknown chain mode %d", o.chain);
  if (o.jv != PHIX_JV_ANALYTIC && o.jv != PHIX_JV_FD) fail(ctx, PHIX_EINVAL, "unknown jv mode %d", o.jv);
  if (o.leja_augmented != 0 && o.leja_augmented != 1) fail(ctx, PHIX_EINVAL, "leja_augmented must be 0 or 1");
  return o;
}

template <typename F>
phix_status guarded(phix_ctx* ctx, phix_stats* stats, F&& body) {
  if (!ctx) return PHIX_EINVAL;
  ctx->err.clear();
  phix_stats st{};
  long l0 = ctx->launches;
  phix_status rc = PHIX_OK;
  for (int attempt = 0; attempt < 2; ++attempt) {
    // a second attempt runs with full-length tables; the body changes none
    // of its inputs before its last flush, so it can run again
    st = phix_stats{};
    ctx->ran_out = false;
    ctx->full_tables = attempt > 0;
    bool rerun = false;
    try {
      rc = body(st);
      flush(ctx);  // outcomes of the passes still queued
      rerun = ctx->ran_out;
    } catch (const Rerun&) {
      rerun = true;
    } catch (const Fail& f) {
      rc = f.st;
      // drop queued passes: their stats target is this call's local record
      (void)cudaStreamSynchronize(ctx->stream);
      ctx->pend.clear();
      ctx->nslot = 0;
    }
    if (!rerun) break;
    rc = PHIX_OK;
  }
  ctx->full_tables = false;
  ctx->ran_out = false;
  if (rc == PHIX_OK && st.status != PHIX_OK) {
    rc = (phix_status)st.status;
    if (ctx->err.empty())
      set_err(ctx, "%s", rc == PHIX_ENOTCONV ? "iteration did not converge within m_max" : "non-finite norm");
  }
  st.status = rc;
  st.launches = (int)(ctx->launches - l0);
  if (stats) *stats = st;
  return rc;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int phix_version(void) { return PHIX_VERSION; }
size_t phix_opts_size(void) { return sizeof(phix_opts); }
size_t phix_stats_size(void) { return sizeof(phix_stats); }

void phix_opts_default(phix_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->prec = PHIX_DF64;
  o->safety = 1.2;
  o->rho_re = -1.0;
  o->rho_hi = 0.0;
  o->rho_im = 0.0;
  o->gamma_cap = 200.0;
  o->iota_cap = 4.0;
  o->m_max = 500;
  o->m_min = 3;
  o->power_max_it = 50;
  o->power_rel = 1e-2;
  o->power_seed = 0x5EED;
  o->kiops_m_init = 16;
  o->kiops_m_max = 64;
  o->kiops_m_step = 8;
  o->kiops_max_substeps = 10000;
  o->kiops_fused = 1;
  o->chain = PHIX_CHAIN_AUTO;
  o->jv = PHIX_JV_ANALYTIC;
  o->leja_augmented = 0;
}

phix_status phix_create(phix_ctx** out, void* stream) {
  if (!out) return PHIX_EINVAL;
  *out = nullptr;
  phix_ctx* ctx = new phix_ctx();
  ctx->stream = static_cast<cudaStream_t>(stream);
  try {
    CK(cudaGetDevice(&ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device));
    ctx->l2_bytes = l2;
    ctx->grid_iter = ctx->nsm * 8;   // upper bound; chains use the occupancy of their kernel
    ctx->grid_stream = ctx->nsm * 8;
    CK(cudaMalloc(&ctx->ctl, sizeof(LejaCtl) * NSLOT));
    CK(cudaMallocHost(&ctx->ctl_h, sizeof(LejaCtl) * NSLOT));
    for (int i = 0; i < 2 * NSLOT + 3; ++i) {  // + one pair for KIOPS, one for the power-iteration read-back
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    CK(cudaMalloc(&ctx->partials, sizeof(double) * (size_t)std::max(ctx->grid_iter, ctx->grid_stream) * (KMAX + 1)));
    CK(cudaMalloc(&ctx->scal, sizeof(double) * 16));
    CK(cudaMallocHost(&ctx->scal_h, sizeof(double) * 16));
    CK(cudaMalloc(&ctx->counter, sizeof(unsigned int)));
    CK(cudaMallocHost(&ctx->kc_h, sizeof(KiopsCtl)));
    {
      void* mb = nullptr;
      CK(cudaHostAlloc(&mb, sizeof(KiopsMailbox), cudaHostAllocMapped));
      ctx->kmb_h = static_cast<KiopsMailbox*>(mb);
      std::memset(mb, 0, sizeof(KiopsMailbox));
      void* md = nullptr;
      CK(cudaHostGetDevicePointer(&md, mb, 0));
      ctx->kmb_d = static_cast<KiopsMailbox*>(md);
    }
    CK(cudaMemset(ctx->counter, 0, sizeof(unsigned int)));
    CK(cudaMemset(ctx->ctl, 0, sizeof(LejaCtl) * NSLOT));
    CK(cudaDeviceSynchronize());
  } catch (const Fail& f) {
    phix_destroy(ctx);
    return f.st;
  }
  *out = ctx;
  return PHIX_OK;
}

phix_status phix_destroy(phix_ctx* ctx) {
  if (!ctx) return PHIX_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < S_NSLOT; ++i)
    if (ctx->buf[i]) cudaFree(ctx->buf[i]);
  if (ctx->ctl) cudaFree(ctx->ctl);
  if (ctx->ctl_h) cudaFreeHost(ctx->ctl_h);
  if (ctx->partials) cudaFree(ctx->partials);
  if (ctx->scal) cudaFree(ctx->scal);
  if (ctx->scal_h) cudaFreeHost(ctx->scal_h);
  if (ctx->counter) cudaFree(ctx->counter);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : ctx->bgraphs) cudaGraphExecDestroy(g.exec);
  if (ctx->ptab_h) cudaFreeHost(ctx->ptab_h);
  if (ctx->ptab_d) cudaFree(ctx->ptab_d);
  if (ctx->kc_h) cudaFreeHost(ctx->kc_h);
  if (ctx->kmb_h) cudaFreeHost(ctx->kmb_h);
  delete ctx;
  return PHIX_OK;
}

const char* phix_last_error(const phix_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

phix_status phix_leja_points(double* xi, int m) {
  if (!xi || m < 1 || m > 4096) return PHIX_EINVAL;
  return leja_points_host(xi, m) == 0 ? PHIX_OK : PHIX_EINVAL;
}

phix_status phix_divided_differences(int l, double a, double b, int m, double* d) {
  if (!d || m < 1 || m > 4096 || l < 0 || l > 20) return PHIX_EINVAL;
  DDTable t;
  t.l = l;
  t.a = a;
  t.b = b;
  t.grow(m);
  std::memcpy(d, t.d.data(), sizeof(double) * m);
  return PHIX_OK;
}


phix_status phix_phi_action_batched(phix_ctx* ctx, const phix_batch_problem* probs, int nprob, int nout,
                                    const int* l, double tol, const phix_opts* opts, int* per_prob,
                                    phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    if (!probs || nprob < 1 || !l || nout < 1 || nout > 3 || !(tol > 0)) fail(ctx, PHIX_EINVAL, "bad batch arguments");
    phix_opts o = resolve_opts(ctx, opts);
    if (o.prec != PHIX_FP64 && o.prec != PHIX_DF64 && o.prec != PHIX_FP32_JV)
      fail(ctx, PHIX_EINVAL, "batched actions support PHIX_FP64, PHIX_DF64, PHIX_FP32_JV");
    if (o.m_max > 500) fail(ctx, PHIX_EINVAL, "batched actions need m_max <= 500");
    for (int k = 0; k < nout; ++k)
      if (l[k] < 0 || l[k] > 2) fail(ctx, PHIX_EINVAL, "batched actions support l in 0..2");
    const size_t pb = batched_prob_bytes();
    std::vector<unsigned char> hp(pb * (size_t)nprob);
    std::vector<std::pair<double, int>> ord(nprob);
    unsigned long long off = 0, key = 1469598103934665603ull;
    for (int i = 0; i < nprob; ++i) {
      const phix_batch_problem& q = probs[i];
      if (q.nx < 3 || q.ny < 3 || !q.v || !(q.rho_re > 0) || !(q.h > 0) || !std::isfinite(q.h))
        fail(ctx, PHIX_EINVAL, "problem %d: bad grid, vector, step or interval", i);
      for (int k = 0; k < nout; ++k)
        if (!q.out[k]) fail(ctx, PHIX_EINVAL, "problem %d: out[%d] is NULL", i, k);
      batched_fill_prob(hp.data() + pb * i, q.nx, q.ny, q.D, q.ax, q.ay, q.h, q.rho_re, q.rho_hi, q.rho_im, q.v,
                        q.out, nout, off);
      const size_t N = (size_t)q.nx * q.ny;
      off += 10 * N;
      ord[i] = std::make_pair(-(double)N * (1.0 + q.h * q.rho_re), i);  // largest work first
      key = (key ^ (unsigned long long)N) * 1099511628211ull;
    }
    std::sort(ord.begin(), ord.end());
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = ord[i].second;
    const size_t eb = 8;
    void* dprob = ws(ctx, S_BPROB, pb * nprob);
    // the order (largest work first) and, after it, a tuning subsample: every
    // 8th problem of that order, which keeps the size and stiffness mix
    const int nsub = nprob >= 512 ? (nprob + 7) / 8 : nprob;
    std::vector<int> sub(nsub);
    for (int i = 0; i < nsub; ++i) sub[i] = order[(size_t)i * nprob / nsub];
    int* dorder = static_cast<int*>(ws(ctx, S_BORDER, sizeof(int) * (size_t)(nprob + nsub)));
    void* arena = ws(ctx, S_BWS, off * eb);
    unsigned int* q = static_cast<unsigned int*>(ws(ctx, S_BQ, sizeof(unsigned int)));
    const int M = o.m_max + 1;
    double* xi = static_cast<double*>(ws(ctx, S_XI, sizeof(double) * M));
    CK(cudaMemcpyAsync(xi, leja_table(M), sizeof(double) * M, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dprob, hp.data(), pb * nprob, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dorder + nprob, sub.data(), sizeof(int) * nsub, cudaMemcpyHostToDevice, ctx->stream));
    key = (key ^ (unsigned long long)o.prec) * 1099511628211ull;
    key = (key ^ (unsigned long long)nprob) * 1099511628211ull;
    using Cfg = phix_ctx::BatchCfg;
    // one graph per (arena, problem table, prec, launch configuration, problem
    // subset): queue reset + persistent launch
    auto graph_for = [&](const Cfg& c, bool subset) -> cudaGraphExec_t {
      const int grid = ctx->nsm * c.per_sm;
      unsigned long long gk = key ^ (unsigned long long)(uintptr_t)arena;
      for (unsigned long long v : {(unsigned long long)c.bt, (unsigned long long)c.smem, (unsigned long long)grid,
                                   (unsigned long long)subset})
        gk = (gk ^ v) * 1099511628211ull;
      for (auto& g : ctx->bgraphs)
        if (g.key == gk && g.grid == grid) return g.exec;
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      cudaError_t e1 = cudaMemsetAsync(q, 0, sizeof(unsigned int), cs);
      cudaError_t e2 = launch_batched(o.prec, dprob, subset ? dorder + nprob : dorder, subset ? nsub : nprob, q, arena,
                                      xi, o.m_max, o.m_min, tol, o.gamma_cap, o.iota_cap, nout, l, grid, c.bt, c.smem,
                                      cs);
      cudaError_t e3 = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      CK(e1);
      CK(e2);
      CK(e3);
      cudaGraphExec_t ex;
      cudaError_t e4 = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      CK(e4);
      if (ctx->bgraphs.size() >= 32) {
        cudaGraphExecDestroy(ctx->bgraphs.front().exec);
        ctx->bgraphs.erase(ctx->bgraphs.begin());
      }
      ctx->bgraphs.push_back(phix_ctx::BatchGraph{gk, grid, ex});
      return ex;
    };
    Cfg cfg;
    bool tuned = false;
    for (auto& t : ctx->btune)
      if (t.first == key) {
        cfg = t.second;
        tuned = true;
      }
    cudaEvent_t ev0, ev1;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    if (o.profile && !tuned) {
      // autotune on the subsample: threads per CTA x shared-memory residency
      // of small passes x CTAs per SM (the resident maximum and half of it)
      float best = 1e30f;
      for (int bt : {256, 512, 1024})
        for (unsigned int sm : {0u, 48u << 10, 100u << 10}) {
          const int occ = std::min(4, batched_blocks_per_sm(o.prec, bt, sm));
          if (occ < 1) continue;
          for (int per : {occ, std::max(1, occ / 2)}) {
            Cfg c;
            c.bt = bt;
            c.smem = sm;
            c.per_sm = per;
            cudaGraphExec_t ex = graph_for(c, true);
            CK(cudaEventRecord(ev0, ctx->stream));
            CK(cudaGraphLaunch(ex, ctx->stream));
            CK(cudaEventRecord(ev1, ctx->stream));
            CK(cudaEventSynchronize(ev1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev0, ev1));
            if (ms < best) {
              best = ms;
              cfg = c;
            }
            if (per == 1) break;
          }
        }
      ctx->btune.push_back(std::make_pair(key, cfg));
    }
    ctx->blast = cfg;
    const int per_sm = cfg.per_sm;
    cudaGraphExec_t ex = graph_for(cfg, false);
    CK(cudaEventRecord(ev0, ctx->stream));
    CK(cudaGraphLaunch(ex, ctx->stream));
    ctx->launches += 1;
    CK(cudaEventRecord(ev1, ctx->stream));
    CK(cudaMemcpyAsync(hp.data(), dprob, pb * nprob, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (o.profile) {
      st.iter_ms = ms;
      st.iter_launches = 1;
    }
    st.substeps = per_sm;  // CTAs per SM used (tuned when profile = 1); phix_batched_config has the rest
    int worst = PHIX_OK;
    for (int i = 0; i < nprob; ++i) {
      int s_, it, sb;
      batched_read_prob(hp.data() + pb * i, &s_, &it, &sb);
      if (per_prob) per_prob[i] = s_;
      st.iters += it;
      st.jv += it;
      st.passes += 1;
      if (s_ != PHIX_OK && worst == PHIX_OK) worst = s_;
    }
    if (worst != PHIX_OK) {
      st.status = worst;
      set_err(ctx, "a batched problem returned status %d", worst);
    }
    return PHIX_OK;
  });
}

phix_status phix_batched_config(const phix_ctx* ctx, int* threads_per_cta, int* smem_bytes, int* ctas_per_sm) {
  if (!ctx) return PHIX_EINVAL;
  if (threads_per_cta) *threads_per_cta = ctx->blast.bt;
  if (smem_bytes) *smem_bytes = (int)ctx->blast.smem;
  if (ctas_per_sm) *ctas_per_sm = ctx->blast.per_sm;
  return PHIX_OK;
}

// blocks of the features reduction: about four points per thread, at most 512
int features_grid(const phix_ctx* ctx, const phix_jop* op) {
  const long long n = (long long)op->nx * op->ny;
  return (int)std::max(1LL, std::min<long long>({(long long)ctx->grid_stream, 512LL, (n + 1023) / 1024}));
}

phix_status phix_features(phix_ctx* ctx, const phix_jop* op, double h, float* feats) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    check_op(ctx, op, true);
    if (op->kind == PHIX_OP_ADVDIFF) fail(ctx, PHIX_EINVAL, "features are defined for Gray-Scott and Burgers");
    if (!feats || !(h > 0)) fail(ctx, PHIX_EINVAL, "bad features arguments");
    unsigned int* cnt = static_cast<unsigned int*>(ws(ctx, S_MCNT, sizeof(unsigned int)));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), ctx->stream));
    KL(launch_features(op->kind, op->nx, op->ny, op->param, h, op->state, ctx->partials, cnt, feats,
                       features_grid(ctx, op), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_learned_targets(phix_ctx* ctx, const phix_jop* op, double h, double rho, const phix_opts* opts,
                                 float* t) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    check_op(ctx, op, true);
    if (op->kind != PHIX_OP_GRAYSCOTT && op->kind != PHIX_OP_BURGERS)
      fail(ctx, PHIX_EINVAL, "targets are defined for Gray-Scott and Burgers");
    if (!t || !(h > 0) || !(rho > 0) || !std::isfinite(rho)) fail(ctx, PHIX_EINVAL, "bad targets arguments");
    const phix_opts o = resolve_opts(ctx, opts);
    const double Dmax = op->kind == PHIX_OP_GRAYSCOTT ? std::max(op->param[0], op->param[1]) : op->param[0];
    const double rho_diff = 4.0 * Dmax * ((double)op->nx * op->nx + (double)op->ny * op->ny);
    double rho_im = 0.0;
    if (op->kind == PHIX_OP_BURGERS) {
      // Bendixson bound of the skew part of J: max|U| (nx + ny)
      CK(cudaMemsetAsync(ctx->scal, 0, sizeof(double), ctx->stream));
      KL(launch_maxabs(op->state, (size_t)op->nx * op->ny, ctx->scal, ctx->grid_stream, ctx->stream));
      CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      rho_im = ctx->scal_h[0] * (double)(op->nx + op->ny);
    }
    // the substep count of a phi_1 action of step h on the interval the Leja
    // path takes from this estimate (the complex-spectrum half-width rule)
    const double gamma = std::max(0.25 * o.safety * rho, 2.0 * rho_im);
    const int s = substeps_for(h, 1.0, gamma, rho_im, o);
    t[0] = (float)std::log(rho / rho_diff);
    t[1] = (float)std::log1p(rho_im / rho_diff);
    t[2] = (float)std::log((double)s);
    return PHIX_OK;
  });
}

phix_status phix_mlp_forward(phix_ctx* ctx, const float* params, const float* X, int n, float* Y) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    if (!params || !X || !Y || n < 1) fail(ctx, PHIX_EINVAL, "bad mlp_forward arguments");
    KL(launch_mlp_forward(params, X, n, Y, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_mlp_grad(phix_ctx* ctx, const float* params, const float* X, const float* T, int n, float* G,
                          float* loss) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    if (!params || !X || !T || !G || n < 1 || n > 65536) fail(ctx, PHIX_EINVAL, "bad mlp_grad arguments");
    float* dl = static_cast<float*>(ws(ctx, S_MY, sizeof(float) * 4));
    KL(launch_mlp_grad(params, X, T, n, G, dl, ctx->stream));
    float hl = 0.f;
    CK(cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = hl;
    return PHIX_OK;
  });
}

phix_status phix_mlp_train(phix_ctx* ctx, float* params, float* m, float* v, int* step, const float* X,
                           const float* T, int n, int batch, int nsteps, float lr, float* loss) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    if (!params || !m || !v || !step || !X || !T || batch < 1 || n < batch || n % batch != 0 || nsteps < 0 ||
        !(lr > 0))
      fail(ctx, PHIX_EINVAL, "bad mlp_train arguments");
    float* G = static_cast<float*>(ws(ctx, S_MG, sizeof(float) * mlp_nparam()));
    float* dl = static_cast<float*>(ws(ctx, S_MY, sizeof(float) * 4));
    const int nb = n / batch;
    for (int s = 0; s < nsteps; ++s) {
      const int b = (*step) % nb;
      KL(launch_mlp_grad(params, X + (size_t)b * batch * PHIX_MLP_NFEAT, T + (size_t)b * batch * 3, batch, G, dl,
                         ctx->stream));
      *step += 1;
      KL(launch_adam(params, m, v, G, *step, lr, ctx->stream));
    }
    float hl = 0.f;
    CK(cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = hl;
    return PHIX_OK;
  });
}

phix_status phix_phi_action_learned(phix_ctx* ctx, const phix_jop* op, double h, const double* v, int nout,
                                    const int* l, const double* scale, double* const* out, double tol,
                                    const float* params, const phix_opts* opts, phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    check_op(ctx, op, true);
    if (op->kind == PHIX_OP_ADVDIFF) fail(ctx, PHIX_EINVAL, "the learned interval is trained for Gray-Scott and Burgers");
    if (!v || !out || !l || !scale || !params || nout < 1 || nout > KMAX || !(h > 0) || !(tol > 0))
      fail(ctx, PHIX_EINVAL, "bad arguments");
    phix_opts o = resolve_opts(ctx, opts);
    float* feats = static_cast<float*>(ws(ctx, S_MFEAT, sizeof(float) * PHIX_MLP_NFEAT));
    float* y = static_cast<float*>(ws(ctx, S_MY, sizeof(float) * 4));
    unsigned int* cnt = static_cast<unsigned int*>(ws(ctx, S_MCNT, sizeof(unsigned int)));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), ctx->stream));
    KL(launch_features(op->kind, op->nx, op->ny, op->param, h, op->state, ctx->partials, cnt, feats,
                       features_grid(ctx, op), ctx->stream));
    KL(launch_mlp_forward(params, feats, 1, y, ctx->stream));
    float yh[3];
    CK(cudaMemcpyAsync(yh, y, sizeof(float) * 3, cudaMemcpyDeviceToHost, ctx->stream));
    OpState os = make_opstate(ctx, op, op->state, o.prec);  // synchronises nothing; stream-ordered
    CK(cudaStreamSynchronize(ctx->stream));
    const double Dmax = op->kind == PHIX_OP_GRAYSCOTT ? std::max(op->param[0], op->param[1]) : op->param[0];
    const double rho_diff = 4.0 * Dmax * ((double)op->nx * op->nx + (double)op->ny * op->ny);
    const double rho = rho_diff * std::exp((double)yh[0]);
    const double rho_im = std::max(0.0, rho_diff * std::expm1((double)yh[1]));
    if (!std::isfinite(rho) || !(rho > 0)) fail(ctx, PHIX_ENAN, "network produced a non-finite interval");
    phix_opts ol = o;
    ol.rho_re = o.safety * rho;
    ol.rho_hi = 0.0;
    ol.rho_im = rho_im;
    Interval iv;
    iv.c = -0.5 * ol.rho_re;
    iv.gamma = 0.25 * ol.rho_re;
    iv.rho = rho;
    st.rho = rho;
    leja_phi(ctx, os, o.prec, h, v, nout, l, scale, out, tol, ol, iv, st);
    flush(ctx);  // the fallback decision needs the passes' outcome
    if (ctx->ran_out) throw Rerun{};
    if (st.status != PHIX_OK) {
      // fallback: the method's own power iteration, then recompute
      st.status = PHIX_OK;
      st.rejections = 1;
      phix_opts of = o;
      of.rho_im = rho_im;
      Interval ivp = interval_for(ctx, os, o.prec, of, st);
      leja_phi(ctx, os, o.prec, h, v, nout, l, scale, out, tol, of, ivp, st);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_small_expm(phix_ctx* ctx, int n, const double* d, const double* u, const double* l,
                            double tau, double* F, int* method) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    if (n < 1 || n > KIOPS_MMAX + 1 || !d || !F || (n > 1 && (!u || !l)) || !std::isfinite(tau))
      fail(ctx, PHIX_EINVAL, "bad small_expm arguments");
    int* md = static_cast<int*>(ws(ctx, S_KMODE, sizeof(int)));
    KL(small_expm_e1(n, d, u, l, tau, F, md, ctx->stream));
    int mh = 0;
    CK(cudaMemcpyAsync(&mh, md, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (method) *method = mh;
    return PHIX_OK;
  });
}

phix_status phix_rhs(phix_ctx* ctx, const phix_jop* op, const double* u, double* f) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    check_op(ctx, op, false);
    if (!u || !f || u == f) fail(ctx, PHIX_EINVAL, "u/f NULL or aliased");
    OpDesc d{};
    d.kind = op->kind;
    d.nx = op->nx;
    d.ny = op->ny;
    for (int i = 0; i < 8; ++i) d.p[i] = op->param[i];
    KL(launch_rhs(d, u, f, ctx->grid_stream, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_spectrum(phix_ctx* ctx, const phix_jop* op, const phix_opts* opts, double* rho,
                          phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    check_op(ctx, op, true);
    if (!rho) fail(ctx, PHIX_EINVAL, "rho is NULL");
    phix_opts o = resolve_opts(ctx, opts);
    OpState os = make_opstate(ctx, op, op->state, o.prec);
    int mv = 0;
    *rho = power_iteration(ctx, os, o.prec, o, &mv);
    st.power_mv = mv;
    st.rho = *rho;
    return PHIX_OK;
  });
}

phix_status phix_phi_action(phix_ctx* ctx, const phix_jop* op, double h, const double* v, int nout,
                            const int* l, const double* scale, double* const* out, double tol,
                            phix_method method, const phix_opts* opts, phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    check_op(ctx, op, true);
    if (!v || !out || !l || !scale) fail(ctx, PHIX_EINVAL, "NULL argument");
    if (nout < 1 || nout > KMAX) fail(ctx, PHIX_EINVAL, "nout must be in 1..%d", KMAX);
    if (!(h >= 0) || !std::isfinite(h)) fail(ctx, PHIX_EINVAL, "h must be finite and >= 0");
    if (!(tol > 0)) fail(ctx, PHIX_EINVAL, "tol must be > 0");
    for (int k = 0; k < nout; ++k) {
      if (l[k] < 0 || l[k] > 8) fail(ctx, PHIX_EINVAL, "l[%d] = %d out of 0..8", k, l[k]);
      if (!(scale[k] > 0)) fail(ctx, PHIX_EINVAL, "scale[%d] must be > 0", k);
      if (!out[k] || out[k] == v) fail(ctx, PHIX_EINVAL, "out[%d] is NULL or aliases v", k);
    }
    phix_opts o = resolve_opts(ctx, opts);
    if (method != PHIX_LEJA && method != PHIX_KIOPS) fail(ctx, PHIX_EINVAL, "unknown method %d", (int)method);
    const int prec = method == PHIX_KIOPS ? kiops_prec(o.prec) : (int)o.prec;
    OpState os = make_opstate(ctx, op, op->state, prec);
    if (h == 0.0) {
      for (int k = 0; k < nout; ++k) lincomb(ctx, os.N, {1.0 / factorial(l[k])}, {v}, out[k]);
      CK(cudaStreamSynchronize(ctx->stream));
      return PHIX_OK;
    }
    phi_actions(ctx, os, method, prec, h, v, nout, l, scale, out, tol, o, nullptr, st);
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_phi_combination(phix_ctx* ctx, const phix_jop* op, double h, const double* const* b,
                                 int p, double* out, double tol, phix_method method,
                                 const phix_opts* opts, phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    check_op(ctx, op, true);
    if (!b || !out) fail(ctx, PHIX_EINVAL, "NULL argument");
    if (p < 0 || p > 8) fail(ctx, PHIX_EINVAL, "p must be in 0..8");
    phix_opts o = resolve_opts(ctx, opts);
    if (method != PHIX_LEJA && method != PHIX_KIOPS) fail(ctx, PHIX_EINVAL, "unknown method %d", (int)method);
    for (int j = 0; j <= p; ++j)
      if (b[j] && b[j] == out) fail(ctx, PHIX_EINVAL, "out aliases b[%d]", j);
    if (method == PHIX_KIOPS) {
      // one augmented Krylov run (Theorem of Sec. 2.1)
      OpState os = make_opstate(ctx, op, op->state, kiops_prec(o.prec));
      std::vector<std::vector<KOut>> outs(1, std::vector<KOut>(1, KOut{out, 1.0}));
      kiops_run(ctx, os, o.prec, h, b, p, std::vector<double>(1, 1.0), outs, tol, o, st);
      CK(cudaStreamSynchronize(ctx->stream));
      return PHIX_OK;
    }
    OpState os = make_opstate(ctx, op, op->state, o.prec);
    if (o.leja_augmented) {
      // exp of the augmented matrix of the Theorem of Sec. 2.1 by one Leja
      // pass (Appendix A): start vector [b_0; e_p], interval h [alpha, 0]
      Interval iv = interval_for(ctx, os, o.prec, o, st);
      GenAug aug;
      aug.hgamma = h * iv.gamma;
      aug.hc = h * iv.c;
      double* zero = wsd(ctx, S_GZ, os.N);
      CK(cudaMemsetAsync(zero, 0, os.N * sizeof(double), ctx->stream));
      bool any = false;
      for (int j = 1; j <= p; ++j) {
        aug.src.push_back(b[j] ? b[j] : zero);  // a NULL b_j is a zero column
        any = any || b[j];
      }
      if (!any) aug.src.clear();
      const double* b0 = b[0] ? b[0] : zero;
      if (aug.src.empty() && p > 0) {  // only b_0: a plain phi_0 pass
        p = 0;
      }
      int l0 = 0;
      const double a0 = h * iv.c, g0 = h * iv.gamma;
      const std::vector<std::vector<double>> d = pass_tables(ctx, 1, &l0, &a0, &g0, tol, o);
      std::vector<const std::vector<double>*> dp(1, &d[0]);
      double* outs[1] = {out};
      phix_opts og = o;
      og.jv = o.jv;
      general_pass(ctx, os, b0, 1, dp, iv.c, iv.gamma, tol, og, outs, st, p > 0 ? &aug : nullptr);
      CK(cudaStreamSynchronize(ctx->stream));
      return PHIX_OK;
    }
    CK(cudaMemsetAsync(out, 0, os.N * sizeof(double), ctx->stream));
    Interval iv = interval_for(ctx, os, o.prec, o, st);
    double* tmp = wsd(ctx, S_O3, os.N);
    for (int j = 0; j <= p; ++j) {
      if (!b[j]) continue;
      if (b[j] == out) fail(ctx, PHIX_EINVAL, "out aliases b[%d]", j);
      int lj = j;
      double s1 = 1.0;
      double* outs[1] = {tmp};
      leja_phi(ctx, os, o.prec, h, b[j], 1, &lj, &s1, outs, tol, o, iv, st);
      lincomb(ctx, os.N, {1.0, 1.0}, {out, tmp}, out);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PHIX_OK;
  });
}

// One step of an exponential integrator of Sec. 5 (the driver of every
// scheme; `scheme` selects the stage program).  The phi-functions are grouped
// as Sec. 5 describes per scheme and method: Leja evaluates the terms acting
// on f(u) h in one vertical pass and the rest individually; KIOPS evaluates
// the internal stages vertically (output times of one run) and the solution
// stages of EPIRK4s3, EPIRK4s3A and EXPRB53s3 as one horizontal combination
// (Theorem of Sec. 2.1); LeKry takes the internal stages (and the error term
// of the EPIRK4 family) by Leja and the combinations by KIOPS.
// uh != NULL: the state is in HOST memory: it is copied in, stepped, and
// copied back (on success) before the call returns.
static phix_status exp_step(phix_ctx* ctx, int scheme, const phix_jop* op, double* u_in, double* uh, double h,
                            double tol, phix_method method, const phix_opts* opts, double* err_est,
                            phix_stats* stats) {
  return guarded(ctx, stats, [&](phix_stats& st) -> phix_status {
    check_op(ctx, op, false);
    if (!u_in && !uh) fail(ctx, PHIX_EINVAL, "u_inout is NULL");
    if (!(h > 0) || !std::isfinite(h)) fail(ctx, PHIX_EINVAL, "h must be finite and > 0");
    if (!(tol > 0)) fail(ctx, PHIX_EINVAL, "tol must be > 0");
    if (scheme < PHIX_EXPRB43 || scheme > PHIX_EPIRK5P1) fail(ctx, PHIX_EINVAL, "unknown scheme %d", scheme);
    phix_opts o = resolve_opts(ctx, opts);
    if (method != PHIX_LEJA && method != PHIX_KIOPS && method != PHIX_LEKRY)
      fail(ctx, PHIX_EINVAL, "unknown method %d", (int)method);
    if (method == PHIX_LEKRY && (scheme == PHIX_EXPRB43 || scheme == PHIX_EPIRK5P1))
      fail(ctx, PHIX_EINVAL, "scheme %d has no LeKry form (no linear combination of phi-functions)", scheme);
    if (method == PHIX_LEKRY && o.prec != PHIX_FP64 && o.prec != PHIX_DF64)
      fail(ctx, PHIX_EINVAL, "LeKry needs prec PHIX_FP64 or PHIX_DF64 (one state format for both methods)");
    // iteration arithmetic: KIOPS runs float64 or double-float
    const int prec = method == PHIX_KIOPS ? kiops_prec(o.prec) : (int)o.prec;
    const phix_method inner = method == PHIX_KIOPS ? PHIX_KIOPS : PHIX_LEJA;  // internal stages
    const size_t N = (size_t)op->nx * op->ny * ncomp_of(op->kind);
    double* u = u_in;
    if (uh) {
      u = wsd(ctx, S_UH, N);
      CK(cudaMemcpyAsync(u, uh, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    OpState os = make_opstate(ctx, op, u, prec);
    double* F = wsd(ctx, S_F, N);
    double* FH = wsd(ctx, S_FH, N);
    double* A = wsd(ctx, S_A, N);
    double* B = wsd(ctx, S_B, N);
    double* RA = wsd(ctx, S_RA, N);
    double* RB = wsd(ctx, S_RB, N);
    double* T0 = wsd(ctx, S_T0, N);
    double* Q = wsd(ctx, S_Q, N);
    double* T3 = wsd(ctx, S_T3, N);
    double* T4 = wsd(ctx, S_T4, N);
    double* P1 = wsd(ctx, S_O1, N);
    double* P2 = wsd(ctx, S_O2, N);
    double* P3 = wsd(ctx, S_O3, N);
    double* O4 = wsd(ctx, S_O4, N);
    double* O5 = wsd(ctx, S_O5, N);
    double* O6 = wsd(ctx, S_O6, N);
    // the power iteration first, then f(u) and h f(u) (which do not need the
    // estimate) run on the device while the host reads the estimate and
    // builds the first pass's coefficient tables
    Interval ivv{};
    const bool split = method != PHIX_KIOPS && !(o.rho_re > 0) && !general_kind(os.d.kind) && o.jv != PHIX_JV_FD;
    const int pslot = split ? power_iteration_split(ctx, os, prec, o) : -1;
    KL(launch_rhs(os.d, u, F, ctx->grid_stream, ctx->stream));
    lincomb(ctx, N, {h}, {F}, FH);
    if (split) {
      int mv = 0;
      const double rho = power_iteration_collect(ctx, pslot, &mv);
      ivv = interval_from_estimate(rho, mv, o, st);
    } else if (method != PHIX_KIOPS) {
      ivv = interval_for(ctx, os, prec, o, st);
    }
    const Interval* iv = method != PHIX_KIOPS ? &ivv : nullptr;
    // phi_{l_k}(s_k h J) x for up to four outputs, by `how` (Leja vertical or KIOPS output times)
    auto vert = [&](phix_method how, const double* x, std::vector<int> l, std::vector<double> s,
                    std::vector<double*> out) {
      phi_actions(ctx, os, how, prec, h, x, (int)l.size(), l.data(), s.data(), out.data(), tol, o,
                  how == PHIX_LEJA ? iv : nullptr, st);
    };
    // sum_j phi_j(hJ) b_j by one KIOPS run (Theorem of Sec. 2.1)
    auto horiz = [&](std::vector<const double*> b, double* out) {
      std::vector<std::vector<KOut>> outs(1, std::vector<KOut>(1, KOut{out, 1.0}));
      kiops_run(ctx, os, prec, h, b.data(), (int)b.size() - 1, std::vector<double>(1, 1.0), outs, tol, o, st);
    };
    auto remainder = [&](const double* x, double* R) {
      KL(launch_remainder(os.d, u, x, R, ctx->grid_stream, ctx->stream));
    };
    // the step: u_new = u + sum_i cn[i] xn[i]; error estimate ||sum_i ce[i] xe[i]||
    std::vector<double> cn, ce;
    std::vector<const double*> xn, xe;
    if (scheme == PHIX_EXPRB43) {
      // Eq. (exprb43)
      vert(method, FH, {1, 1}, {0.5, 1.0}, {P1, P2});
      lincomb(ctx, N, {1.0, 0.5}, {u, P1}, A);                 // a = u + 1/2 phi_1(h/2 J) f h
      remainder(A, RA);
      lincomb(ctx, N, {h}, {RA}, T0);
      vert(method, T0, {1}, {1.0}, {Q});
      lincomb(ctx, N, {1.0, 1.0, 1.0}, {u, P2, Q}, B);         // b = u + phi_1 f h + phi_1 R(a) h
      remainder(B, RB);
      lincomb(ctx, N, {16.0 * h, -2.0 * h}, {RA, RB}, T0);
      vert(method, T0, {3}, {1.0}, {T3});
      lincomb(ctx, N, {-48.0 * h, 12.0 * h}, {RA, RB}, T0);
      vert(method, T0, {4}, {1.0}, {T4});
      cn = {1.0, 1.0, 1.0};
      xn = {P2, T3, T4};                                        // u4 = u + phi_1 f h + T3 + T4
      ce = {1.0};
      xe = {T4};                                                // u4 - u3
    } else if (scheme == PHIX_EPIRK4S3 || scheme == PHIX_EPIRK4S3A) {
      // Eq. (epirk4s3) / Eq. (epirk4s3a): one structure, their coefficients
      const bool a4 = scheme == PHIX_EPIRK4S3A;
      const double ca = a4 ? 0.5 : 1.0 / 8.0, cb = a4 ? 2.0 / 3.0 : 1.0 / 9.0;
      // w3 = 1892 Ra + 1458 (Rb - 2 Ra) | 32 Ra - 27/2 Rb ;  w4 = -42336 Ra - 34992 (Rb - 2 Ra) | -144 Ra + 81 Rb
      const double w3a = a4 ? 32.0 : 1892.0 - 2.0 * 1458.0, w3b = a4 ? -13.5 : 1458.0;
      const double w4a = a4 ? -144.0 : -42336.0 + 2.0 * 34992.0, w4b = a4 ? 81.0 : -34992.0;
      if (method == PHIX_LEJA)
        vert(PHIX_LEJA, FH, {1, 1, 1}, {ca, cb, 1.0}, {P1, P3, P2});
      else
        vert(inner, FH, {1, 1}, {ca, cb}, {P1, P3});
      lincomb(ctx, N, {1.0, ca}, {u, P1}, A);
      lincomb(ctx, N, {1.0, cb}, {u, P3}, B);
      remainder(A, RA);
      remainder(B, RB);
      lincomb(ctx, N, {w3a * h, w3b * h}, {RA, RB}, T0);
      if (method == PHIX_LEJA) {
        vert(PHIX_LEJA, T0, {3}, {1.0}, {T3});
        cn = {1.0, 1.0, 1.0};
        xn = {P2, T3, T4};
      } else {
        horiz({nullptr, FH, nullptr, T0}, T3);                  // u3 - u = phi_1 f h + phi_3 w3 h
        cn = {1.0, 1.0};
        xn = {T3, T4};
      }
      lincomb(ctx, N, {w4a * h, w4b * h}, {RA, RB}, T0);
      vert(method == PHIX_KIOPS ? PHIX_KIOPS : PHIX_LEJA, T0, {4}, {1.0}, {T4});
      ce = {1.0};
      xe = {T4};
    } else if (scheme == PHIX_EXPRB53S3) {
      // Eq. (exprb5s3)
      if (method == PHIX_LEJA)
        vert(PHIX_LEJA, FH, {1, 1, 1}, {0.5, 0.9, 1.0}, {P1, P3, P2});
      else
        vert(inner, FH, {1, 1}, {0.5, 0.9}, {P1, P3});
      lincomb(ctx, N, {1.0, 0.5}, {u, P1}, A);                 // a = u + 1/2 phi_1(h/2 J) f h
      remainder(A, RA);
      lincomb(ctx, N, {h}, {RA}, T0);
      vert(inner, T0, {3, 3}, {0.5, 0.9}, {Q, O4});
      // b = u + 9/10 phi_1(9h/10 J) f h + (27/25 phi_3(h/2 J) + 729/125 phi_3(9h/10 J)) R(a) h
      lincomb(ctx, N, {1.0, 0.9, 27.0 / 25.0, 729.0 / 125.0}, {u, P3, Q, O4}, B);
      remainder(B, RB);
      if (method == PHIX_LEJA) {
        lincomb(ctx, N, {2.0 * h, (150.0 / 81.0) * h}, {RA, RB}, T0);
        vert(PHIX_LEJA, T0, {3}, {1.0}, {T3});
        lincomb(ctx, N, {18.0 * h, (-250.0 / 81.0) * h}, {RA, RB}, T0);
        vert(PHIX_LEJA, T0, {3}, {1.0}, {T4});
        lincomb(ctx, N, {-60.0 * h, (500.0 / 27.0) * h}, {RA, RB}, T0);
        vert(PHIX_LEJA, T0, {4}, {1.0}, {O5});
        cn = {1.0, 1.0, 1.0};
        xn = {P2, T4, O5};                                      // u5 = u + phi_1 f h + T4 + O5
        ce = {1.0, 1.0, -1.0};
        xe = {T4, O5, T3};                                      // u5 - u3
      } else {
        lincomb(ctx, N, {2.0 * h, (150.0 / 81.0) * h}, {RA, RB}, T0);
        horiz({nullptr, FH, nullptr, T0}, T3);                  // u3 - u
        lincomb(ctx, N, {18.0 * h, (-250.0 / 81.0) * h}, {RA, RB}, T0);
        lincomb(ctx, N, {-60.0 * h, (500.0 / 27.0) * h}, {RA, RB}, O6);
        horiz({nullptr, FH, nullptr, T0, O6}, T4);              // u5 - u
        cn = {1.0};
        xn = {T4};
        ce = {1.0, -1.0};
        xe = {T4, T3};
      }
    } else {
      // EPIRK5P1, Eq. (epirk5p1) and its coefficient table: three vertical passes
      const double a11 = 0.35129592695058193092, a21 = 0.84405472011657126298, a22 = 1.6905891609568963624;
      const double b1 = 1.0, b2 = 1.2727127317356892397, b3 = 2.2714599265422622275;
      const double g11 = 0.35129592695058193092, g21 = 0.84405472011657126298, g22 = 0.5, g31 = 1.0;
      const double g32 = 0.71111095364366870359, g32h = 0.5, g33 = 0.62378111953371494809, g33h = 1.0;
      vert(method, FH, {1, 1, 1}, {g11, g21, g31}, {P1, P3, P2});
      lincomb(ctx, N, {1.0, a11}, {u, P1}, A);
      remainder(A, RA);
      lincomb(ctx, N, {h}, {RA}, T0);
      vert(method, T0, {1, 1, 1}, {g22, g32h, g32}, {Q, O4, O5});
      lincomb(ctx, N, {1.0, a21, a22}, {u, P3, Q}, B);
      remainder(B, RB);
      lincomb(ctx, N, {-2.0 * h, h}, {RA, RB}, T0);
      vert(method, T0, {3, 3}, {g33, g33h}, {T3, T4});
      cn = {b1, b2, b3};
      xn = {P2, O5, T3};                                        // u5
      ce = {b2, b3, -b2, -b3};
      xe = {O5, T3, O4, T4};                                    // u5 - u4
    }
    // err = ||u_high - u_low||
    const double* ev = xe[0];
    if (xe.size() > 1 || ce[0] != 1.0) {
      lincomb(ctx, N, ce, xe, O6);
      ev = O6;
    }
    KL(launch_norm2(N, ev, nullptr, ctx->partials, ctx->counter, ctx->scal, ctx->grid_stream, ctx->stream));
    CK(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    flush(ctx);  // u changes only when every pass succeeded
    if (ctx->ran_out) throw Rerun{};
    if (st.status == PHIX_OK) {
      cn.insert(cn.begin(), 1.0);
      xn.insert(xn.begin(), u);
      lincomb(ctx, N, cn, xn, u);
      if (uh) CK(cudaMemcpyAsync(uh, u, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    st.err_est = std::sqrt(ctx->scal_h[0]);
    if (err_est) *err_est = st.err_est;
    return PHIX_OK;
  });
}

phix_status phix_exprb43_step(phix_ctx* ctx, const phix_jop* op, double* u_inout, double h, double tol,
                              phix_method method, const phix_opts* opts, double* err_est,
                              phix_stats* stats) {
  return exp_step(ctx, PHIX_EXPRB43, op, u_inout, nullptr, h, tol, method, opts, err_est, stats);
}

phix_status phix_epirk4s3_step(phix_ctx* ctx, const phix_jop* op, double* u_inout, double h, double tol,
                               phix_method method, const phix_opts* opts, double* err_est,
                               phix_stats* stats) {
  return exp_step(ctx, PHIX_EPIRK4S3, op, u_inout, nullptr, h, tol, method, opts, err_est, stats);
}

phix_status phix_step(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u_inout, double h, double tol,
                      phix_method method, const phix_opts* opts, double* err_est, phix_stats* stats) {
  return exp_step(ctx, (int)scheme, op, u_inout, nullptr, h, tol, method, opts, err_est, stats);
}

phix_status phix_step_host(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u_host_inout, double h,
                           double tol, phix_method method, const phix_opts* opts, double* err_est,
                           phix_stats* stats) {
  return exp_step(ctx, (int)scheme, op, nullptr, u_host_inout, h, tol, method, opts, err_est, stats);
}

// ---- automatic step-size control (Sec. 2.3) --------------------------------
static double cost_factor(double c_n, double c_prev, double dt_n, double dt_prev) {
  const double alpha = 0.65241444, beta = 0.26862269, lambda = 1.37412002, delta = 0.64446017;
  const double den = std::log(dt_n) - std::log(dt_prev);
  const double D = std::fabs(den) < 1e-14 ? 0.0 : (std::log(c_n) - std::log(c_prev)) / den;
  const double sf = std::exp(-alpha * std::tanh(beta * D));
  if (sf >= 1.0 && sf < lambda) return lambda;
  if (sf >= delta && sf < 1.0) return delta;
  return sf;
}

phix_status phix_integrate(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u, const phix_adapt* ad,
                           phix_method method, const phix_opts* opts, double* dts, phix_adapt_stats* stats) {
  phix_adapt_stats as{};
  auto finish = [&](phix_status rc) {
    as.status = rc;
    if (stats) *stats = as;
    return rc;
  };
  if (!ctx) return finish(PHIX_EINVAL);
  double* backup = nullptr;
  size_t N = 0;
  phix_status rc = guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    check_op(ctx, op, false);
    if (!u || !ad) fail(ctx, PHIX_EINVAL, "u_inout or adapt is NULL");
    if (!(ad->t_end > 0) || !(ad->dt0 > 0) || !(ad->tol > 0) || ad->max_steps < 1 ||
        (ad->controller != PHIX_CONTROL_TRADITIONAL && ad->controller != PHIX_CONTROL_COST))
      fail(ctx, PHIX_EINVAL, "bad phix_adapt (t_end, dt0, tol > 0; max_steps >= 1; controller)");
    if (scheme < PHIX_EXPRB43 || scheme > PHIX_EPIRK5P1) fail(ctx, PHIX_EINVAL, "unknown scheme %d", (int)scheme);
    N = (size_t)op->nx * op->ny * ncomp_of(op->kind);
    backup = wsd(ctx, S_UB, N);
    return PHIX_OK;
  });
  if (rc != PHIX_OK) return finish(rc);
  const int order = scheme == PHIX_EPIRK5P1 ? 4 : 3;  // of the embedded estimate
  const double itol = ad->iter_tol > 0 ? ad->iter_tol : ad->tol;
  double t = 0.0, dt = ad->dt0;
  double hist_c[2] = {0, 0}, hist_dt[2] = {0, 0};
  long long spent = 0;
  int nhist = 0;
  while (t < ad->t_end * (1 - 1e-14)) {
    if (as.accepted + as.rejected >= ad->max_steps) {
      as.t = t;
      set_err(ctx, "max_steps reached at t = %g", t);
      return finish(PHIX_ENOTCONV);
    }
    dt = std::min(dt, ad->t_end - t);
    if (ad->dt_max > 0) dt = std::min(dt, ad->dt_max);
    if (cudaMemcpyAsync(backup, u, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
      set_err(ctx, "step backup copy failed");
      return finish(PHIX_ECUDA);
    }
    double en = 0.0;
    phix_stats st{};
    rc = exp_step(ctx, (int)scheme, op, u, nullptr, dt, itol, method, opts, &en, &st);
    spent += st.jv + st.power_mv;
    as.matvecs += st.jv + st.power_mv;
    if (rc != PHIX_OK && rc != PHIX_ENOTCONV) return finish(rc);
    const double err = en / std::sqrt((double)N);
    const double dt_trad = err == 0.0 ? HUGE_VAL : dt * std::pow(ad->tol / err, 1.0 / (order + 1));
    if (rc != PHIX_OK || err > ad->tol) {
      // rejected: the step changed u only if its phi-actions succeeded
      if (rc == PHIX_OK &&
          cudaMemcpyAsync(u, backup, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
        set_err(ctx, "step restore copy failed");
        return finish(PHIX_ECUDA);
      }
      as.rejected += 1;
      dt = rc == PHIX_OK ? 0.9 * dt_trad : 0.5 * dt;  // the retry aims below tol
      continue;
    }
    t += dt;
    if (dts) dts[as.accepted] = dt;
    as.accepted += 1;
    hist_c[0] = hist_c[1];
    hist_dt[0] = hist_dt[1];
    hist_c[1] = (double)spent / dt;
    hist_dt[1] = dt;
    ++nhist;
    spent = 0;
    double nxt = dt_trad;
    if (ad->controller == PHIX_CONTROL_COST && nhist >= 2)
      nxt = std::min(nxt, dt * cost_factor(hist_c[1], hist_c[0], hist_dt[1], hist_dt[0]));
    else if (std::isinf(nxt))
      nxt = dt;
    dt = nxt;
  }
  as.t = t;
  as.dt_next = dt;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return finish(PHIX_ECUDA);
  return finish(PHIX_OK);
}

// ---- domain-decomposed Newton-Leja pass: the per-block kernels -------------
static phix_status block_check(phix_ctx* ctx, const phix_block* b) {
  if (!b) fail(ctx, PHIX_EINVAL, "block is NULL");
  if (b->kind < 0 || b->kind > 2) fail(ctx, PHIX_EINVAL, "unknown operator kind %d", b->kind);
  if (b->gnx < 3 || b->gny < 3 || b->bx < 1 || b->by < 1 || b->x0 < 0 || b->y0 < 0 ||
      b->x0 + b->bx > b->gnx || b->y0 + b->by > b->gny)
    fail(ctx, PHIX_EINVAL, "block %dx%d at (%d, %d) does not fit the %dx%d grid", b->bx, b->by, b->x0, b->y0, b->gnx,
         b->gny);
  return PHIX_OK;
}

phix_status phix_block_newton(phix_ctx* ctx, const phix_block* blk, const double* y_in, double* y_out, int K,
                              double* const* p, const double* dk, double a, double b, double* norms) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    block_check(ctx, blk);
    if (!y_in || !norms || K < 0 || K > KMAX || (K > 0 && (!p || !dk)))
      fail(ctx, PHIX_EINVAL, "bad arguments (y_in, norms, K in 0..%d, p and dk for K > 0)", KMAX);
    for (int k = 0; k < K; ++k)
      if (!p[k]) fail(ctx, PHIX_EINVAL, "p[%d] is NULL", k);
    if (blk->kind != PHIX_OP_ADVDIFF && !blk->state) fail(ctx, PHIX_EINVAL, "operator kind %d needs a state", blk->kind);
    double k8[8];
    uniform_coeffs(blk->kind, blk->gnx, blk->gny, blk->param, k8);
    KL(launch_block_newton(blk->kind, blk->bx, blk->by, ncomp_of(blk->kind), K, y_in, y_out, p, blk->state, k8, dk, a,
                           b, ctx->partials, ctx->counter, norms, ctx->grid_stream, ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_block_faces(phix_ctx* ctx, const phix_block* blk, int dir, double* y_pad, double* faces) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    block_check(ctx, blk);
    if (!y_pad || !faces || (dir != 0 && dir != 1)) fail(ctx, PHIX_EINVAL, "bad arguments");
    KL(launch_block_faces(blk->bx, blk->by, ncomp_of(blk->kind), dir, y_pad, faces, ctx->stream));
    return PHIX_OK;
  });
}

phix_status phix_block_start(phix_ctx* ctx, const phix_block* blk, uint64_t seed, double* y_pad) {
  return guarded(ctx, nullptr, [&](phix_stats&) -> phix_status {
    block_check(ctx, blk);
    if (!y_pad) fail(ctx, PHIX_EINVAL, "y_pad is NULL");
    KL(launch_block_splitmix(blk->bx, blk->by, ncomp_of(blk->kind), blk->gnx, blk->gny, blk->x0, blk->y0, seed, y_pad,
                             ctx->grid_stream, ctx->stream));
    return PHIX_OK;
  });
}

int phix_leja_stop(int K, int m, int m_min, const double* dkm, double tol, double ysq, const double* psq) {
  if (!std::isfinite(ysq)) return -1;
  bool ok = m >= m_min;
  for (int k = 0; k < K; ++k) {
    if (!std::isfinite(psq[k])) return -1;
    ok = ok && std::fabs(dkm[k]) * std::sqrt(ysq) <= tol * std::sqrt(psq[k]);
  }
  return ok ? 1 : 0;
}

}  // extern "C"
