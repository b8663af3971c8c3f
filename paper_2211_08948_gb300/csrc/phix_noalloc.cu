// phix_phi_action_noalloc: the Leja phi-action for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc or any allocating routine: a host
// application that hands the whole device to its own memory pool and forbids
// outside allocations, a code running under a hard device-memory budget, or a
// latency-critical loop that cannot afford the device-wide synchronisation an
// allocation may cause.  This entry point creates no context and allocates
// nothing: its scratch (control block, reduction partials, the Newton basis
// pair, the accumulators and the Jacobian state arrays) lives in the fixed
// file-scope array below, which every GPU that loads the library holds until
// the process exits.  The caller still provides the input and output vectors.
#include <cmath>
#include <cstring>
#include <mutex>

#include "phix_internal.h"

using namespace phix;

namespace {

// The scratch itself.  In host code `noalloc_scratch` names a host-side
// stand-in, not device memory: kernels must be given the device address
// obtained from cudaGetSymbolAddress (below), never the symbol itself.
static __device__ __align__(256) unsigned char noalloc_scratch[PHIX_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
constexpr int MAX_GRID = 2048;
constexpr size_t CTL_BYTES = 256;
constexpr size_t PARTIAL_BYTES = sizeof(double) * MAX_GRID * (KMAX + 1);

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;  // device address of noalloc_scratch
  int nsm = 0;
};
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_mu;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t PTAB_MAX = ptab_bytes(PHIX_NOALLOC_MMAX + 1);  // parameter block of the longest chain

// The fixed part of the scratch (control block, partials, parameter block),
// as the header states it.
static_assert(CTL_BYTES + align256(PARTIAL_BYTES) + align256(PTAB_MAX) == PHIX_NOALLOC_OVERHEAD_BYTES,
              "PHIX_NOALLOC_OVERHEAD_BYTES must match the scratch layout");

// Host staging of one call: the parameter block and the coefficient tables.
// Thread-local (one per host thread, in static storage rather than on the
// stack), so calls from several host threads do not share it.
struct HostStage {
  alignas(16) unsigned char ptab[PTAB_MAX];
  double d[KMAX][PHIX_NOALLOC_MMAX + 1];
  double beta[PHIX_NOALLOC_MMAX + 1];
};
thread_local HostStage g_stage;

// Once per device, with that device current: the scratch's device address.
phix_status setup_device(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return PHIX_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess) {
      (void)cudaGetLastError();
      return PHIX_ECUDA;
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      return PHIX_ECUDA;
    }
    (void)leja_table(PHIX_NOALLOC_MMAX + 1);  // host Leja table built once here
    s.scratch = static_cast<unsigned char*>(p);
    s.nsm = nsm;
    s.done = true;
  }
  *out = &s;
  return PHIX_OK;
}

struct Ctl {
  cudaStream_t st;
  LejaCtl* ctl;
  LejaCtl h;  // pageable host copy (no pinned allocation)
};

bool read_ctl(Ctl& c) {
  if (cudaMemcpyAsync(&c.h, c.ctl, sizeof(LejaCtl), cudaMemcpyDeviceToHost, c.st) != cudaSuccess) return false;
  return cudaStreamSynchronize(c.st) == cudaSuccess;
}

}  // namespace

extern "C" phix_status phix_phi_action_noalloc(const phix_jop* op, double h, const double* v, int nout,
                                               const int* l, const double* scale, double* const* out,
                                               double tol, const phix_opts* opts, void* cuda_stream,
                                               phix_stats* stats) {
  phix_stats st;
  std::memset(&st, 0, sizeof st);
  auto finish = [&](phix_status rc) {
    st.status = rc;
    if (stats) *stats = st;
    return rc;
  };
  // ---- arguments ---------------------------------------------------------
  if (!op || !v || !l || !scale || !out || nout < 1 || nout > KMAX) return finish(PHIX_EINVAL);
  if (op->kind < 0 || op->kind > 2 || op->nx < 3 || op->ny < 3) return finish(PHIX_EINVAL);
  if (op->kind != PHIX_OP_ADVDIFF && !op->state) return finish(PHIX_EINVAL);
  if (!(h > 0) || !std::isfinite(h) || !(tol > 0)) return finish(PHIX_EINVAL);
  phix_opts o;
  phix_opts_default(&o);
  if (opts) o = *opts;
  if (o.prec < PHIX_FP64 || o.prec > PHIX_FP32 || o.m_max < 1 || o.m_max > PHIX_NOALLOC_MMAX || o.m_min < 0 ||
      !(o.safety > 0) || o.power_max_it < 1)
    return finish(PHIX_EINVAL);
  for (int k = 0; k < nout; ++k) {
    if (l[k] < 0 || l[k] > 8 || !(scale[k] > 0) || !out[k] || out[k] == v) return finish(PHIX_EINVAL);
  }
  const int prec = o.prec;
  const int ncomp = op->kind == PHIX_OP_GRAYSCOTT ? 2 : 1;
  const size_t plane = (size_t)op->nx * op->ny;
  const size_t N = plane * ncomp;
  const size_t eb = prec == P_FP32 ? 4 : 8;
  const size_t sb = (prec == P_FP64 || prec == P_DF64) ? 8 : 4;
  const size_t st_planes = op->kind == PHIX_OP_GRAYSCOTT ? 2 : (op->kind == PHIX_OP_BURGERS ? 1 : 0);
  // scratch layout: control block | partials | parameter block | y0 | y1 | p_0..p_{K-1} | state planes
  const size_t vec = align256(N * eb);
  const size_t ptb = align256(PTAB_MAX);
  const size_t need = CTL_BYTES + align256(PARTIAL_BYTES) + ptb + (2 + (size_t)nout) * vec +
                      align256(st_planes * plane * sb);
  if (need > (size_t)PHIX_NOALLOC_SCRATCH_BYTES) return finish(PHIX_ETOOBIG);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return finish(PHIX_ECUDA);
  DeviceSetup* ds = nullptr;
  phix_status rc = setup_device(dev, &ds);
  if (rc != PHIX_OK) return finish(rc);

  unsigned char* base = ds->scratch;
  Ctl c;
  c.st = static_cast<cudaStream_t>(cuda_stream);
  c.ctl = reinterpret_cast<LejaCtl*>(base);
  double* partials = reinterpret_cast<double*>(base + CTL_BYTES);
  unsigned char* ptab = base + CTL_BYTES + align256(PARTIAL_BYTES);
  unsigned char* q = ptab + ptb;
  void* y[2] = {q, q + vec};
  void* p[KMAX] = {};
  for (int k = 0; k < nout; ++k) p[k] = q + (2 + k) * vec;
  void* stp = st_planes ? (void*)(q + (2 + nout) * vec) : nullptr;
  const int grid = std::min(MAX_GRID, ds->nsm * 4);
  const int grid_stream = grid;

  // ---- operator coefficients ---------------------------------------------
  const double idx2 = (double)op->nx * op->nx, idy2 = (double)op->ny * op->ny;
  const double* pa = op->param;
  double kJ[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nscaled = 5;
  if (op->kind == PHIX_OP_ADVDIFF) {
    kJ[0] = pa[0] * idx2 + 0.5 * pa[1] * op->nx;
    kJ[1] = pa[0] * idx2 - 0.5 * pa[1] * op->nx;
    kJ[2] = pa[0] * idy2 + 0.5 * pa[2] * op->ny;
    kJ[3] = pa[0] * idy2 - 0.5 * pa[2] * op->ny;
    kJ[4] = -2.0 * pa[0] * (idx2 + idy2);
  } else if (op->kind == PHIX_OP_GRAYSCOTT) {
    kJ[0] = pa[0] * idx2;
    kJ[1] = pa[0] * idy2;
    kJ[2] = -2.0 * pa[0] * (idx2 + idy2) - pa[2];
    kJ[3] = pa[1] * idx2;
    kJ[4] = pa[1] * idy2;
    kJ[5] = -2.0 * pa[1] * (idx2 + idy2) - (pa[2] + pa[3]);
    nscaled = 6;
  } else {
    kJ[0] = pa[0] * idx2;
    kJ[1] = pa[0] * idy2;
    kJ[2] = -2.0 * pa[0] * (idx2 + idy2);
    kJ[3] = 0.5 * op->nx;
    kJ[4] = 0.5 * op->ny;
    nscaled = 3;
  }
  auto ok = [&](cudaError_t e) {
    st.launches++;
    return e == cudaSuccess;
  };
  if (st_planes && !ok(launch_prep_state(prec, op->kind, op->nx, op->ny, op->state, stp, grid_stream, c.st)))
    return finish(PHIX_ECUDA);

  // ---- spectral interval -------------------------------------------------
  double alpha_i, beta_i;
  if (o.rho_re > 0) {
    alpha_i = -o.rho_re;
    beta_i = o.rho_hi;
    st.rho = o.rho_re;
  } else {
    // parameter block staged in this thread's static buffer (sized for
    // PHIX_NOALLOC_MMAX + 1 entries), copied into the scratch
    if (o.power_max_it > PHIX_NOALLOC_MMAX) return finish(PHIX_EINVAL);
    unsigned char* hp = g_stage.ptab;
    ptab_fill(hp, 0, 0, o.power_max_it, 0.0, o.power_rel, kJ, 1.0, nullptr, nullptr);
    if (cudaMemcpyAsync(ptab, hp, ptab_bytes(o.power_max_it + 1), cudaMemcpyHostToDevice, c.st) != cudaSuccess)
      return finish(PHIX_ECUDA);
    if (cudaMemsetAsync(c.ctl, 0, sizeof(LejaCtl), c.st) != cudaSuccess) return finish(PHIX_ECUDA);
    if (!ok(launch_power_start(prec, N, o.power_seed, y[0], c.ctl, partials, grid, c.st))) return finish(PHIX_ECUDA);
    ChainSpec cs{};
    cs.prec = prec;
    cs.op = op->kind;
    cs.mode = MODE_POWER;
    cs.nx = op->nx;
    cs.ny = op->ny;
    cs.y[0] = y[0];
    cs.y[1] = y[1];
    cs.st = stp;
    cs.ctl = c.ctl;
    cs.partials = partials;
    cs.ptab = ptab;
    cs.grid = grid;
    int launched = 0, target = std::min(o.power_max_it, 16);
    for (;;) {
      for (int m = launched + 1; m <= target; ++m)
        if (!ok(launch_iter(cs, c.st))) return finish(PHIX_ECUDA);
      launched = target;
      if (!read_ctl(c)) return finish(PHIX_ECUDA);
      if (c.h.done || launched >= o.power_max_it) break;
      target = std::min(o.power_max_it, launched + 8);
    }
    if (c.h.status == PHIX_ENAN) return finish(PHIX_ENAN);
    st.power_mv = c.h.iters;
    st.rho = c.h.rho;
    alpha_i = -o.safety * c.h.rho;
    beta_i = o.rho_hi;
  }
  // half-width covering twice the imaginary extent (complex spectra), the
  // interval anchored at its right end beta
  const double gamma = std::max(0.25 * (beta_i - alpha_i), 2.0 * std::max(0.0, o.rho_im));
  const double cc = beta_i - 2.0 * gamma;
  if (gamma == 0.0) {
    // zero spectrum (e.g. a zero operator): phi_l(0) v = v / l!, as phix_phi_action gives
    for (int k = 0; k < nout; ++k) {
      double f = 1.0;
      for (int i = 2; i <= l[k]; ++i) f *= i;
      const double c1 = 1.0 / f;
      const double* x1 = v;
      if (!ok(launch_lincomb(N, 1, &c1, &x1, out[k], grid_stream, c.st))) return finish(PHIX_ECUDA);
    }
    if (cudaStreamSynchronize(c.st) != cudaSuccess) return finish(PHIX_ECUDA);
    return finish(PHIX_OK);
  }
  // one vertical pass only: a substepped action needs more vectors than the scratch holds
  for (int k = 0; k < nout; ++k) {
    double s_re = o.gamma_cap > 0 ? scale[k] * h * gamma / o.gamma_cap : 0.0;
    double s_im = (o.iota_cap > 0 && o.rho_im > 0) ? scale[k] * h * o.rho_im / o.iota_cap : 0.0;
    if (s_re > 1.0 + 1e-12 || s_im > 1.0 + 1e-12) return finish(PHIX_EINVAL);
  }

  // ---- divided differences (host, in this thread's static buffer) ---------
  const int M = o.m_max + 1;
  const double* xi = leja_table(M);
  double (*d)[PHIX_NOALLOC_MMAX + 1] = g_stage.d;
  for (int k = 0; k < nout; ++k) {
    const double a0 = scale[k] * h * cc, b0 = scale[k] * h * gamma;
    for (int i = 0; i < M; ++i) d[k][i] = phi_host(l[k], a0 + b0 * xi[i]);
    divided_differences_host(xi, d[k], M);
  }

  // ---- Newton-Leja pass ----------------------------------------------------
  {
    unsigned char* hp = g_stage.ptab;
    double* beta = g_stage.beta;
    beta[0] = 0.0;
    for (int m = 1; m < M; ++m) beta[m] = -(cc / gamma + xi[m - 1]);
    const double* dk[KMAX] = {};
    for (int k = 0; k < nout; ++k) dk[k] = d[k];
    const double al = 1.0 / gamma;
    double k8[8];
    for (int j = 0; j < 8; ++j) k8[j] = j < nscaled ? al * kJ[j] : kJ[j];
    ptab_fill(hp, nout, o.m_min, o.m_max, tol, 0.0, k8, al, beta, dk);
    if (cudaMemcpyAsync(ptab, hp, ptab_bytes(M), cudaMemcpyHostToDevice, c.st) != cudaSuccess)
      return finish(PHIX_ECUDA);
  }
  if (cudaMemsetAsync(c.ctl, 0, sizeof(LejaCtl), c.st) != cudaSuccess) return finish(PHIX_ECUDA);
  if (!ok(launch_scale(v, N, c.ctl, partials, grid, c.st))) return finish(PHIX_ECUDA);
  InitLaunch IL{};
  IL.prec = prec;
  IL.ncomp = ncomp;
  IL.nx = op->nx;
  IL.ny = op->ny;
  IL.v = v;
  IL.y0 = y[0];
  for (int k = 0; k < nout; ++k) IL.p[k] = p[k];
  IL.ctl = c.ctl;
  IL.partials = partials;
  IL.ptab = ptab;
  IL.grid = grid;
  if (!ok(launch_init(IL, c.st))) return finish(PHIX_ECUDA);
  ChainSpec cs{};
  cs.prec = prec;
  cs.op = op->kind;
  cs.mode = MODE_NEWTON;
  cs.nx = op->nx;
  cs.ny = op->ny;
  cs.y[0] = y[0];
  cs.y[1] = y[1];
  for (int k = 0; k < nout; ++k) cs.p[k] = p[k];
  cs.st = stp;
  cs.ctl = c.ctl;
  cs.partials = partials;
  cs.ptab = ptab;
  cs.grid = grid;
  int launched = 0, target = std::min(o.m_max, 32);
  for (;;) {
    for (int m = launched + 1; m <= target; ++m)
      if (!ok(launch_iter(cs, c.st))) return finish(PHIX_ECUDA);
    launched = target;
    if (!read_ctl(c)) return finish(PHIX_ECUDA);
    if (c.h.done || launched >= o.m_max) break;
    target = std::min(o.m_max, launched + 8);
  }
  if (!ok(launch_finalize(prec, N, nout, p, out, c.ctl, grid_stream, c.st))) return finish(PHIX_ECUDA);
  if (cudaStreamSynchronize(c.st) != cudaSuccess) return finish(PHIX_ECUDA);
  st.iters = c.h.iters;
  st.jv = c.h.iters;
  st.passes = 1;
  st.substeps = 1;
  return finish(c.h.done ? (phix_status)c.h.status : PHIX_ENOTCONV);
}
