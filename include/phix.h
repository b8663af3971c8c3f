/*
 * phix: actions of the phi-functions of exponential integrators, phi_l(hJ)v,
 * on GB300 (sm_103a), by real-Leja interpolation and by a KIOPS-style Krylov
 * method, plus the EXPRB43 and EPIRK4s3 time steps built on them.
 *
 * The method is that of Deka & Einkemmer, "A comparison of Leja- and
 * Krylov-based iterative schemes for Exponential Integrators"
 * (arXiv:2211.08948):
 *   phi-functions ........ Sec. 1   (phi_0 = e^z, phi_{l+1} = (phi_l - 1/l!)/z)
 *   Krylov / augmented ... Sec. 2.1 (Theorem: exp of [[A, B], [0, K]])
 *   Leja interpolation ... Sec. 2.2 (Newton form at Leja points, stop test)
 *   vertical form ........ Sec. 4
 *   EPIRK4s3 ............. Sec. 5.1, Eq. (epirk4s3)   LeKry ... Sec. 5.1
 *   EPIRK4s3A ............ Sec. 5.2, Eq. (epirk4s3a)
 *   EPIRK5P1 ............. Sec. 5.3, Eq. (epirk5p1)
 *   EXPRB43 .............. Sec. 5.4, Eq. (exprb43)
 *   EXPRB53s3 ............ Sec. 5.5, Eq. (exprb5s3)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.  Every vector argument is a DEVICE pointer to float64 data owned
 *   by the caller, contiguous, 8-byte aligned (16-byte alignment enables the
 *   vectorised kernels).  Vectors are planar: species-major, then row y,
 *   then column x; length N = ncomp * nx * ny.  The library never frees or
 *   keeps caller memory.  Scalars and small arrays (l[], scale[], b[]) are
 *   HOST memory.  The context owns a device workspace that grows on demand.
 * Streams.  All work is enqueued on the stream given to phix_create.  Entry
 *   points that need a decision from the device (iteration counts,
 *   convergence) synchronise that stream; on return all outputs are valid.
 * Grid.  Periodic unit square, dx = 1/nx, dy = 1/ny, second-order centred
 *   differences (Sec. 3).
 * Errors.  Every function returns a phix_status; no exception crosses the
 *   ABI, the GPU never traps.  phix_last_error() gives a message.  On
 *   PHIX_ENOTCONV outputs hold the last iterate.  Inputs are never written,
 *   except u_inout of the step functions (on success only).
 * Threads.  A context is not thread-safe; use one per host thread/stream.
 */
#ifndef PHIX_H
#define PHIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Rises whenever the layout of a public struct changes: callers must be built
 * against the header of the library they load (101: phix_opts.kiops_fused;
 * 102: phix_opts.chain; 103: phix_opts.jv, phix_opts.leja_augmented). */
#define PHIX_VERSION 103

typedef struct phix_ctx phix_ctx;

typedef enum {
  PHIX_OK = 0,
  PHIX_EINVAL = 1,    /* bad argument (sizes, pointers, enum values)        */
  PHIX_ENOTCONV = 2,  /* Leja: m_max reached; KIOPS: substep limit reached  */
  PHIX_ENAN = 3,      /* a norm became NaN/Inf                              */
  PHIX_ETIMEOUT = 4,  /* a bounded device wait expired                      */
  PHIX_ECUDA = 5,     /* a CUDA runtime call failed                         */
  PHIX_ENOMEM = 6,    /* workspace allocation failed                        */
  PHIX_ETOOBIG = 7    /* phix_phi_action_noalloc: the problem does not fit its
                         fixed scratch (PHIX_NOALLOC_SCRATCH_BYTES)           */
} phix_status;

/* How the phi-functions are evaluated.  PHIX_LEKRY (Sec. 5.1) is a policy of
 * the step functions: internal stages by Leja, the solution combinations by
 * KIOPS; the phi-action entry points take PHIX_LEJA or PHIX_KIOPS only.     */
typedef enum { PHIX_LEJA = 0, PHIX_KIOPS = 1, PHIX_LEKRY = 2 } phix_method;

/* Exponential integrators of Sec. 5 (each embedded with a lower-order
 * solution whose difference is the error estimate).                       */
typedef enum {
  PHIX_EXPRB43 = 0,   /* Eq. (exprb43),  Sec. 5.4: order 4, estimate order 3        */
  PHIX_EPIRK4S3 = 1,  /* Eq. (epirk4s3), Sec. 5.1: order 4, estimate order 3        */
  PHIX_EPIRK4S3A = 2, /* Eq. (epirk4s3a), Sec. 5.2: order 4, estimate order 3       */
  PHIX_EXPRB53S3 = 3, /* Eq. (exprb5s3), Sec. 5.5: order 5, estimate order 3        */
  PHIX_EPIRK5P1 = 4   /* Eq. (epirk5p1) and its table, Sec. 5.3: order 5, est. 4    */
} phix_scheme;

/* Arithmetic of the iteration (Newton-Leja step / Arnoldi).  Inputs and
 * outputs are always float64; divided differences, Leja points, the small
 * Krylov exponential and all scalar control are float64 in every mode.    */
typedef enum {
  PHIX_FP64 = 0,    /* native float64 everywhere                            */
  PHIX_DF64 = 1,    /* double-float: pairs of float32 (hi, lo), ~2^-47
                       relative per operation, float64-class results          */
  PHIX_FP32_JV = 2, /* stencil J*y in float32 on hi parts, the Newton update
                       and accumulation in double-float                      */
  PHIX_FP32 = 3     /* float32 iteration                                    */
} phix_prec;

typedef enum {
  PHIX_OP_ADVDIFF = 0,   /* f(u) = D lap u + ax u_x + ay u_y (linear), 1 species        */
  PHIX_OP_GRAYSCOTT = 1, /* Sec. 3: f_u = Du lap u - u v^2 + F(1-u),
                                    f_v = Dv lap v + u v^2 - (F+k) v, 2 species     */
  PHIX_OP_BURGERS = 2,   /* f(u) = nu lap u - u (u_x + u_y), 1 species                  */
  /* The paper's no-flow problems (Sec. 3): cell-centred grids with homogeneous
   * Neumann boundaries (ghost cell = boundary cell), dx = L/nx, dy = L/ny.
   * Leja and KIOPS iterate in float64 for these whatever opts->prec.         */
  PHIX_OP_ADR = 3,        /* f(u) = a lap u + b (u_x + u_y) + g u (1-u)(u-1/2) on [0,1]^2;
                             param: a, b, g                                              */
  PHIX_OP_ALLEN_CAHN = 4, /* f(u) = a lap u + u - u^3 on [-1,1]^2 (L = 2); param: a       */
  PHIX_OP_BRUSSELATOR = 5 /* f_u = a lap u + 1 + u^2 v - 4u, f_v = a lap v + 3u - u^2 v
                             on [0,1]^2, 2 species; param: a                             */
} phix_op_kind;

/* A Jacobian operator J = J(state) of one of the right-hand sides above.  */
typedef struct {
  int kind;            /* phix_op_kind                                               */
  int nx, ny;          /* grid, nx, ny >= 3                                          */
  double param[8];     /* ADVDIFF: D, ax, ay | GRAYSCOTT: Du, Dv, F, k | BURGERS: nu */
  const double* state; /* device, linearisation point u^n (GRAYSCOTT, BURGERS); may
                          be NULL for ADVDIFF.  Ignored by the step functions, which
                          linearise at u_inout.                                      */
} phix_jop;

/* Tunables; fill with phix_opts_default() and override fields.            */
typedef struct {
  phix_prec prec;      /* iteration arithmetic (default PHIX_DF64)                     */
  double safety;       /* spectral interval [-safety*rho, 0] from power iteration (1.2) */
  double rho_re;       /* > 0: |Re lambda|max of J supplied by the caller: the interval
                          is [-rho_re, rho_hi] and no power iteration runs (default -1) */
  double rho_hi;       /* upper end of the real interval, with rho_re or with the power
                          iteration's [-safety*rho, rho_hi] (default 0; > 0 for spectra
                          reaching into the right half-plane, e.g. Allen-Cahn)         */
  double rho_im;       /* >= 0: bound on |Im lambda(J)|, used for substep counts (0)   */
  double gamma_cap;    /* Leja: max s*h*gamma per substep (default 200)                */
  double iota_cap;     /* Leja: max s*h*rho_im per substep, 0 = off (default 4)        */
  int m_max;           /* Leja: max Newton iterations per pass (default 500)           */
  int m_min;           /* Leja: first iteration where the stop test applies (3)       */
  int power_max_it;    /* power iteration: max matvecs (50), at most 4000             */
  double power_rel;    /* power iteration: stop at this relative change (1e-2)        */
  uint64_t power_seed; /* SplitMix64 stream of the power-iteration start vector        */
  int kiops_m_init;    /* KIOPS: initial Krylov dimension (16)                         */
  int kiops_m_max;     /* KIOPS: max Krylov dimension (64)                             */
  int kiops_m_step;    /* KIOPS: basis growth on rejection (8)                         */
  int kiops_max_substeps; /* KIOPS: substep limit -> PHIX_ENOTCONV (10000)             */
  int profile;         /* 1: time the iteration loops with CUDA events on the
                          context's stream and report them in phix_stats; 2: as 1, and
                          launch every iteration kernel on its own instead of in a
                          conditional CUDA graph, for per-kernel profilers (slower:
                          the host polls the chain) (default 0)                         */
  int kernel;          /* Leja Newton-step kernel: PHIX_KERNEL_AUTO (default) takes the
                          TMA-staged kernel when one iteration's operands exceed the L2
                          cache and the single-step kernel otherwise; PHIX_KERNEL_SINGLE,
                          PHIX_KERNEL_TMA and PHIX_KERNEL_FUSED2 force one (TMA needs
                          rows of a multiple of 16 bytes, i.e. nx even, nx % 4 == 0 for
                          4-byte state; FUSED2 nx % 64 == 0 and ny % 16 == 0; each falls
                          back to the single-step kernel otherwise).  The two-iteration
                          kernel computes iterations m and m + 1 in one launch from y_{m-1}
                          staged with a two-point ring, storing y_{m+1} and p_m: half the
                          memory traffic per iteration, the same results bit for bit as
                          one iteration per launch for the same stop iteration (on
                          GB300 no faster: the double-float arithmetic binds).          */
  int kiops_fused;     /* KIOPS: 1 (default) runs each Arnoldi step as one pass (the
                          orthogonalisation of step j staged in shared memory and pass 1
                          of step j + 1 read from it) when nx % 64 == 0 and ny % 8 == 0;
                          0, or other grids: two passes per step                      */
  int jv;              /* Leja: PHIX_JV_ANALYTIC (default) or PHIX_JV_FD, the "numerical"
                          Jacobian of Sec. 4: J w ~ (f(u + eps w) - f(u)) / eps with
                          eps = sqrt(2^-52) (1 + ||u||) / ||w||, in float64 (a comparison
                          variant: one right-hand-side stencil per Newton iteration)     */
  int leja_augmented;  /* phix_phi_combination with PHIX_LEJA: 0 (default) sums the
                          individual phi_j actions; 1 interpolates exp of the augmented
                          matrix of the Theorem of Sec. 2.1 (Appendix A), float64        */
  int chain;           /* Leja Newton pass with the single-step kernel:
                          PHIX_CHAIN_PERSISTENT runs the whole pass in ONE cooperative
                          launch (every block resident, one grid-wide barrier per
                          iteration, the stop test taken by every block on the same
                          totals; a barrier wait that exceeds 2 s ends the pass with
                          PHIX_ETIMEOUT); PHIX_CHAIN_AUTO (default) and
                          PHIX_CHAIN_GRAPH run one launch per iteration inside a
                          CUDA graph: the chain length predicted from the divided
                          differences as plain launches, then a conditional WHILE
                          node of 8 launches per evaluation (measured faster on
                          GB300; a launch after the stop returns at once).
                          The TMA-staged kernel always runs one launch per iteration. */
} phix_opts;

typedef enum { PHIX_CHAIN_AUTO = 0, PHIX_CHAIN_PERSISTENT = 1, PHIX_CHAIN_GRAPH = 2 } phix_chain;
typedef enum { PHIX_JV_ANALYTIC = 0, PHIX_JV_FD = 1 } phix_jv;

typedef enum { PHIX_KERNEL_AUTO = 0, PHIX_KERNEL_SINGLE = 1, PHIX_KERNEL_TMA = 2, PHIX_KERNEL_FUSED2 = 3 } phix_kernel;

/* Per-call statistics (host struct, filled on return).                    */
typedef struct {
  int status;        /* phix_status of the call                                       */
  int iters;         /* Leja Newton iterations / KIOPS Arnoldi steps (all passes)      */
  int jv;            /* Jacobian-vector products in the iteration                      */
  int substeps;      /* Leja ODE-identity substeps / KIOPS accepted substeps           */
  int power_mv;      /* power-iteration matvecs                                        */
  int rejections;    /* KIOPS rejected substep attempts                                */
  int passes;        /* Leja Newton passes / KIOPS runs                                */
  int launches;      /* device kernels launched by the call                            */
  double rho;        /* |lambda|max estimate used for the Leja interval                */
  double err_est;    /* step functions: ||u4 - u3||_2                                  */
  /* opts.profile = 1 only: the Newton-Leja iterations / KIOPS Arnoldi steps that
     did work, the device time of the loops that ran them (CUDA events around each
     Newton loop, which includes the few no-op launches that end it, and around
     each run of Arnoldi steps) and their algorithmic HBM bytes (each vector read
     or written once per iteration or step).                                           */
  int iter_launches;
  double iter_ms;
  double iter_bytes;
  int tma_passes;    /* Leja Newton passes that ran the TMA-staged kernel              */
} phix_stats;

void phix_opts_default(phix_opts* opts);
int phix_version(void);
/* sizeof(phix_opts) and sizeof(phix_stats) as the library was built: a caller's
 * mirror of the structs (e.g. a foreign-function binding) checks its layout. */
size_t phix_opts_size(void);
size_t phix_stats_size(void);

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*,
 * NULL = legacy default stream) on the current device.  Returns PHIX_EINVAL
 * if ctx is NULL, PHIX_ECUDA if no device is usable.                       */
phix_status phix_create(phix_ctx** ctx, void* cuda_stream);
/* Free the context's workspace (after synchronising its stream).          */
phix_status phix_destroy(phix_ctx* ctx);
/* Message of the last failed call on ctx (empty string if none).          */
const char* phix_last_error(const phix_ctx* ctx);

/* Vertical/individual actions, Sec. 2.2 and Sec. 4:
 *   out[k] = phi_{l[k]}(scale[k] * h * J) v,   k = 0 .. nout-1,
 * without any h^l factor.  l[k] in 0..8, scale[k] > 0, 1 <= nout <= 4.
 * PHIX_LEJA: one Newton basis shared by all outputs when no substeps are
 * needed (vertical form), else each output by ODE-identity substeps.
 * PHIX_KIOPS: one Krylov run per distinct l with output times scale[k].
 * tol: relative 2-norm stop tolerance (Leja: |d_m| ||y_m|| <= tol ||p_m||;
 * KIOPS: error per unit step relative to the augmented vector norm).
 * v and out[k] are device vectors of length N; out[k] may not alias v.    */
phix_status phix_phi_action(phix_ctx* ctx, const phix_jop* op, double h, const double* v,
                            int nout, const int* l, const double* scale, double* const* out,
                            double tol, phix_method method, const phix_opts* opts,
                            phix_stats* stats);

/* Horizontal combination, Theorem of Sec. 2.1:
 *   out = sum_{j=0}^{p} phi_j(h J) b[j]     (b[j] == NULL means zero),
 * 0 <= p <= 8.  KIOPS: one augmented Krylov run.  LEJA: one individual
 * phi_j action per non-NULL b[j] (the paper's Leja evaluates phi_l
 * individually, App. A), summed.                                          */
phix_status phix_phi_combination(phix_ctx* ctx, const phix_jop* op, double h,
                                 const double* const* b, int p, double* out, double tol,
                                 phix_method method, const phix_opts* opts, phix_stats* stats);

/* Right-hand side f(u) of the operator's PDE (Sec. 1 "f(u)", Sec. 3
 * discretisation), float64: f and u are device vectors of length N
 * (f may not alias u).  op->state is ignored.                             */
phix_status phix_rhs(phix_ctx* ctx, const phix_jop* op, const double* u, double* f);

/* Spectrum estimate of J (Sec. 2.2 "power iterations"): *rho = ||J v_k||
 * for the power iterate v_k from a SplitMix64 start vector.               */
phix_status phix_spectrum(phix_ctx* ctx, const phix_jop* op, const phix_opts* opts,
                          double* rho, phix_stats* stats);

/* One EXPRB43 step, Eq. (exprb43): u_inout <- u4 (4th order).  J and f at
 * u_inout; *err_est = ||u4 - u3||_2 (the embedded 3rd-order estimate).
 * Leja: phi_1(h/2 J) f h and phi_1(h J) f h vertically, the other three
 * actions individually.  KIOPS: the first two as output times 1/2, 1 of
 * one run, the rest individually.                                         */
phix_status phix_exprb43_step(phix_ctx* ctx, const phix_jop* op, double* u_inout, double h,
                              double tol, phix_method method, const phix_opts* opts,
                              double* err_est, phix_stats* stats);

/* One EPIRK4s3 step, Eq. (epirk4s3) (= phix_step with PHIX_EPIRK4S3).
 * Leja: phi_1 at scales 1/8, 1/9, 1 on f h vertically, then phi_3 and phi_4
 * on the remainder combinations.  KIOPS: output times 1/8, 1/9 of one run,
 * u_3 as one horizontal combination, phi_4 individually.                   */
phix_status phix_epirk4s3_step(phix_ctx* ctx, const phix_jop* op, double* u_inout, double h,
                               double tol, phix_method method, const phix_opts* opts,
                               double* err_est, phix_stats* stats);

/* One step of any scheme of Sec. 5: u_inout <- the higher-order solution;
 * J and f at u_inout; *err_est = ||u_high - u_low||_2.  Grouping of the
 * phi-functions (Sec. 5):
 *   PHIX_LEJA   the terms on f(u) h in one vertical Newton pass (EXPRB43:
 *               scales 1/2, 1; EPIRK4s3: 1/8, 1/9, 1; EPIRK4s3A: 1/2, 2/3, 1;
 *               EXPRB53s3: 1/2, 9/10, 1, then phi_3 at 1/2, 9/10 on R(a) h;
 *               EPIRK5P1: three passes of three / three / two outputs), every
 *               phi-function of a remainder combination individually;
 *   PHIX_KIOPS  internal stages as output times of one Krylov run; the
 *               solutions of EPIRK4s3, EPIRK4s3A and EXPRB53s3 as one
 *               horizontal combination sum_j phi_j(hJ) b_j each; EXPRB43 and
 *               EPIRK5P1 as for Leja;
 *   PHIX_LEKRY  EPIRK4s3, EPIRK4s3A, EXPRB53s3 only (else PHIX_EINVAL):
 *               internal stages by Leja, solution combinations by KIOPS, the
 *               phi_4 error term of the EPIRK4 family by Leja; opts->prec must
 *               be PHIX_FP64 or PHIX_DF64.
 * u_inout is a DEVICE vector of length N.                                  */
phix_status phix_step(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u_inout, double h,
                      double tol, phix_method method, const phix_opts* opts, double* err_est,
                      phix_stats* stats);

/* As phix_step with the state in HOST memory (N doubles; page-locked memory
 * gives full copy bandwidth, pageable memory works): the call copies it to
 * the device, takes the step and, on success, copies the new state back
 * before it returns.  On failure u_host_inout is unchanged.                 */
phix_status phix_step_host(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u_host_inout,
                           double h, double tol, phix_method method, const phix_opts* opts,
                           double* err_est, phix_stats* stats);

/* ---- Automatic step-size control (Sec. 2.3) -------------------------------
 * phix_integrate advances u' = f(u) from t = 0 to t_end with phix_step and a
 * step-size controller:
 *   traditional: dt_{n+1} = dt_n (tol / e_n)^(1/(p+1));
 *   cost:        dt_{n+1} = min(dt_traditional, dt_n * F) with the cost
 *                controller's factor F of Sec. 2.3 (alpha 0.65241444, beta
 *                0.26862269, lambda 1.37412002, delta 0.64446017) applied to the
 *                cost per unit time c_n = (Jacobian products of step n) / dt_n;
 * e_n = ||u_high - u_low||_2 / sqrt(N); a step with e_n > tol (or whose
 * phi-actions fail to converge) is rejected and retried (with 0.9 times the
 * traditional step, or half the step after a failure); p is the order of
 * the scheme's embedded estimate (3; EPIRK5P1: 4); the last step lands on
 * t_end.  The cost controller starts from the third step (it needs two
 * accepted steps).                                                          */
typedef enum { PHIX_CONTROL_TRADITIONAL = 0, PHIX_CONTROL_COST = 1 } phix_controller;
typedef struct {
  double t_end;     /* > 0                                                         */
  double dt0;       /* first trial step, > 0                                       */
  double tol;       /* accept e_n <= tol                                           */
  double iter_tol;  /* tolerance of the phi-actions (<= 0: tol)                   */
  double dt_max;    /* > 0: largest step (bounds the step on linear problems, where
                       e_n = 0); <= 0: none                                        */
  int controller;   /* phix_controller                                             */
  int max_steps;    /* accepted + rejected attempts; then PHIX_ENOTCONV            */
} phix_adapt;
typedef struct {
  int status, accepted, rejected;
  double t;             /* time reached (t_end on success)                         */
  double dt_next;       /* the step the controller proposes after the last one      */
  long long matvecs;    /* Jacobian-vector products of every attempt               */
} phix_adapt_stats;
/* u_inout: DEVICE state (length N), advanced in place.  dts (HOST, may be
 * NULL): the accepted step sizes, at most max_steps entries.               */
phix_status phix_integrate(phix_ctx* ctx, phix_scheme scheme, const phix_jop* op, double* u_inout,
                           const phix_adapt* ad, phix_method method, const phix_opts* opts, double* dts,
                           phix_adapt_stats* stats);

/* One problem of a batch: a periodic advection-diffusion operator
 * J = D lap + ax d/dx + ay d/dy on an nx x ny grid, a step h, its spectral
 * interval and the vectors.                                               */
typedef struct {
  int nx, ny;          /* grid, >= 3                                                 */
  double D, ax, ay;    /* operator coefficients                                      */
  double h;            /* step: outputs are phi_{l[k]}(h J) v                        */
  double rho_re;       /* > 0: Leja interval [-rho_re, rho_hi] of the real spectrum  */
  double rho_hi;
  double rho_im;       /* >= 0: bound on |Im lambda(J)| (substep count, iota_cap)    */
  const double* v;     /* device, nx*ny                                              */
  double* out[3];      /* device, nx*ny each, out[k] for l[k], k < nout             */
} phix_batch_problem;

/* Batched actions (many small independent problems; Sec. 2.2 per problem): for
 * every problem i < nprob, out[k] = phi_{l[k]}(h_i J_i) v_i, k < nout <= 3,
 * l[k] in 0..2, all in ONE persistent kernel launch replayed from a CUDA
 * graph: each CTA takes whole problems from a largest-first queue and runs
 * the vertical Leja pass (or the ODE-identity substeps) with block-level
 * reductions.  opts->prec: PHIX_FP64, PHIX_DF64 or PHIX_FP32_JV; opts->m_max
 * <= 500.  opts->profile = 1 additionally autotunes the launch on the first
 * call per batch shape (the problem sizes, count and precision): threads per
 * CTA (256, 512, 1024) x dynamic shared memory per CTA (0, 48 KiB, 100 KiB:
 * a vertical pass whose basis pair and accumulators fit runs on shared
 * memory) x CTAs per SM (the resident maximum and half of it), each timed on
 * a subsample (every 8th problem in largest-first order) and cached in the
 * context; it also reports the launch time in iter_ms.  Without profile the
 * tuned configuration of the shape is used if there is one, else 512
 * threads, no shared-memory passes, 2 CTAs per SM (phix_batched_config).
 * per_prob (HOST, may be NULL) receives each problem's status; stats->iters
 * sums the Newton iterations of all problems.  Problems are read from HOST
 * memory (the array), vectors are device memory.                           */
phix_status phix_phi_action_batched(phix_ctx* ctx, const phix_batch_problem* probs, int nprob, int nout,
                                    const int* l, double tol, const phix_opts* opts, int* per_prob,
                                    phix_stats* stats);

/* The launch configuration of the context's last batched call.           */
phix_status phix_batched_config(const phix_ctx* ctx, int* threads_per_cta, int* smem_bytes, int* ctas_per_sm);

/* Learned spectral interval (a trained predictor of the interval; replaces the power
 * iterations of Sec. 2.2 by a prediction, with power iteration as fallback).
 * MLP 16 -> 64 -> 64 -> 3, GELU, bfloat16 weights / float32 accumulation;
 * params: PHIX_MLP_NPARAM float32 values W1[64x16] b1[64] W2[64x64] b2[64]
 * W3[3x64] b3[3] (DEVICE).  Outputs y: rho = rho_diff e^{y0},
 * rho_im = rho_diff (e^{y1} - 1), substeps e^{y2}, rho_diff = 4 Dmax (nx^2+ny^2).
 * Features (16 float32, DEVICE): see phix_features.  All arrays DEVICE.    */
#define PHIX_MLP_NPARAM 5443
#define PHIX_MLP_NFEAT 16
/* feats[16] of the operator op at op->state with step h: kind, log sizes,
 * log D, log h, max/mean |state|, max/mean centred differences, reaction
 * extrema (Gray-Scott) or divergence and advection bounds (Burgers).      */
phix_status phix_features(phix_ctx* ctx, const phix_jop* op, double h, float* feats);
/* Training targets of the network for op at op->state (DEVICE) with step h
 * and a power-iteration estimate rho (t: HOST float[3]): t0 = log(rho /
 * rho_diff); t1 = log(1 + rho_im / rho_diff), rho_im the Bendixson bound of
 * the skew part of J (Burgers: max|U| (nx + ny), Gray-Scott: 0); t2 =
 * log(substeps) of a phi_1 action of step h on the interval the Leja path
 * takes from rho (half-width max(safety rho / 4, 2 rho_im); opts->gamma_cap,
 * opts->iota_cap; opts may be NULL).                                      */
phix_status phix_learned_targets(phix_ctx* ctx, const phix_jop* op, double h, double rho, const phix_opts* opts,
                                 float* t);
/* Y[n x 3] = MLP(X[n x 16]).                                              */
phix_status phix_mlp_forward(phix_ctx* ctx, const float* params, const float* X, int n, float* Y);
/* G[NPARAM] = gradient of the mean loss over (X, T) (n <= 65536 samples);
 * *loss (HOST) receives the loss.  Loss per sample sum_j w_j (y_j - t_j)^2,
 * w_0 = 4 when y_0 < t_0, else 1.                                         */
phix_status phix_mlp_grad(phix_ctx* ctx, const float* params, const float* X, const float* T, int n, float* G,
                          float* loss);
/* nsteps Adam steps (lr; beta 0.9 / 0.999, eps 1e-8) on contiguous batches
 * of `batch` rows of (X, T) (n a multiple of batch; the caller shuffles).
 * m, v: Adam moments (NPARAM each, zero-initialised by the caller);
 * *step (HOST) is the Adam step counter, advanced; *loss (HOST, may be NULL)
 * the last batch's loss.                                                  */
phix_status phix_mlp_train(phix_ctx* ctx, float* params, float* m, float* v, int* step, const float* X,
                           const float* T, int n, int batch, int nsteps, float lr, float* loss);
/* As phix_phi_action (Leja), with the spectral interval [-safety*rho, 0]
 * and imaginary bound rho_im from the network instead of power iteration
 * (the same safety factor as the power-iteration interval: the network's
 * loss weighs under-estimates 4x, and on 10k held-out states of sides
 * 128..1024 its rho was within 0.95..1.07 of the power iteration's, 1 %
 * below 0.989).
 * If the Leja pass does not converge or produces a non-finite norm, falls
 * back to power iteration and recomputes (stats->rejections = 1,
 * stats->power_mv counts the fallback's matvecs).                         */
phix_status phix_phi_action_learned(phix_ctx* ctx, const phix_jop* op, double h, const double* v, int nout,
                                    const int* l, const double* scale, double* const* out, double tol,
                                    const float* params, const phix_opts* opts, phix_stats* stats);

/* The small exponential of the Krylov method (Sec. 2.1: "computing the
 * exponential of the Hessenberg matrix"): F = exp(tau T) e_1 for an n x n
 * tridiagonal T (the Hessenberg matrix of window-2 incomplete
 * orthogonalisation), 1 <= n <= 129.  d[n] diagonal, u[n-1] super- and
 * l[n-1] sub-diagonal, F[n] output: DEVICE float64 arrays.  One CTA:
 * Chebyshev expansion on the exact real range of the field of values, or a
 * shifted Taylor series with scaling when T is strongly non-normal; normwise
 * accuracy ~1e-15 ||exp(tau T)||.  *method (host, may be NULL) receives 0
 * (Chebyshev) or 1 (Taylor).  Synchronises the context's stream.          */
phix_status phix_small_expm(phix_ctx* ctx, int n, const double* d, const double* u, const double* l,
                            double tau, double* F, int* method);

/* No counterpart in the paper: a library-interface addition.
 *
 * phix_phi_action_noalloc: the same vertical Leja computation as
 * phix_phi_action with PHIX_LEJA, for callers that cannot allocate device
 * memory: a host application that gives the whole device to its own memory
 * pool and forbids outside allocations, a code under a hard device-memory
 * budget, or a latency-critical loop that cannot pay the device-wide
 * synchronisation an allocation may cause.  It takes no context and calls no
 * cudaMalloc/cudaFree or other allocating routine.  Its scratch (control
 * block, reduction partials, Newton basis, accumulators, Jacobian state
 * arrays) is one fixed array of PHIX_NOALLOC_SCRATCH_BYTES in device memory,
 * held by every GPU that loads the library until the process exits.
 *   - Limits: PHIX_NOALLOC_OVERHEAD_BYTES (control block, reduction
 *     partials, parameter block: 190 KiB) + (2 + nout) vectors of N * e bytes
 *     + the state planes (Gray-Scott 2, Burgers 1, of nx * ny * s bytes), each
 *     rounded up to 256 bytes, must fit in PHIX_NOALLOC_SCRATCH_BYTES, with
 *     e = 8 bytes (PHIX_FP64, PHIX_DF64, PHIX_FP32_JV) or 4 (PHIX_FP32) and
 *     s = 8 (PHIX_FP64, PHIX_DF64) or 4; e.g. Gray-Scott up to 512 x 512 with
 *     nout = 4 in double-float.  Larger problems return PHIX_ETOOBIG.
 *     opts->m_max and opts->power_max_it <= PHIX_NOALLOC_MMAX.  Only one
 *     vertical pass: an action that would need substeps (gamma_cap,
 *     iota_cap) returns PHIX_EINVAL.  A zero spectral interval (e.g. a zero
 *     operator) gives phi_l(0) v = v / l!, as phix_phi_action does.
 *   - Host staging (parameter block, coefficient tables, ~180 KB) is static
 *     per host thread, not on the caller's stack.
 *   - The first call on a device sets that device up (looks up the scratch's
 *     device address); make that first call before any stream capture.
 *   - Every call, on any stream, shares the one scratch array, which keeps
 *     the last call's contents (the call clears what must start at zero):
 *     calls that overlap on the GPU race and give wrong results.  Issue them
 *     one after another (the call synchronises `cuda_stream` before return).
 *   - Arguments as phix_phi_action; cuda_stream is a cudaStream_t (NULL =
 *     legacy default stream); stats may be NULL.  No message string: the
 *     return value (also stats->status) is the error.                       */
#define PHIX_NOALLOC_SCRATCH_BYTES (32u << 20)
#define PHIX_NOALLOC_MMAX 1000
#define PHIX_NOALLOC_OVERHEAD_BYTES 194560u
phix_status phix_phi_action_noalloc(const phix_jop* op, double h, const double* v, int nout,
                                    const int* l, const double* scale, double* const* out,
                                    double tol, const phix_opts* opts, void* cuda_stream,
                                    phix_stats* stats);

/* ---- Domain decomposition (multi-GPU Leja) -------------------------------
 * The Newton-Leja pass needs, per iteration, one stencil product and one
 * reduction of squared norms (Sec. 2.2; the paper's low-communication case
 * for Leja, Sec. 1 and Sec. 2.1), so it splits into rectangular blocks of the
 * global periodic grid: each block is stored with a one-cell halo ring that
 * the caller fills between iterations (a 4-face exchange), and the per-block
 * norms are summed over all blocks by the caller (an allreduce).  These calls
 * are the per-block kernels; the Python driver domain.py does the exchange,
 * the (optionally lagged) allreduce and the stop test.  All float64, all
 * asynchronous on the context's stream.
 *
 * Block layout: per species a padded (bx + 2) x (by + 2) plane, row-major,
 * interior at rows 1..by and columns 1..bx (species planes back to back);
 * accumulators p_k are unpadded bx x by planes per species.                 */
typedef struct {
  int kind;            /* phix_op_kind                                              */
  int gnx, gny;        /* the global grid (dx = 1/gnx, dy = 1/gny, periodic)        */
  int x0, y0;          /* first column / row of this block in the global grid       */
  int bx, by;          /* block interior size, >= 1, inside the global grid         */
  double param[8];     /* as phix_jop                                                */
  const double* state; /* DEVICE, padded like y with filled halos: GRAYSCOTT (u, v),
                          BURGERS (U); may be NULL for ADVDIFF                         */
} phix_block;

/* One Newton-Leja (or power) iteration on a block:
 *   y_out == NULL:  p_k = dk[k] * y_in (interior), the pass's first term;
 *   else:           y_out = a * J y_in + b * y_in on the interior of y_out
 *                   (Newton: a = 1/gamma, b = -(c/gamma + xi_m); power: a =
 *                   1/||y_in||, b = 0), p_k += dk[k] * y_out.
 * y_in must have its halo filled.  norms (DEVICE, K + 1 doubles) receives
 * ||y||^2 (y = y_in when initialising, else y_out) and ||p_k||^2 over the
 * block interior.  0 <= K <= 4; p: HOST array of K device planes; dk: HOST
 * array of K coefficients d_k[m].                                           */
phix_status phix_block_newton(phix_ctx* ctx, const phix_block* blk, const double* y_in, double* y_out, int K,
                              double* const* p, const double* dk, double a, double b, double* norms);

/* Faces of a padded block: dir = 0 packs the interior faces of y_pad into
 * faces, dir = 1 writes faces into the halo ring of y_pad.  faces (DEVICE):
 * [S | N | W | E], each face all species back to back: ncomp*bx values for S
 * and N (rows y = 1 and y = by; halos y = 0 and y = by + 1), ncomp*by for W
 * and E (columns 1 and bx; halos 0 and bx + 1).                              */
phix_status phix_block_faces(phix_ctx* ctx, const phix_block* blk, int dir, double* y_pad, double* faces);

/* Interior of y_pad <- the power iteration's SplitMix64 start vector at this
 * block's GLOBAL indices (species, row, column of the gnx x gny grid).      */
phix_status phix_block_start(phix_ctx* ctx, const phix_block* blk, uint64_t seed, double* y_pad);

/* Host utility: the stop test of Sec. 2.2 on global squared norms:
 * 1 if m >= m_min and |dkm[k]| sqrt(ysq) <= tol sqrt(psq[k]) for every
 * k < K; 0 if not; -1 if a norm is not finite.  HOST arrays.                */
int phix_leja_stop(int K, int m, int m_min, const double* dkm, double tol, double ysq, const double* psq);

/* Host utility: the first m real Leja points on [-2, 2] (xi_0 = 2,
 * xi_1 = -2, xi_2 = 0, then greedy max-product), Sec. 2.2.  xi is a HOST
 * array of length m, 1 <= m <= 4096.                                      */
phix_status phix_leja_points(double* xi, int m);

/* Host utility: Newton divided differences of xi -> phi_l(a + b*xi) on the
 * first m Leja points (the coefficients d_m of Sec. 2.2).  HOST arrays.   */
phix_status phix_divided_differences(int l, double a, double b, int m, double* d);

#ifdef __cplusplus
}
#endif

#endif /* PHIX_H */
