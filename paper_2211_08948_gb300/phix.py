"""Thin ctypes binding of libphix (include/phix.h), same function names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Vector arguments are torch CUDA tensors of dtype float64 (their
device memory is passed by pointer) or raw device addresses (int).  The
library must exist (``python -m paper_2211_08948_gb300.build``); loading
fails loudly otherwise.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphix.so")

PHIX_OK, PHIX_EINVAL, PHIX_ENOTCONV, PHIX_ENAN, PHIX_ETIMEOUT, PHIX_ECUDA, PHIX_ENOMEM, PHIX_ETOOBIG = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOTCONV", 3: "ENAN", 4: "ETIMEOUT", 5: "ECUDA", 6: "ENOMEM",
                7: "ETOOBIG"}
PHIX_NOALLOC_SCRATCH_BYTES = 32 << 20
PHIX_NOALLOC_MMAX = 1000
PHIX_NOALLOC_OVERHEAD_BYTES = 194560
PHIX_MLP_NPARAM = 5443
PHIX_MLP_NFEAT = 16
PHIX_LEJA, PHIX_KIOPS, PHIX_LEKRY = 0, 1, 2
PHIX_EXPRB43, PHIX_EPIRK4S3, PHIX_EPIRK4S3A, PHIX_EXPRB53S3, PHIX_EPIRK5P1 = range(5)
PHIX_KERNEL_AUTO, PHIX_KERNEL_SINGLE, PHIX_KERNEL_TMA, PHIX_KERNEL_FUSED2 = 0, 1, 2, 3
PHIX_CHAIN_AUTO, PHIX_CHAIN_PERSISTENT, PHIX_CHAIN_GRAPH = 0, 1, 2
PHIX_CONTROL_TRADITIONAL, PHIX_CONTROL_COST = 0, 1
PHIX_FP64, PHIX_DF64, PHIX_FP32_JV, PHIX_FP32 = 0, 1, 2, 3
PHIX_OP_ADVDIFF, PHIX_OP_GRAYSCOTT, PHIX_OP_BURGERS = 0, 1, 2
PHIX_OP_ADR, PHIX_OP_ALLEN_CAHN, PHIX_OP_BRUSSELATOR = 3, 4, 5
PHIX_JV_ANALYTIC, PHIX_JV_FD = 0, 1

# every symbol include/phix.h declares
EXPORTS = [
    "phix_opts_default", "phix_version", "phix_create", "phix_destroy", "phix_last_error",
    "phix_phi_action", "phix_phi_combination", "phix_spectrum", "phix_exprb43_step",
    "phix_epirk4s3_step", "phix_rhs", "phix_small_expm", "phix_phi_action_batched", "phix_features",
    "phix_mlp_forward", "phix_mlp_grad", "phix_mlp_train", "phix_phi_action_learned", "phix_leja_points", "phix_divided_differences", "phix_phi_action_noalloc",
    "phix_step", "phix_step_host", "phix_block_newton", "phix_block_faces", "phix_block_start",
    "phix_leja_stop", "phix_opts_size", "phix_stats_size", "phix_integrate", "phix_batched_config",
    "phix_learned_targets",
]


class phix_jop(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("param", ctypes.c_double * 8), ("state", ctypes.c_void_p)]


class phix_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("safety", ctypes.c_double), ("rho_re", ctypes.c_double),
                ("rho_hi", ctypes.c_double), ("rho_im", ctypes.c_double),
                ("gamma_cap", ctypes.c_double), ("iota_cap", ctypes.c_double),
                ("m_max", ctypes.c_int), ("m_min", ctypes.c_int), ("power_max_it", ctypes.c_int),
                ("power_rel", ctypes.c_double), ("power_seed", ctypes.c_uint64),
                ("kiops_m_init", ctypes.c_int), ("kiops_m_max", ctypes.c_int),
                ("kiops_m_step", ctypes.c_int), ("kiops_max_substeps", ctypes.c_int),
                ("profile", ctypes.c_int), ("kernel", ctypes.c_int), ("kiops_fused", ctypes.c_int),
                ("jv", ctypes.c_int), ("leja_augmented", ctypes.c_int), ("chain", ctypes.c_int)]


class phix_batch_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("D", ctypes.c_double), ("ax", ctypes.c_double),
                ("ay", ctypes.c_double), ("h", ctypes.c_double), ("rho_re", ctypes.c_double),
                ("rho_hi", ctypes.c_double), ("rho_im", ctypes.c_double), ("v", ctypes.c_void_p),
                ("out", ctypes.c_void_p * 3)]


class phix_block(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("gnx", ctypes.c_int), ("gny", ctypes.c_int), ("x0", ctypes.c_int),
                ("y0", ctypes.c_int), ("bx", ctypes.c_int), ("by", ctypes.c_int),
                ("param", ctypes.c_double * 8), ("state", ctypes.c_void_p)]


class phix_adapt(ctypes.Structure):
    _fields_ = [("t_end", ctypes.c_double), ("dt0", ctypes.c_double), ("tol", ctypes.c_double),
                ("iter_tol", ctypes.c_double), ("dt_max", ctypes.c_double), ("controller", ctypes.c_int),
                ("max_steps", ctypes.c_int)]


class phix_adapt_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("accepted", ctypes.c_int), ("rejected", ctypes.c_int),
                ("t", ctypes.c_double), ("dt_next", ctypes.c_double), ("matvecs", ctypes.c_longlong)]


class phix_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("jv", ctypes.c_int),
                ("substeps", ctypes.c_int), ("power_mv", ctypes.c_int), ("rejections", ctypes.c_int),
                ("passes", ctypes.c_int), ("launches", ctypes.c_int), ("rho", ctypes.c_double),
                ("err_est", ctypes.c_double), ("iter_launches", ctypes.c_int), ("iter_ms", ctypes.c_double),
                ("iter_bytes", ctypes.c_double), ("tma_passes", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PhixError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("phix %s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load(path=None):
    """Load libphix.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libphix.so not built at %s: run python -m paper_2211_08948_gb300.build" % p)
    lib = ctypes.CDLL(p)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    lib.phix_opts_default.argtypes = [ctypes.POINTER(phix_opts)]
    lib.phix_opts_default.restype = None
    lib.phix_version.restype = I
    lib.phix_opts_size.restype = ctypes.c_size_t
    lib.phix_stats_size.restype = ctypes.c_size_t
    lib.phix_create.argtypes = [ctypes.POINTER(P), P]
    lib.phix_destroy.argtypes = [P]
    lib.phix_last_error.argtypes = [P]
    lib.phix_last_error.restype = ctypes.c_char_p
    lib.phix_phi_action.argtypes = [P, ctypes.POINTER(phix_jop), D, P, I, ctypes.POINTER(I),
                                    ctypes.POINTER(D), ctypes.POINTER(P), D, I,
                                    ctypes.POINTER(phix_opts), ctypes.POINTER(phix_stats)]
    lib.phix_phi_combination.argtypes = [P, ctypes.POINTER(phix_jop), D, ctypes.POINTER(P), I, P, D, I,
                                         ctypes.POINTER(phix_opts), ctypes.POINTER(phix_stats)]
    lib.phix_rhs.argtypes = [P, ctypes.POINTER(phix_jop), P, P]
    F = ctypes.c_float
    lib.phix_features.argtypes = [P, ctypes.POINTER(phix_jop), D, P]
    lib.phix_learned_targets.argtypes = [P, ctypes.POINTER(phix_jop), D, D, ctypes.POINTER(phix_opts),
                                         ctypes.POINTER(F)]
    lib.phix_mlp_forward.argtypes = [P, P, P, I, P]
    lib.phix_mlp_grad.argtypes = [P, P, P, P, I, P, ctypes.POINTER(F)]
    lib.phix_mlp_train.argtypes = [P, P, P, P, ctypes.POINTER(I), P, P, I, I, I, F, ctypes.POINTER(F)]
    lib.phix_phi_action_learned.argtypes = [P, ctypes.POINTER(phix_jop), D, P, I, ctypes.POINTER(I),
                                            ctypes.POINTER(D), ctypes.POINTER(P), D, P,
                                            ctypes.POINTER(phix_opts), ctypes.POINTER(phix_stats)]
    lib.phix_phi_action_batched.argtypes = [P, ctypes.POINTER(phix_batch_problem), I, I, ctypes.POINTER(I), D,
                                            ctypes.POINTER(phix_opts), ctypes.POINTER(I), ctypes.POINTER(phix_stats)]
    lib.phix_small_expm.argtypes = [P, I, P, P, P, D, P, ctypes.POINTER(I)]
    lib.phix_spectrum.argtypes = [P, ctypes.POINTER(phix_jop), ctypes.POINTER(phix_opts),
                                  ctypes.POINTER(D), ctypes.POINTER(phix_stats)]
    lib.phix_block_newton.argtypes = [P, ctypes.POINTER(phix_block), P, P, I, ctypes.POINTER(P),
                                      ctypes.POINTER(D), D, D, P]
    lib.phix_block_faces.argtypes = [P, ctypes.POINTER(phix_block), I, P, P]
    lib.phix_block_start.argtypes = [P, ctypes.POINTER(phix_block), ctypes.c_uint64, P]
    lib.phix_leja_stop.argtypes = [I, I, I, ctypes.POINTER(D), D, D, ctypes.POINTER(D)]
    lib.phix_leja_stop.restype = I
    lib.phix_integrate.argtypes = [P, I, ctypes.POINTER(phix_jop), P, ctypes.POINTER(phix_adapt), I,
                                   ctypes.POINTER(phix_opts), ctypes.POINTER(D), ctypes.POINTER(phix_adapt_stats)]
    for f in (lib.phix_step, lib.phix_step_host):
        f.argtypes = [P, I, ctypes.POINTER(phix_jop), P, D, D, I, ctypes.POINTER(phix_opts),
                      ctypes.POINTER(D), ctypes.POINTER(phix_stats)]
    for f in (lib.phix_exprb43_step, lib.phix_epirk4s3_step):
        f.argtypes = [P, ctypes.POINTER(phix_jop), P, D, D, I, ctypes.POINTER(phix_opts),
                      ctypes.POINTER(D), ctypes.POINTER(phix_stats)]
    lib.phix_phi_action_noalloc.argtypes = [ctypes.POINTER(phix_jop), D, P, I, ctypes.POINTER(I),
                                            ctypes.POINTER(D), ctypes.POINTER(P), D,
                                            ctypes.POINTER(phix_opts), P, ctypes.POINTER(phix_stats)]
    lib.phix_leja_points.argtypes = [ctypes.POINTER(D), I]
    lib.phix_divided_differences.argtypes = [I, D, D, I, ctypes.POINTER(D)]
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("phix_opts_default", "phix_version", "phix_last_error"):
            fn.restype = I
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not (x.is_cuda and x.dtype.is_floating_point and x.element_size() == 8 and x.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def _hptr(x):
    """Address of a contiguous float64 CPU tensor (or a raw host address)."""
    if isinstance(x, int):
        return x
    if x.is_cuda or x.dtype != _torch_f64(x) or not x.is_contiguous():
        raise ValueError("expected a contiguous float64 CPU tensor")
    return x.data_ptr()


def _torch_f64(x):
    import torch
    return torch.float64


def _fptr(x):
    if x is None:
        return None
    if not (x.is_cuda and x.dtype.is_floating_point and x.element_size() == 4 and x.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return x.data_ptr()


def _check(ctx, st):
    if st != PHIX_OK:
        msg = load().phix_last_error(ctx).decode() if ctx else ""
        raise PhixError(st, msg)


def phix_opts_default(**overrides):
    o = phix_opts()
    load().phix_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def phix_version():
    return load().phix_version()


def phix_create(stream=None):
    """Context on the current device bound to `stream` (torch.cuda.Stream, raw handle or None)."""
    handle = None
    if stream is not None:
        handle = stream if isinstance(stream, int) else stream.cuda_stream
    ctx = ctypes.c_void_p()
    _check(None, load().phix_create(ctypes.byref(ctx), handle))
    return ctx


def phix_destroy(ctx):
    load().phix_destroy(ctx)


def phix_last_error(ctx):
    return load().phix_last_error(ctx).decode()


def make_jop(kind, nx, ny, params, state=None):
    """phix_jop for `kind` on an nx x ny grid; `state` (tensor) is kept alive
    by the returned object so its device memory stays valid."""
    op = phix_jop()
    op.kind, op.nx, op.ny = kind, nx, ny
    for i, p in enumerate(params):
        op.param[i] = p
    op.state = _ptr(state)
    op._keepalive = state
    return op


def phix_phi_action(ctx, op, h, v, l, scale, out, tol, method=PHIX_LEJA, opts=None, check=True):
    """out[k] = phi_{l[k]}(scale[k] h J) v; returns phix_stats."""
    n = len(l)
    st = phix_stats()
    L = (ctypes.c_int * n)(*l)
    S = (ctypes.c_double * n)(*scale)
    O = (ctypes.c_void_p * n)(*[_ptr(o) for o in out])
    rc = load().phix_phi_action(ctx, ctypes.byref(op), h, _ptr(v), n, L, S, O, tol, method,
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st


def phix_phi_action_noalloc(op, h, v, l, scale, out, tol, opts=None, stream=None, check=True):
    """Context-free Leja action whose scratch is the library's fixed device
    array (no device allocation); returns phix_stats.  Calls must not overlap
    on the GPU: they share that array."""
    n = len(l)
    st = phix_stats()
    L = (ctypes.c_int * n)(*l)
    S = (ctypes.c_double * n)(*scale)
    O = (ctypes.c_void_p * n)(*[_ptr(o) for o in out])
    handle = None
    if stream is not None:
        handle = stream if isinstance(stream, int) else stream.cuda_stream
    rc = load().phix_phi_action_noalloc(ctypes.byref(op), h, _ptr(v), n, L, S, O, tol,
                                        ctypes.byref(opts) if opts is not None else None, handle,
                                        ctypes.byref(st))
    if check and rc != PHIX_OK:
        raise PhixError(rc, "phix_phi_action_noalloc failed")
    return st


def phix_phi_combination(ctx, op, h, b, out, tol, method=PHIX_LEJA, opts=None, check=True):
    """out = sum_j phi_j(h J) b[j] (b[j] None = 0); returns phix_stats."""
    p = len(b) - 1
    st = phix_stats()
    B = (ctypes.c_void_p * (p + 1))(*[_ptr(x) for x in b])
    rc = load().phix_phi_combination(ctx, ctypes.byref(op), h, B, p, _ptr(out), tol, method,
                                     ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st


def phix_phi_action_batched(ctx, problems, l, tol, opts=None, check=True):
    """problems: list of dicts nx, ny, D, ax, ay, h, rho_re, rho_hi, rho_im, v (tensor), out (list of
    tensors, one per l).  Returns (phix_stats, per-problem status list)."""
    n = len(problems)
    arr = (phix_batch_problem * n)()
    for i, q in enumerate(problems):
        a = arr[i]
        a.nx, a.ny = q["nx"], q["ny"]
        a.D, a.ax, a.ay, a.h = q["D"], q["ax"], q["ay"], q["h"]
        a.rho_re, a.rho_hi, a.rho_im = q["rho_re"], q.get("rho_hi", 0.0), q.get("rho_im", 0.0)
        a.v = _ptr(q["v"])
        for k, o in enumerate(q["out"]):
            a.out[k] = _ptr(o)
    L = (ctypes.c_int * len(l))(*l)
    per = (ctypes.c_int * n)()
    st = phix_stats()
    rc = load().phix_phi_action_batched(ctx, arr, n, len(l), L, tol,
                                        ctypes.byref(opts) if opts is not None else None, per, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st, list(per)


def phix_features(ctx, op, h, feats):
    """feats (float32[16]) <- features of op at op.state with step h."""
    _check(ctx, load().phix_features(ctx, ctypes.byref(op), h, _fptr(feats)))


def phix_learned_targets(ctx, op, h, rho, opts=None):
    """The network's three training targets for op at op.state (a list)."""
    t = (ctypes.c_float * 3)()
    _check(ctx, load().phix_learned_targets(ctx, ctypes.byref(op), h, rho,
                                            ctypes.byref(opts) if opts is not None else None, t))
    return list(t)


def phix_mlp_forward(ctx, params, X, Y):
    _check(ctx, load().phix_mlp_forward(ctx, _fptr(params), _fptr(X), X.shape[0], _fptr(Y)))


def phix_mlp_grad(ctx, params, X, T, G):
    loss = ctypes.c_float()
    _check(ctx, load().phix_mlp_grad(ctx, _fptr(params), _fptr(X), _fptr(T), X.shape[0], _fptr(G),
                                     ctypes.byref(loss)))
    return loss.value


def phix_mlp_train(ctx, params, m, v, step, X, T, batch, nsteps, lr):
    """Returns (new step counter, last batch loss)."""
    s = ctypes.c_int(step)
    loss = ctypes.c_float()
    _check(ctx, load().phix_mlp_train(ctx, _fptr(params), _fptr(m), _fptr(v), ctypes.byref(s), _fptr(X), _fptr(T),
                                      X.shape[0], batch, nsteps, lr, ctypes.byref(loss)))
    return s.value, loss.value


def phix_phi_action_learned(ctx, op, h, v, l, scale, out, tol, params, opts=None, check=True):
    n = len(l)
    st = phix_stats()
    L = (ctypes.c_int * n)(*l)
    S = (ctypes.c_double * n)(*scale)
    O = (ctypes.c_void_p * n)(*[_ptr(o) for o in out])
    rc = load().phix_phi_action_learned(ctx, ctypes.byref(op), h, _ptr(v), n, L, S, O, tol, _fptr(params),
                                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st


def phix_small_expm(ctx, d, u, l, tau, F):
    """F <- exp(tau T) e_1 for the tridiagonal T = tridiag(l, d, u); returns 0 (Chebyshev) or 1 (Taylor)."""
    m = ctypes.c_int()
    _check(ctx, load().phix_small_expm(ctx, d.numel(), _ptr(d), _ptr(u), _ptr(l), tau, _ptr(F), ctypes.byref(m)))
    return m.value


def phix_rhs(ctx, op, u, f):
    """f <- f(u) (float64)."""
    _check(ctx, load().phix_rhs(ctx, ctypes.byref(op), _ptr(u), _ptr(f)))


def phix_spectrum(ctx, op, opts=None):
    rho = ctypes.c_double()
    st = phix_stats()
    _check(ctx, load().phix_spectrum(ctx, ctypes.byref(op), ctypes.byref(opts) if opts is not None else None,
                                     ctypes.byref(rho), ctypes.byref(st)))
    return rho.value, st


def _step(fn, ctx, op, u, h, tol, method, opts, check, ptr=_ptr):
    err = ctypes.c_double()
    st = phix_stats()
    rc = fn(ctx, ctypes.byref(op), ptr(u), h, tol, method,
            ctypes.byref(opts) if opts is not None else None, ctypes.byref(err), ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st


def phix_exprb43_step(ctx, op, u, h, tol, method=PHIX_LEJA, opts=None, check=True):
    """u <- EXPRB43 step (in place); returns phix_stats (err_est = ||u4 - u3||)."""
    return _step(load().phix_exprb43_step, ctx, op, u, h, tol, method, opts, check)


def phix_epirk4s3_step(ctx, op, u, h, tol, method=PHIX_LEJA, opts=None, check=True):
    return _step(load().phix_epirk4s3_step, ctx, op, u, h, tol, method, opts, check)


def phix_step(ctx, scheme, op, u, h, tol, method=PHIX_LEJA, opts=None, check=True):
    """u <- one step of `scheme` (PHIX_EXPRB43 .. PHIX_EPIRK5P1), in place on the
    device vector u; returns phix_stats (err_est = ||u_high - u_low||)."""
    fn = load().phix_step
    return _step(lambda c, o, x, *a: fn(c, scheme, o, x, *a), ctx, op, u, h, tol, method, opts, check)


def phix_step_host(ctx, scheme, op, u_host, h, tol, method=PHIX_LEJA, opts=None, check=True):
    """As phix_step with the state in host memory: u_host is a CPU float64
    tensor (page-locked for full copy bandwidth) or a raw host address."""
    fn = load().phix_step_host
    return _step(lambda c, o, x, *a: fn(c, scheme, o, x, *a), ctx, op, u_host, h, tol, method, opts, check,
                 ptr=_hptr)


def phix_integrate(ctx, scheme, op, u, t_end, dt0, tol, method=PHIX_LEJA, controller=PHIX_CONTROL_COST,
                   iter_tol=0.0, dt_max=0.0, max_steps=10000, opts=None, check=True):
    """Advance the device state u from 0 to t_end with step-size control (Sec. 2.3).
    Returns (phix_adapt_stats, list of accepted step sizes)."""
    ad = phix_adapt(t_end=t_end, dt0=dt0, tol=tol, iter_tol=iter_tol, dt_max=dt_max, controller=controller,
                    max_steps=max_steps)
    dts = (ctypes.c_double * max_steps)()
    st = phix_adapt_stats()
    rc = load().phix_integrate(ctx, scheme, ctypes.byref(op), _ptr(u), ctypes.byref(ad), method,
                               ctypes.byref(opts) if opts is not None else None, dts, ctypes.byref(st))
    if check:
        _check(ctx, rc)
    return st, list(dts[:st.accepted])


def phix_batched_config(ctx):
    """(threads per CTA, dynamic shared memory bytes, CTAs per SM) of the last batched call."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().phix_batched_config(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def make_block(kind, gnx, gny, x0, y0, bx, by, params, state=None):
    """phix_block for one block of the gnx x gny grid; `state` (padded device
    tensor) is kept alive by the returned object."""
    b = phix_block()
    b.kind, b.gnx, b.gny, b.x0, b.y0, b.bx, b.by = kind, gnx, gny, x0, y0, bx, by
    for i, p in enumerate(params):
        b.param[i] = p
    b.state = _ptr(state)
    b._keepalive = state
    return b


def phix_block_newton(ctx, blk, y_in, y_out, p, dk, a, b, norms):
    """One block iteration (y_out None: initialise p_k = dk[k] y_in)."""
    K = len(p)
    P = (ctypes.c_void_p * max(1, K))(*[_ptr(t) for t in p])
    Dk = (ctypes.c_double * max(1, K))(*dk)
    _check(ctx, load().phix_block_newton(ctx, ctypes.byref(blk), _ptr(y_in), _ptr(y_out), K, P, Dk, a, b,
                                         _ptr(norms)))


def phix_block_faces(ctx, blk, direction, y_pad, faces):
    _check(ctx, load().phix_block_faces(ctx, ctypes.byref(blk), direction, _ptr(y_pad), _ptr(faces)))


def phix_block_start(ctx, blk, seed, y_pad):
    _check(ctx, load().phix_block_start(ctx, ctypes.byref(blk), seed, _ptr(y_pad)))


def phix_leja_stop(K, m, m_min, dkm, tol, ysq, psq):
    D = ctypes.c_double * max(1, K)
    return load().phix_leja_stop(K, m, m_min, D(*dkm), tol, ysq, D(*psq))


def phix_leja_points(m):
    a = (ctypes.c_double * m)()
    _check(None, load().phix_leja_points(a, m))
    return list(a)


def phix_divided_differences(l, a, b, m):
    d = (ctypes.c_double * m)()
    _check(None, load().phix_divided_differences(l, a, b, m, d))
    return list(d)
