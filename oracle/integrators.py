"""EXPRB43 (Eq. exprb43, Sec. 5.4) and EPIRK4s3 (Eq. epirk4s3, Sec. 5.1) steps.

Both linearise f at u^n (Sec. 1): J = J(u^n), R(k) = F(k) - F(u^n).
Leja evaluates each phi_l separately; the stages that share f(u^n) run in
the vertical form (Sec. 4).  KIOPS evaluates the shared stages as several
output times of one Krylov run and the rest individually.
"""
import numpy as np

from . import leja as _leja
from . import kiops as _kiops
from .operators import with_state, remainder


def _phi_actions(opu, v, h, outputs, method, tol, spec, stats, leja_kw, kiops_kw):
    if method == "leja":
        alpha, beta = spec
        res, info = _leja.leja_phi(opu.jv, v, h, alpha, beta, outputs, tol, **leja_kw)
        stats["iters"] += info["iters"]
        stats["jv"] += info["jv"]
        stats["actions"] += len(outputs)
        if info["status"] != 0:
            stats["status"] = info["status"]
        return res
    res, infos = _kiops.kiops_phi(lambda x: h * opu.jv(x), v, outputs, tol, **kiops_kw)
    for info in infos:
        stats["jv"] += info["matvecs"]
        if info["status"] != 0:
            stats["status"] = info["status"]
    stats["actions"] += len(outputs)
    return res


def spectrum(opu, safety=1.2, seed=0x5EED, max_it=50, rel=1e-2):
    """Leja interval [alpha, beta] = [-safety * rho, 0] from power iteration (Sec. 2.2)."""
    n = opu.n * opu.ny * opu.ncomp
    rho, mv = _leja.power_iteration(opu.jv, n, seed=seed, max_it=max_it, rel=rel)
    return (-safety * rho, 0.0), mv


def exprb43_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """One EXPRB43 step.  Returns (u4, u3, stats); u4 - u3 is the error estimate."""
    leja_kw = leja_kw or {}
    kiops_kw = kiops_kw or {}
    opu = with_state(op, u)
    stats = dict(iters=0, jv=0, actions=0, power_mv=0, status=0)
    if method == "leja" and spec is None:
        spec, stats["power_mv"] = spectrum(opu)
    stats["spec"] = spec
    fu = op.f(u)
    P1, P2 = _phi_actions(opu, fu * h, h, [(1, 0.5), (1, 1.0)], method, tol, spec, stats, leja_kw, kiops_kw)
    a = u + 0.5 * P1
    Ra = remainder(opu, u, a, fu)
    (Q,) = _phi_actions(opu, Ra * h, h, [(1, 1.0)], method, tol, spec, stats, leja_kw, kiops_kw)
    b = u + P2 + Q
    Rb = remainder(opu, u, b, fu)
    (T3,) = _phi_actions(opu, (16.0 * Ra - 2.0 * Rb) * h, h, [(3, 1.0)], method, tol, spec, stats, leja_kw, kiops_kw)
    u3 = u + P2 + T3
    (T4,) = _phi_actions(opu, (-48.0 * Ra + 12.0 * Rb) * h, h, [(4, 1.0)], method, tol, spec, stats, leja_kw, kiops_kw)
    u4 = u3 + T4
    return u4, u3, stats


def epirk4s3_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """One EPIRK4s3 step.  Returns (u4, u3, stats)."""
    leja_kw = leja_kw or {}
    kiops_kw = kiops_kw or {}
    opu = with_state(op, u)
    stats = dict(iters=0, jv=0, actions=0, power_mv=0, status=0)
    if method == "leja" and spec is None:
        spec, stats["power_mv"] = spectrum(opu)
    stats["spec"] = spec
    fu = op.f(u)
    P8, P9, P1 = _phi_actions(opu, fu * h, h, [(1, 1.0 / 8.0), (1, 1.0 / 9.0), (1, 1.0)],
                              method, tol, spec, stats, leja_kw, kiops_kw)
    a = u + P8 / 8.0
    b = u + P9 / 9.0
    Ra = remainder(opu, u, a, fu)
    Rb = remainder(opu, u, b, fu)
    (T3,) = _phi_actions(opu, (1892.0 * Ra + 1458.0 * (Rb - 2.0 * Ra)) * h, h, [(3, 1.0)],
                         method, tol, spec, stats, leja_kw, kiops_kw)
    u3 = u + P1 + T3
    (T4,) = _phi_actions(opu, (-42336.0 * Ra - 34992.0 * (Rb - 2.0 * Ra)) * h, h, [(4, 1.0)],
                         method, tol, spec, stats, leja_kw, kiops_kw)
    u4 = u3 + T4
    return u4, u3, stats
