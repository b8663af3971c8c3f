"""Exponential integrators of Sec. 5, each as the paper prints it:

  EPIRK4s3   Eq. epirk4s3  (Sec. 5.1)     EXPRB43    Eq. exprb43   (Sec. 5.4)
  EPIRK4s3A  Eq. epirk4s3a (Sec. 5.2)     EXPRB53s3  Eq. exprb5s3  (Sec. 5.5)
  EPIRK5P1   Eq. epirk5p1 and the coefficient table of Sec. 5.3

All linearise f at u^n (Sec. 1): J = J(u^n), R(k) = F(k) - F(u^n) with
F(x) = f(x) - J x.  Each step returns (u_high, u_low, stats); u_high is the
new state and ||u_high - u_low|| the embedded error estimate.

How the phi-functions of a step are grouped follows the paper's text for
each scheme and method:
* "leja": the terms that act on the same vector f(u^n) h are computed in
  one Newton basis ("vertical", Sec. 4); every phi-function applied to a
  combination of remainders is computed on its own.
* "kiops": internal stages in vertical form (several output times of one
  Krylov run), and for EPIRK4s3, EPIRK4s3A and EXPRB53s3 the solutions
  u_3 (and u_5) as ONE linear combination sum_j phi_j(hJ) b_j ("horizontal",
  Theorem of Sec. 2.1); EXPRB43 computes its remaining terms individually,
  EPIRK5P1 everything vertically.
* "lekry" (Sec. 5.1): the internal stages by Leja (vertical), the solution
  combinations by KIOPS (horizontal); the error-estimate term of EPIRK4s3 /
  EPIRK4s3A, which the paper allows to be computed either way, by Leja.
  LeKry exists for EPIRK4s3, EPIRK4s3A and EXPRB53s3 only (the other two
  schemes have no linear combination to evaluate, Sec. 5.3 and 5.4).
"""
import numpy as np

from . import leja as _leja
from . import kiops as _kiops
from .operators import with_state, remainder

# EPIRK5P1 coefficients, the table of Sec. 5.3 (g32h, g33h are the hatted values)
EPIRK5P1 = dict(
    a11=0.35129592695058193092, a21=0.84405472011657126298, a22=1.6905891609568963624,
    b1=1.0, b2=1.2727127317356892397, b3=2.2714599265422622275,
    g11=0.35129592695058193092, g21=0.84405472011657126298, g22=0.5,
    g31=1.0, g32=0.71111095364366870359, g32h=0.5, g33=0.62378111953371494809, g33h=1.0)

ORDER = {"exprb43": (4, 3), "epirk4s3": (4, 3), "epirk4s3a": (4, 3), "exprb53s3": (5, 3), "epirk5p1": (5, 4)}


class _Ctx:
    """Shared state of one step: the linearised operator, h, tolerances and
    the statistics the step accumulates."""

    def __init__(self, op, u, h, method, tol, spec, leja_kw, kiops_kw):
        if method not in ("leja", "kiops", "lekry"):
            raise ValueError("method must be leja, kiops or lekry")
        self.opu = with_state(op, u)
        self.h = h
        self.tol = tol
        self.leja_kw = leja_kw or {}
        self.kiops_kw = kiops_kw or {}
        self.stats = dict(iters=0, jv=0, actions=0, power_mv=0, status=0)
        if method in ("leja", "lekry") and spec is None:
            spec, self.stats["power_mv"] = spectrum(self.opu)
        self.spec = spec
        self.stats["spec"] = spec

    def vertical(self, v, outputs, how):
        """phi_{l_k}(s_k h J) v for outputs [(l_k, s_k)]: one Leja basis or one
        KIOPS run per distinct l with the output times s_k."""
        st = self.stats
        if how == "leja":
            alpha, beta = self.spec
            res, info = _leja.leja_phi(self.opu.jv, v, self.h, alpha, beta, outputs, self.tol, **self.leja_kw)
            st["iters"] += info["iters"]
            st["jv"] += info["jv"]
            if info["status"] != 0:
                st["status"] = info["status"]
        else:
            res, infos = _kiops.kiops_phi(lambda x: self.h * self.opu.jv(x), v, outputs, self.tol, **self.kiops_kw)
            for info in infos:
                st["jv"] += info["matvecs"]
                if info["status"] != 0:
                    st["status"] = info["status"]
        st["actions"] += len(outputs)
        return res

    def horizontal(self, bs):
        """sum_j phi_j(hJ) bs[j] (bs[j] None = 0) by one KIOPS run (Theorem of Sec. 2.1)."""
        (w,), info = _kiops.kiops(lambda x: self.h * self.opu.jv(x), bs, [1.0], self.tol, **self.kiops_kw)
        self.stats["jv"] += info["matvecs"]
        self.stats["actions"] += 1
        if info["status"] != 0:
            self.stats["status"] = info["status"]
        return w


def spectrum(opu, safety=1.2, seed=0x5EED, max_it=50, rel=1e-2):
    """Leja interval [alpha, beta] = [-safety * rho, 0] from power iteration (Sec. 2.2)."""
    n = opu.n * opu.ny * opu.ncomp
    rho, mv = _leja.power_iteration(opu.jv, n, seed=seed, max_it=max_it, rel=rel)
    return (-safety * rho, 0.0), mv


def _inner(method):
    """Method of the internal stages: Leja for leja and lekry, KIOPS for kiops."""
    return "kiops" if method == "kiops" else "leja"


def exprb43_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """EXPRB43, Eq. exprb43.  Returns (u4, u3, stats)."""
    if method == "lekry":
        raise ValueError("EXPRB43 has no LeKry form (Sec. 5.4)")
    c = _Ctx(op, u, h, method, tol, spec, leja_kw, kiops_kw)
    fu = op.f(u)
    P1, P2 = c.vertical(fu * h, [(1, 0.5), (1, 1.0)], method)
    a = u + 0.5 * P1
    Ra = remainder(c.opu, u, a, fu)
    (Q,) = c.vertical(Ra * h, [(1, 1.0)], method)
    b = u + P2 + Q
    Rb = remainder(c.opu, u, b, fu)
    (T3,) = c.vertical((16.0 * Ra - 2.0 * Rb) * h, [(3, 1.0)], method)
    u3 = u + P2 + T3
    (T4,) = c.vertical((-48.0 * Ra + 12.0 * Rb) * h, [(4, 1.0)], method)
    u4 = u3 + T4
    return u4, u3, c.stats


def _epirk4_family(op, u, h, method, tol, spec, leja_kw, kiops_kw, ca, cb, w3, w4):
    """EPIRK4s3 and EPIRK4s3A share one structure (Sec. 5.2): internal stages
    a = u + ca phi_1(ca hJ) f h, b = u + cb phi_1(cb hJ) f h; then
    u3 = u + phi_1(hJ) f h + phi_3(hJ) w3(Ra, Rb) h, u4 = u3 + phi_4(hJ) w4(Ra, Rb) h."""
    c = _Ctx(op, u, h, method, tol, spec, leja_kw, kiops_kw)
    fu = op.f(u)
    if method == "leja":
        Pa, Pb, P1 = c.vertical(fu * h, [(1, ca), (1, cb), (1, 1.0)], "leja")
    else:
        Pa, Pb = c.vertical(fu * h, [(1, ca), (1, cb)], _inner(method))
    a = u + ca * Pa
    b = u + cb * Pb
    Ra = remainder(c.opu, u, a, fu)
    Rb = remainder(c.opu, u, b, fu)
    W3 = w3(Ra, Rb) * h
    W4 = w4(Ra, Rb) * h
    if method == "leja":
        (T3,) = c.vertical(W3, [(3, 1.0)], "leja")
        u3 = u + P1 + T3
    else:
        u3 = u + c.horizontal([None, fu * h, None, W3])
    (T4,) = c.vertical(W4, [(4, 1.0)], "kiops" if method == "kiops" else "leja")
    u4 = u3 + T4
    return u4, u3, c.stats


def epirk4s3_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """EPIRK4s3, Eq. epirk4s3.  Returns (u4, u3, stats)."""
    return _epirk4_family(op, u, h, method, tol, spec, leja_kw, kiops_kw, 1.0 / 8.0, 1.0 / 9.0,
                          lambda Ra, Rb: 1892.0 * Ra + 1458.0 * (Rb - 2.0 * Ra),
                          lambda Ra, Rb: -42336.0 * Ra - 34992.0 * (Rb - 2.0 * Ra))


def epirk4s3a_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """EPIRK4s3A, Eq. epirk4s3a.  Returns (u4, u3, stats)."""
    return _epirk4_family(op, u, h, method, tol, spec, leja_kw, kiops_kw, 0.5, 2.0 / 3.0,
                          lambda Ra, Rb: 32.0 * Ra - 13.5 * Rb,
                          lambda Ra, Rb: -144.0 * Ra + 81.0 * Rb)


def exprb53s3_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """EXPRB53s3, Eq. exprb5s3.  Returns (u5, u3, stats)."""
    c = _Ctx(op, u, h, method, tol, spec, leja_kw, kiops_kw)
    fu = op.f(u)
    inner = _inner(method)
    if method == "leja":
        Ph, Pn, P1 = c.vertical(fu * h, [(1, 0.5), (1, 0.9), (1, 1.0)], "leja")
    else:
        Ph, Pn = c.vertical(fu * h, [(1, 0.5), (1, 0.9)], inner)
    a = u + 0.5 * Ph
    Ra = remainder(c.opu, u, a, fu)
    Q3h, Q3n = c.vertical(Ra * h, [(3, 0.5), (3, 0.9)], inner)
    b = u + 0.9 * Pn + (27.0 / 25.0) * Q3h + (729.0 / 125.0) * Q3n
    Rb = remainder(c.opu, u, b, fu)
    W3 = (2.0 * Ra + (150.0 / 81.0) * Rb) * h
    W5a = (18.0 * Ra - (250.0 / 81.0) * Rb) * h
    W5b = (-60.0 * Ra + (500.0 / 27.0) * Rb) * h
    if method == "leja":
        (T3,) = c.vertical(W3, [(3, 1.0)], "leja")
        (T5a,) = c.vertical(W5a, [(3, 1.0)], "leja")
        (T5b,) = c.vertical(W5b, [(4, 1.0)], "leja")
        u3 = u + P1 + T3
        u5 = u + P1 + T5a + T5b
    else:
        u3 = u + c.horizontal([None, fu * h, None, W3])
        u5 = u + c.horizontal([None, fu * h, None, W5a, W5b])
    return u5, u3, c.stats


def epirk5p1_step(op, u, h, method="leja", tol=1e-8, spec=None, leja_kw=None, kiops_kw=None):
    """EPIRK5P1, Eq. epirk5p1 with the coefficient table of Sec. 5.3; every
    phi-function in vertical form, three passes.  Returns (u5, u4, stats)."""
    if method == "lekry":
        raise ValueError("EPIRK5P1 has no LeKry form (Sec. 5.3)")
    g = EPIRK5P1
    c = _Ctx(op, u, h, method, tol, spec, leja_kw, kiops_kw)
    fu = op.f(u)
    P11, P21, P31 = c.vertical(fu * h, [(1, g["g11"]), (1, g["g21"]), (1, g["g31"])], method)
    a = u + g["a11"] * P11
    Ra = remainder(c.opu, u, a, fu)
    Q22, Q32h, Q32 = c.vertical(Ra * h, [(1, g["g22"]), (1, g["g32h"]), (1, g["g32"])], method)
    b = u + g["a21"] * P21 + g["a22"] * Q22
    Rb = remainder(c.opu, u, b, fu)
    T33, T33h = c.vertical((-2.0 * Ra + Rb) * h, [(3, g["g33"]), (3, g["g33h"])], method)
    u4 = u + g["b1"] * P31 + g["b2"] * Q32h + g["b3"] * T33h
    u5 = u + g["b1"] * P31 + g["b2"] * Q32 + g["b3"] * T33
    return u5, u4, c.stats


STEPS = {"exprb43": exprb43_step, "epirk4s3": epirk4s3_step, "epirk4s3a": epirk4s3a_step,
         "exprb53s3": exprb53s3_step, "epirk5p1": epirk5p1_step}
