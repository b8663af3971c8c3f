"""Automatic step-size control, Sec. 2.3: the traditional controller and the
cost controller, driving the embedded error estimates of the integrators of
Sec. 5 (oracle.integrators).

TEST INFRASTRUCTURE: part of the CPU oracle (see oracle/__init__.py).

What the paper fixes (Sec. 2.3):
* traditional: dt_{n+1} = dt_n (tol / e_n)^(1/(p+1));
* cost: dt_{n+1} = dt_n * lambda if 1 <= s < lambda, delta if delta <= s < 1,
  s = exp(-alpha tanh(beta D)) otherwise, D = (ln c_n - ln c_{n-1}) /
  (ln dt_n - ln dt_{n-1}); alpha = 0.65241444, beta = 0.26862269,
  lambda = 1.37412002, delta = 0.64446017;
* the step actually taken is min(dt_traditional, dt_cost).

Readings where the paper is silent (the CUDA library follows the same):
* e_n = ||u_high - u_low||_2 / sqrt(N), the root-mean-square difference of
  the two embedded solutions, compared with tol; a step with e_n > tol is
  rejected and retried with 0.9 times the traditional step computed from it
  (the paper gives no rule for rejected steps; without the factor the retry
  aims exactly at tol and is rejected again whenever rounding puts e_n a
  hair above it, repeatedly).  A step whose phi-actions fail to converge is
  retried with half the step.
* p + 1 is the power of dt in e_n: p is the order of the lower-order
  (embedded) solution, the error estimator's order (3 for EXPRB43, EPIRK4s3,
  EPIRK4s3A and EXPRB53s3, 4 for EPIRK5P1).
* c_n is the cost per unit of simulated time: the Jacobian-vector products
  of step n (iteration matvecs and power-iteration matvecs, rejected attempts
  of that step included) divided by dt_n.  (Per-step cost grows with dt for
  any iterative scheme, so D would be positive for every step size; per unit
  time is the quantity whose minimum the controller seeks.)
* The cost controller needs two accepted steps; before that (and when
  dt_n == dt_{n-1}, where D is undefined, read as D = 0) it uses what it has:
  the traditional step alone for the first two steps, D = 0 otherwise.
* e_n == 0 (a linear problem) gives an unbounded traditional step: the step
  is then limited by dt_max (if set) and by the cost controller.
* The last step is shortened to land on t_end.
"""
import math

import numpy as np

from . import integrators

ALPHA, BETA, LAM, DELTA = 0.65241444, 0.26862269, 1.37412002, 0.64446017
RETRY = 0.9  # factor on the traditional step after a rejection


def traditional(dt, err, tol, order):
    """dt (tol / e)^(1/(order+1)); +inf when err == 0."""
    if err == 0.0:
        return math.inf
    return dt * (tol / err) ** (1.0 / (order + 1))


def cost_factor(c_n, c_prev, dt_n, dt_prev):
    """The cost controller's factor dt_{n+1} / dt_n (Sec. 2.3)."""
    den = math.log(dt_n) - math.log(dt_prev)
    D = 0.0 if abs(den) < 1e-14 else (math.log(c_n) - math.log(c_prev)) / den
    s = math.exp(-ALPHA * math.tanh(BETA * D))
    if 1.0 <= s < LAM:
        return LAM
    if DELTA <= s < 1.0:
        return DELTA
    return s


def integrate(op, u0, t_end, dt0, tol, scheme="exprb43", method="leja", controller="cost", iter_tol=None,
              dt_max=0.0, max_steps=10000, leja_kw=None, kiops_kw=None):
    """Integrate u' = f(u) from 0 to t_end with step-size control.
    Returns (u, info) with info: accepted, rejected, t, dts (accepted step
    sizes), errs (their error estimates), costs (matvecs per accepted step,
    rejected attempts included), status (0, or 2 when max_steps ran out)."""
    step = integrators.STEPS[scheme]
    order = integrators.ORDER[scheme][1]
    itol = tol if iter_tol is None else iter_tol
    u = np.array(u0, dtype=np.float64, copy=True)
    N = u.size
    t, dt = 0.0, dt0
    info = dict(accepted=0, rejected=0, dts=[], errs=[], costs=[], status=0)
    hist = []                       # (c_n, dt_n) of accepted steps
    spent = 0
    while t < t_end * (1 - 1e-14):
        if info["accepted"] + info["rejected"] >= max_steps:
            info["status"] = 2
            break
        dt = min(dt, t_end - t)
        if dt_max > 0:
            dt = min(dt, dt_max)
        uh, ul, st = step(op, u, dt, method=method, tol=itol, leja_kw=leja_kw, kiops_kw=kiops_kw)
        spent += st["jv"] + st["power_mv"]
        err = float(np.linalg.norm(uh - ul)) / math.sqrt(N)
        dt_trad = traditional(dt, err, tol, order)
        if err > tol or st["status"] != 0:
            info["rejected"] += 1
            dt = RETRY * dt_trad if st["status"] == 0 else 0.5 * dt
            continue
        u = uh
        t += dt
        info["accepted"] += 1
        info["dts"].append(dt)
        info["errs"].append(err)
        info["costs"].append(spent)
        hist.append((spent / dt, dt))
        spent = 0
        nxt = dt_trad
        if controller == "cost" and len(hist) >= 2:
            (c_n, d_n), (c_p, d_p) = hist[-1], hist[-2]
            nxt = min(nxt, dt * cost_factor(c_n, c_p, d_n, d_p))
        elif math.isinf(nxt):
            nxt = dt
        dt = nxt
    info["t"] = t
    return u, info
