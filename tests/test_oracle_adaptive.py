"""The oracle's step-size controllers (Sec. 2.3) against what the paper fixes
and what the mathematics implies: the printed constants (golden fixture),
the branch structure of the cost controller, the order exponent of the
traditional controller (a step chosen by it lands its error estimate near
tol in the asymptotic regime), and an adaptive run's invariants (every
accepted estimate <= tol, exact arrival at t_end, global error shrinking
with tol)."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import adaptive, integrators, exact
from oracle.operators import GrayScott, with_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = (x.strip() for x in line.split("="))
            vals[k] = float(v)
    return vals


def test_cost_controller_constants_as_printed():
    g = read_golden("cost_controller.txt")
    assert (adaptive.ALPHA, adaptive.BETA, adaptive.LAM, adaptive.DELTA) == (g["alpha"], g["beta"], g["lambda"],
                                                                             g["delta"])


def test_cost_factor_branches():
    g = read_golden("cost_controller.txt")
    f = adaptive.cost_factor
    # equal costs per unit time: D = 0, s = 1 -> the increase lambda
    assert f(5.0, 5.0, 0.2, 0.1) == g["lambda"]
    # cost per unit time growing slowly with dt (0 < D small): s just below 1 -> delta
    assert f(5.0 * 2 ** 0.1, 5.0, 0.2, 0.1) == g["delta"]
    # falling steeply (D -> -inf): s -> exp(alpha) > lambda, returned as is
    big = f(1e-150, 1e150, 0.2, 0.1)
    assert big == pytest.approx(math.exp(g["alpha"]), rel=1e-9) and big > g["lambda"]
    # rising steeply (D -> +inf): s -> exp(-alpha) < delta, returned as is
    small = f(1e150, 1e-150, 0.2, 0.1)
    assert small == pytest.approx(math.exp(-g["alpha"]), rel=1e-9) and small < g["delta"]
    # the factor never lies strictly between delta and lambda
    for D in np.linspace(-40, 40, 401):
        c = 5.0 * 2.0 ** D
        v = f(c, 5.0, 0.2, 0.1)
        assert v <= g["delta"] or v >= g["lambda"]
    # and it does not increase with D
    vals = [f(5.0 * 2.0 ** D, 5.0, 0.2, 0.1) for D in np.linspace(-40, 40, 401)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))


def _gs(n=8):
    rng = np.random.default_rng(9)
    op = GrayScott(n, 1e-2, 5e-3, 0.04, 0.06)
    u0 = np.concatenate([1 - 0.2 * rng.random(n * n), 0.04 * rng.random(n * n)])
    return op, u0


@pytest.mark.parametrize("scheme", ["exprb43", "epirk5p1"])
def test_traditional_step_lands_error_near_tol(scheme):
    """e(dt) ~ C dt^(p+1): after a step of size dt with estimate e, a step of
    dt (tol/e)^(1/(p+1)) has an estimate close to tol; a wrong order exponent
    misses it by the ratio printed in the assertion."""
    op, u0 = _gs()
    step = integrators.STEPS[scheme]
    order = integrators.ORDER[scheme][1]

    def est(dt):
        uh, ul, _ = step(op, u0, dt, method="kiops", tol=1e-14)
        return np.linalg.norm(uh - ul) / math.sqrt(u0.size)

    dt = 0.5
    e = est(dt)
    tol = e * 1e-2
    e2 = est(adaptive.traditional(dt, e, tol, order))
    assert 0.5 < e2 / tol < 2.0, e2 / tol


@pytest.mark.parametrize("controller", ["traditional", "cost"])
def test_adaptive_run_invariants(controller):
    op, u0 = _gs()
    T = 4.0
    u, info = adaptive.integrate(op, u0, T, 0.05, 1e-7, scheme="exprb43", method="kiops", controller=controller,
                                 iter_tol=1e-12)
    assert info["status"] == 0 and info["t"] == pytest.approx(T, rel=0, abs=1e-12)
    assert sum(info["dts"]) == pytest.approx(T, rel=1e-13)
    assert max(info["errs"]) <= 1e-7
    assert info["accepted"] >= 3
    # a fine fixed-step reference: the adaptive run's global error is of the order of tol
    ref = u0.copy()
    for _ in range(256):
        ref = integrators.exprb43_step(op, ref, T / 256, method="kiops", tol=1e-13)[0]
    gerr = np.linalg.norm(u - ref) / math.sqrt(u.size)
    assert gerr < 1e-5


def test_global_error_shrinks_with_tol():
    op, u0 = _gs()
    T = 4.0
    ref = u0.copy()
    for _ in range(256):
        ref = integrators.exprb43_step(op, ref, T / 256, method="kiops", tol=1e-13)[0]
    errs = []
    for tol in (1e-5, 1e-7):
        u, info = adaptive.integrate(op, u0, T, 0.05, tol, scheme="exprb43", method="kiops", iter_tol=1e-12)
        errs.append(np.linalg.norm(u - ref) / math.sqrt(u.size))
    assert errs[1] < 0.1 * errs[0]
