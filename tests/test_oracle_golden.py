"""The oracle's integrator steps against the stage coefficients the paper
prints (Eq. exprb43, Sec. 5.4; Eq. epirk4s3, Sec. 5.1; Eq. epirk4s3a,
Sec. 5.2; Eq. exprb5s3, Sec. 5.5; Eq. epirk5p1 and its table, Sec. 5.3),
stored in tests/golden/.  With f(x) = d^2 + d^3 + c elementwise (d = x - u0) and the
step taken at u0, the Jacobian J(u0) vanishes, every phi_l(s J h) reduces to
1/l!, and the nonlinear remainder is R(x) = d^2 + d^3: each stage is then an
explicit polynomial in the printed coefficients, so a wrong coefficient,
stage scale or phi index in the oracle changes the result.  (Both powers are
needed: for a purely quadratic R the printed EPIRK4s3 error-estimate
combination vanishes identically, for a purely cubic one its third stage.)"""
import math
import os

import numpy as np
import pytest

from oracle import integrators

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = (s.strip() for s in line.split("="))
        vals[k] = float(v)
    return vals


class Polynomial:
    """f(x) = d^2 + d^3 + c, d = x - u0, on a 1 x n grid; J(u0) = 0."""
    ncomp = 1

    def __init__(self, u0, c):
        self.u0, self.c = u0, c
        self.n, self.ny = u0.size, 1

    def f(self, x):
        d = x - self.u0
        return d * d + d * d * d + self.c

    def jv(self, w):
        return 0.0 * w


def close(got, want):
    """Each stage increment to 1e-11 of its own size (the printed coefficients,
    up to 42336, amplify rounding)."""
    assert np.max(np.abs(want)) > 1e-6  # not a vanishing combination
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def _case():
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, 37)
    c = rng.uniform(0.5, 2.0, 37)
    return u0, c, 0.3


def test_exprb43_matches_printed_coefficients():
    g = read_golden("exprb43.txt")
    u0, c, h = _case()
    u4, u3, st = integrators.exprb43_step(Polynomial(u0, c), u0, h, method="kiops", tol=1e-13)
    R = lambda x: (x - u0) ** 2 + (x - u0) ** 3
    a = u0 + g["c_a"] * c * h                     # phi_1(0) = 1
    b = u0 + c * h + R(a) * h
    e3 = u0 + c * h + (g["r3a"] * R(a) + g["r3b"] * R(b)) * h / math.factorial(3)
    e4 = e3 + (g["r4a"] * R(a) + g["r4b"] * R(b)) * h / math.factorial(4)
    close(u3 - u0, e3 - u0)
    close(u4 - u3, e4 - e3)


@pytest.mark.parametrize("method", ["kiops", "lekry"])
def test_epirk4s3_matches_printed_coefficients(method):
    g = read_golden("epirk4s3.txt")
    u0, c, h = _case()
    u4, u3, st = integrators.epirk4s3_step(Polynomial(u0, c), u0, h, method=method, tol=1e-13)
    R = lambda x: (x - u0) ** 2 + (x - u0) ** 3
    a = u0 + g["c_a"] * c * h
    b = u0 + g["c_b"] * c * h
    d = R(b) - 2.0 * R(a)
    e3 = u0 + c * h + (g["r3a"] * R(a) + g["r3d"] * d) * h / math.factorial(3)
    e4 = e3 + (g["r4a"] * R(a) + g["r4d"] * d) * h / math.factorial(4)
    close(u3 - u0, e3 - u0)
    close(u4 - u3, e4 - e3)


@pytest.mark.parametrize("method", ["kiops", "lekry"])
def test_epirk4s3a_matches_printed_coefficients(method):
    g = read_golden("epirk4s3a.txt")
    u0, c, h = _case()
    u4, u3, st = integrators.epirk4s3a_step(Polynomial(u0, c), u0, h, method=method, tol=1e-13)
    R = lambda x: (x - u0) ** 2 + (x - u0) ** 3
    a = u0 + g["c_a"] * c * h
    b = u0 + g["c_b"] * c * h
    e3 = u0 + c * h + (g["r3a"] * R(a) + g["r3b"] * R(b)) * h / math.factorial(3)
    e4 = e3 + (g["r4a"] * R(a) + g["r4b"] * R(b)) * h / math.factorial(4)
    close(u3 - u0, e3 - u0)
    close(u4 - u3, e4 - e3)


@pytest.mark.parametrize("method", ["kiops", "lekry"])
def test_exprb53s3_matches_printed_coefficients(method):
    g = read_golden("exprb53s3.txt")
    u0, c, h = _case()
    u5, u3, st = integrators.exprb53s3_step(Polynomial(u0, c), u0, h, method=method, tol=1e-13)
    R = lambda x: (x - u0) ** 2 + (x - u0) ** 3
    a = u0 + g["c_a"] * c * h
    b = u0 + g["c_b"] * c * h + (g["q_a"] + g["q_b"]) * R(a) * h / math.factorial(3)
    e3 = u0 + c * h + (g["r3a"] * R(a) + g["r3b"] * R(b)) * h / math.factorial(3)
    e5 = (u0 + c * h + (g["r5a"] * R(a) + g["r5b"] * R(b)) * h / math.factorial(3)
          + (g["r5c"] * R(a) + g["r5d"] * R(b)) * h / math.factorial(4))
    close(u3 - u0, e3 - u0)
    close(u5 - u3, e5 - e3)


def test_epirk5p1_matches_printed_coefficients():
    g = read_golden("epirk5p1.txt")
    u0, c, h = _case()
    u5, u4, st = integrators.epirk5p1_step(Polynomial(u0, c), u0, h, method="kiops", tol=1e-13)
    R = lambda x: (x - u0) ** 2 + (x - u0) ** 3
    a = u0 + g["a11"] * c * h
    b = u0 + g["a21"] * c * h + g["a22"] * R(a) * h
    w = (-2.0 * R(a) + R(b)) * h / math.factorial(3)
    e4 = u0 + g["b1"] * c * h + g["b2"] * R(a) * h + g["b3"] * w
    close(u4 - u0, e4 - u0)
    close(u5 - u0, e4 - u0)   # with J = 0 the hatted and plain scales coincide
