"""2D periodic finite-difference right-hand sides f(u) and Jacobian actions J(u)w.

Sec. 3 of the paper discretises nabla and nabla^2 with second-order centred
differences; the paper's exponential integrators use f and the matrix-free
Jacobian action (Sec. 2, "matrix-free implementation ... computation of the
RHS functions").  Grids are n x n on the periodic unit square, dx = 1/n,
vectors planar (species, y, x), float64.

Grids may be rectangular: n is the number of columns (x), ny (default n) the
number of rows, dx = 1/n, dy = 1/ny.

Operators:
* advection-diffusion  f(u) = D lap(u) + ax u_x + ay u_y    (linear, J = f)
* Gray-Scott (Sec. 3)  f_u = Du lap(u) - u v^2 + F (1 - u)
                       f_v = Dv lap(v) + u v^2 - (F + k) v
* viscous Burgers      f(u) = nu lap(u) - u (u_x + u_y)
The nonlinear remainder of Sec. 1 is R(a) = F(a) - F(u), F(x) = f(x) - J(u)x.
"""
import numpy as np


def _lap(u, dx, dy):
    return (np.roll(u, 1, 1) + np.roll(u, -1, 1) - 2.0 * u) / (dx * dx) \
        + (np.roll(u, 1, 0) + np.roll(u, -1, 0) - 2.0 * u) / (dy * dy)


def _ddx(u, dx):
    # centred difference along x (axis 1): (u[j+1] - u[j-1]) / (2 dx)
    return (np.roll(u, -1, 1) - np.roll(u, 1, 1)) / (2.0 * dx)


def _ddy(u, dy):
    return (np.roll(u, -1, 0) - np.roll(u, 1, 0)) / (2.0 * dy)


class AdvDiff:
    """Linear 2D periodic advection-diffusion (Sec. 3 discretisation)."""
    ncomp = 1

    def __init__(self, n, D, ax, ay, ny=None):
        self.n, self.D, self.ax, self.ay = n, D, ax, ay
        self.ny = n if ny is None else ny
        self.dx, self.dy = 1.0 / n, 1.0 / self.ny

    def f(self, u):
        U = u.reshape(self.ny, self.n)
        return (self.D * _lap(U, self.dx, self.dy) + self.ax * _ddx(U, self.dx)
                + self.ay * _ddy(U, self.dy)).reshape(-1)

    def jv(self, w):
        return self.f(w)


class GrayScott:
    """Gray-Scott reaction-diffusion, Sec. 3 (a = F feed, b = k kill)."""
    ncomp = 2

    def __init__(self, n, Du, Dv, F, k, state=None, ny=None):
        self.n, self.Du, self.Dv, self.F, self.k = n, Du, Dv, F, k
        self.ny = n if ny is None else ny
        self.dx, self.dy = 1.0 / n, 1.0 / self.ny
        self.state = state

    def _split(self, x):
        nn = self.n * self.ny
        return x[:nn].reshape(self.ny, self.n), x[nn:].reshape(self.ny, self.n)

    def f(self, x):
        u, v = self._split(x)
        uvv = u * v * v
        fu = self.Du * _lap(u, self.dx, self.dy) - uvv + self.F * (1.0 - u)
        fv = self.Dv * _lap(v, self.dx, self.dy) + uvv - (self.F + self.k) * v
        return np.concatenate([fu.reshape(-1), fv.reshape(-1)])

    def jv(self, w):
        U, V = self._split(self.state)
        du, dv = self._split(w)
        ju = self.Du * _lap(du, self.dx, self.dy) - (V * V + self.F) * du - 2.0 * U * V * dv
        jvv = self.Dv * _lap(dv, self.dx, self.dy) + V * V * du + (2.0 * U * V - (self.F + self.k)) * dv
        return np.concatenate([ju.reshape(-1), jvv.reshape(-1)])


class Burgers:
    """2D viscous Burgers u_t = nu lap(u) - u (u_x + u_y)."""
    ncomp = 1

    def __init__(self, n, nu, state=None, ny=None):
        self.n, self.nu = n, nu
        self.ny = n if ny is None else ny
        self.dx, self.dy = 1.0 / n, 1.0 / self.ny
        self.state = state

    def f(self, u):
        U = u.reshape(self.ny, self.n)
        return (self.nu * _lap(U, self.dx, self.dy) - U * (_ddx(U, self.dx) + _ddy(U, self.dy))).reshape(-1)

    def jv(self, w):
        U = self.state.reshape(self.ny, self.n)
        W = w.reshape(self.ny, self.n)
        g = _ddx(U, self.dx) + _ddy(U, self.dy)
        return (self.nu * _lap(W, self.dx, self.dy) - W * g
                - U * (_ddx(W, self.dx) + _ddy(W, self.dy))).reshape(-1)


def with_state(op, state):
    """Copy of a nonlinear operator linearised at `state` (J(u^n), Sec. 1)."""
    from . import problems
    if isinstance(op, (problems.ADR, problems.AllenCahn, problems.Brusselator)):
        return problems.with_state(op, state)
    if isinstance(op, GrayScott):
        return GrayScott(op.n, op.Du, op.Dv, op.F, op.k, state, ny=op.ny)
    if isinstance(op, Burgers):
        return Burgers(op.n, op.nu, state, ny=op.ny)
    return op


def remainder(op_at_u, u, a, fu=None, fa=None):
    """R(a) = F(a) - F(u) with F(x) = f(x) - J(u^n) x  (Sec. 1)."""
    fu = op_at_u.f(u) if fu is None else fu
    fa = op_at_u.f(a) if fa is None else fa
    return fa - fu - op_at_u.jv(a - u)
