"""The paper's non-periodic test problems (Sec. 3) on cell-centred grids with
homogeneous Neumann ("no-flow") boundaries, second-order centred
differences (Sec. 3):

  ADR           u_t = a lap u + b (u_x + u_y) + g u (1 - u) (u - 1/2)   on [0, 1]^2
  Allen-Cahn    u_t = a lap u + u - u^3                                 on [-1, 1]^2
  Brusselator   u_t = a lap u + 1 + u^2 v - 4 u,
                v_t = a lap v + 3 u - u^2 v                             on [0, 1]^2

Readings (the CUDA library follows the same):
* cell-centred nodes x_i = x0 + (i + 1/2) dx, dx = L / n; the Neumann
  condition puts a ghost cell equal to the boundary cell on every side
  (u_{-1} = u_0, u_n = u_{n-1}), which makes the discrete Laplacian symmetric
  with the constants in its null space; the centred first derivative uses
  the same ghosts (it vanishes at the wall to first order).
* "b nabla u" of the ADR equation is b (u_x + u_y), advection along the
  diagonal, as in the periodic advection-diffusion operator.
* the Brusselator is the standard form of the cited reference (u^2 v in both
  equations, a lap v in the second); the printed text has u v^2 in the first
  equation and a lap u in the second, which read as transcription slips.
Vectors are planar (species, y, x), float64.
"""
import numpy as np


def _pad(U):
    return np.pad(U, 1, mode="edge")  # Neumann ghosts: the boundary cell repeated


def lap_n(U, dx, dy):
    P = _pad(U)
    return (P[1:-1, 2:] + P[1:-1, :-2] - 2.0 * U) / (dx * dx) + (P[2:, 1:-1] + P[:-2, 1:-1] - 2.0 * U) / (dy * dy)


def ddx_n(U, dx):
    P = _pad(U)
    return (P[1:-1, 2:] - P[1:-1, :-2]) / (2.0 * dx)


def ddy_n(U, dy):
    P = _pad(U)
    return (P[2:, 1:-1] - P[:-2, 1:-1]) / (2.0 * dy)


class ADR:
    """Advection-diffusion-reaction with Neumann boundaries on [0, 1]^2."""
    ncomp = 1
    L = 1.0

    def __init__(self, n, a, b, g, state=None, ny=None):
        self.n, self.a, self.b, self.g = n, a, b, g
        self.ny = n if ny is None else ny
        self.dx, self.dy = self.L / n, self.L / self.ny
        self.state = state

    def f(self, u):
        U = u.reshape(self.ny, self.n)
        return (self.a * lap_n(U, self.dx, self.dy) + self.b * (ddx_n(U, self.dx) + ddy_n(U, self.dy))
                + self.g * U * (1.0 - U) * (U - 0.5)).reshape(-1)

    def jv(self, w):
        U = self.state.reshape(self.ny, self.n)
        W = w.reshape(self.ny, self.n)
        dg = -3.0 * U * U + 3.0 * U - 0.5  # d/du of u (1 - u) (u - 1/2)
        return (self.a * lap_n(W, self.dx, self.dy) + self.b * (ddx_n(W, self.dx) + ddy_n(W, self.dy))
                + self.g * dg * W).reshape(-1)


class AllenCahn:
    """Allen-Cahn with no-flow boundaries on [-1, 1]^2."""
    ncomp = 1
    L = 2.0

    def __init__(self, n, a, state=None, ny=None):
        self.n, self.a = n, a
        self.ny = n if ny is None else ny
        self.dx, self.dy = self.L / n, self.L / self.ny
        self.state = state

    def f(self, u):
        U = u.reshape(self.ny, self.n)
        return (self.a * lap_n(U, self.dx, self.dy) + U - U ** 3).reshape(-1)

    def jv(self, w):
        U = self.state.reshape(self.ny, self.n)
        W = w.reshape(self.ny, self.n)
        return (self.a * lap_n(W, self.dx, self.dy) + (1.0 - 3.0 * U * U) * W).reshape(-1)


class Brusselator:
    """Two-species Brusselator with Neumann boundaries on [0, 1]^2."""
    ncomp = 2
    L = 1.0

    def __init__(self, n, a, state=None, ny=None):
        self.n, self.a = n, a
        self.ny = n if ny is None else ny
        self.dx, self.dy = self.L / n, self.L / self.ny
        self.state = state

    def _split(self, x):
        nn = self.n * self.ny
        return x[:nn].reshape(self.ny, self.n), x[nn:].reshape(self.ny, self.n)

    def f(self, x):
        u, v = self._split(x)
        uuv = u * u * v
        fu = self.a * lap_n(u, self.dx, self.dy) + 1.0 + uuv - 4.0 * u
        fv = self.a * lap_n(v, self.dx, self.dy) + 3.0 * u - uuv
        return np.concatenate([fu.reshape(-1), fv.reshape(-1)])

    def jv(self, w):
        U, V = self._split(self.state)
        du, dv = self._split(w)
        ju = self.a * lap_n(du, self.dx, self.dy) + (2.0 * U * V - 4.0) * du + U * U * dv
        jw = self.a * lap_n(dv, self.dx, self.dy) + (3.0 - 2.0 * U * V) * du - U * U * dv
        return np.concatenate([ju.reshape(-1), jw.reshape(-1)])


def with_state(op, state):
    """Copy of a problem linearised at `state`."""
    if isinstance(op, ADR):
        return ADR(op.n, op.a, op.b, op.g, state, ny=op.ny)
    if isinstance(op, AllenCahn):
        return AllenCahn(op.n, op.a, state, ny=op.ny)
    return Brusselator(op.n, op.a, state, ny=op.ny)
