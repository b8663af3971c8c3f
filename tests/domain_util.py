"""A CPU backend for the domain-decomposed Leja driver (paper_2211_08948_gb300.domain):
the per-block operations written in NumPy on float64 CPU torch tensors, so
that the driver's decomposition, halo exchange, allreduce schedule and stop
logic run under gloo ranks without a GPU.  The block stencils restate the
operators of oracle.operators on a padded block (one halo cell, the global
grid spacing); the coefficient tables come from the oracle."""
import math

import numpy as np
import torch

from oracle import leja


class Desc:
    def __init__(self, kind, gnx, gny, x0, y0, bx, by, params, state):
        self.kind, self.gnx, self.gny, self.x0, self.y0 = kind, gnx, gny, x0, y0
        self.bx, self.by, self.params, self.state = bx, by, list(params), state


def ncomp(kind):
    return 2 if kind == 1 else 1


def block_jv(d, y):
    """J y on the interior of a padded block (numpy arrays of shape (nc, by+2, bx+2))."""
    dx, dy = 1.0 / d.gnx, 1.0 / d.gny
    c = (slice(None), slice(1, -1), slice(1, -1))
    e = y[:, 1:-1, 2:]
    w = y[:, 1:-1, :-2]
    n = y[:, 2:, 1:-1]
    s = y[:, :-2, 1:-1]
    yc = y[c]
    lap = (e + w - 2 * yc) / dx ** 2 + (n + s - 2 * yc) / dy ** 2
    ddx = (e - w) / (2 * dx)
    ddy = (n - s) / (2 * dy)
    p = d.params
    if d.kind == 0:
        return p[0] * lap + p[1] * ddx + p[2] * ddy
    st = d.state.numpy().reshape(y.shape)
    if d.kind == 1:
        U, V = st[0, 1:-1, 1:-1], st[1, 1:-1, 1:-1]
        Du, Dv, F, k = p[:4]
        ju = Du * lap[0] - V * V * yc[0] - 2 * U * V * yc[1] - F * yc[0]
        jv = Dv * lap[1] + V * V * yc[0] + 2 * U * V * yc[1] - (F + k) * yc[1]
        return np.stack([ju, jv])
    Uc = st[:, 1:-1, 1:-1]
    Ux = (st[:, 1:-1, 2:] - st[:, 1:-1, :-2]) / (2 * dx)
    Uy = (st[:, 2:, 1:-1] - st[:, :-2, 1:-1]) / (2 * dy)
    return p[0] * lap - (Ux + Uy) * yc - Uc * (ddx + ddy)


class CpuBackend:
    """Backend interface of the domain driver, on CPU torch tensors."""

    def zeros(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def view(self, buf, sl):
        return buf[sl]

    def copy(self, dst, dsl, src, ssl):
        dst[dsl] = src[ssl]

    def to_host(self, t):
        return t.numpy().copy()

    def accumulate(self, dst, srcs):
        dst.copy_(srcs[0])
        for t in srcs[1:]:
            dst.add_(t)

    def _pad(self, d, t):
        return t.numpy().reshape(ncomp(d.kind), d.by + 2, d.bx + 2)

    def set_interior(self, d, y_pad, v):
        self._pad(d, y_pad)[:, 1:-1, 1:-1] = np.asarray(v).reshape(ncomp(d.kind), d.by, d.bx)

    def block(self, kind, dec, r, params, state):
        b = dec.blocks[r]
        return Desc(kind, dec.nx, dec.ny, b["x0"], b["y0"], b["bx"], b["by"], params, state)

    def newton(self, d, y_in, y_out, p, dk, a, b, norms):
        yi = self._pad(d, y_in)
        if y_out is None:
            y = yi[:, 1:-1, 1:-1].copy()
        else:
            y = a * block_jv(d, yi) + b * yi[:, 1:-1, 1:-1]
            self._pad(d, y_out)[:, 1:-1, 1:-1] = y
        nv = norms.numpy()
        nv[0] = float(np.sum(y * y))
        for k, pk in enumerate(p):
            pv = pk.numpy()
            new = dk[k] * y.reshape(-1) if y_out is None else pv + dk[k] * y.reshape(-1)
            pv[:] = new
            nv[1 + k] = float(np.sum(new * new))

    def faces(self, d, direction, y_pad, buf):
        yp = self._pad(d, y_pad)
        bv = buf.numpy()
        nc, bx, by = ncomp(d.kind), d.bx, d.by
        o = 0
        for name in ("S", "N", "W", "E"):
            if name == "S":
                cell = (slice(None), 0 if direction else 1, slice(1, bx + 1))
            elif name == "N":
                cell = (slice(None), by + 1 if direction else by, slice(1, bx + 1))
            elif name == "W":
                cell = (slice(None), slice(1, by + 1), 0 if direction else 1)
            else:
                cell = (slice(None), slice(1, by + 1), bx + 1 if direction else bx)
            L = nc * (bx if name in ("S", "N") else by)
            if direction:
                yp[cell] = bv[o:o + L].reshape(yp[cell].shape)
            else:
                bv[o:o + L] = yp[cell].reshape(-1)
            o += L

    def start(self, d, seed, y_pad):
        nc = ncomp(d.kind)
        g = leja.splitmix64_uniform(seed, nc * d.gnx * d.gny).reshape(nc, d.gny, d.gnx)
        self._pad(d, y_pad)[:, 1:-1, 1:-1] = g[:, d.y0:d.y0 + d.by, d.x0:d.x0 + d.bx]

    def stop(self, K, m, m_min, dkm, tol, ysq, psq):
        if not math.isfinite(ysq) or not all(math.isfinite(x) for x in psq):
            return -1
        ok = m >= m_min and all(abs(dkm[k]) * math.sqrt(ysq) <= tol * math.sqrt(psq[k]) for k in range(K))
        return 1 if ok else 0

    def leja_points(self, m):
        return list(leja.leja_points(m))

    def divided_differences(self, l, a, b, m):
        xi = leja.leja_points(m)
        return list(leja.phi_coefficients(xi, l, 1.0, a, b))


def oracle_pass(jv, v, h, alpha, beta, outputs, tol, iters_extra=0, m_max=500):
    """The unsplit oracle's vertical Newton-Leja pass (Sec. 2.2), optionally
    carried iters_extra iterations past its stop (the lagged pass's result).
    Returns (list of p_k, iterations)."""
    gamma = 0.25 * (beta - alpha)
    c = 0.5 * (alpha + beta)
    xi = leja.leja_points(m_max + 1)
    coeffs = [leja.phi_coefficients(xi, l, s * h, c, gamma) for (l, s) in outputs]
    p, m, st = leja.leja_pass(jv, v, xi, coeffs, c, gamma, tol, m_max)
    assert st == 0
    if iters_extra:
        p, m2, _ = leja.leja_pass(jv, v, xi, coeffs, c, gamma, 0.0, m + iters_extra)
        assert m2 == m + iters_extra
        m = m2
    return p, m
