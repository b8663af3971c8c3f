"""Comparison variants of the Leja path (Sec. 4; Appendix A).

* Finite-difference ("numerical") Jacobian-vector products: the paper's
  runs form J(u) w from the right-hand side alone (Sec. 4, "computing the
  numerical Jacobian"):  J w ~ (f(u + eps w) - f(u)) / eps.  Reading (the
  paper does not give eps): eps = sqrt(2^-52) (1 + ||u||) / ||w||, the usual
  choice that balances truncation O(eps) against rounding O(2^-52 / eps).
* Augmented-matrix Leja (Appendix A): the linear combination
  sum_{j=0}^{p} phi_j(hJ) b_j evaluated as the exponential of the augmented
  matrix of the Theorem of Sec. 2.1, A~ = [[hJ, B], [0, K]], applied to
  [b_0; e_p] by one Leja interpolation of exp on the spectral interval of hJ
  (the eigenvalues of A~ are those of hJ and 0).  The paper reports this as
  slower than the individual phi-actions; it is kept as a comparison.

TEST INFRASTRUCTURE: part of the CPU oracle (see oracle/__init__.py).
"""
import math

import numpy as np

from . import leja


def fd_jv(f, u, fu=None):
    """w -> (f(u + eps w) - f(u)) / eps with eps = sqrt(2^-52) (1 + ||u||) / ||w||."""
    fu = f(u) if fu is None else fu
    nu = float(np.linalg.norm(u))

    def jv(w):
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            return np.zeros_like(w)
        eps = math.sqrt(2.0 ** -52) * (1.0 + nu) / nw
        return (f(u + eps * w) - fu) / eps

    return jv


def augmented_operator(jv, bs, h):
    """x -> A~ x on R^(N+p) for A~ = [[h J, B], [0, K]], B = [b_p .. b_1] as in
    oracle.kiops (tail entry t = p - j carries b_j), K the upward shift."""
    p = len(bs) - 1
    N = next(len(b) for b in bs if b is not None)
    B = [np.zeros(N) if b is None else np.asarray(b, dtype=np.float64) for b in bs]

    def apply(x):
        y = np.empty_like(x)
        y[:N] = h * jv(x[:N])
        for i in range(1, p + 1):
            y[:N] += B[p + 1 - i] * x[N + i - 1]
        y[N:N + p - 1] = x[N + 1:N + p]
        if p > 0:
            y[N + p - 1] = 0.0
        return y

    return apply, N, p


def leja_combination_augmented(jv, bs, h, alpha, beta, tol, m_max=500):
    """sum_j phi_j(hJ) bs[j] by Leja interpolation of exp on A~ (interval
    [alpha, beta] of J's real spectrum, scaled by h).  Returns (vector, iters)."""
    apply, N, p = augmented_operator(jv, bs, h)
    x0 = np.zeros(N + p)
    if bs[0] is not None:
        x0[:N] = bs[0]
    if p > 0:
        x0[N + p - 1] = 1.0
    gamma = 0.25 * (beta - alpha) * h
    c = 0.5 * (alpha + beta) * h
    xi = leja.leja_points(m_max + 1)
    coeff = leja.phi_coefficients(xi, 0, 1.0, c, gamma)
    (pv,), m, st = leja.leja_pass(apply, x0, xi, [coeff], c, gamma, tol, m_max)
    if st != 0:
        raise RuntimeError("augmented Leja did not converge")
    return pv[:N], m
