"""The oracle's non-periodic problems (Sec. 3) and the comparison variants
(finite-difference Jacobian products, augmented-matrix Leja, Appendix A)
against closed forms and definitions: the cell-centred Neumann Laplacian's
cosine eigenmodes and null space, each Jacobian action as the derivative of
its right-hand side, the finite-difference product against the analytic one,
and the augmented Leja combination against the dense augmented exponential."""
import math

import numpy as np
import pytest

import synth
from oracle import problems, variants, exact, leja, kiops
from oracle.operators import AdvDiff, GrayScott


def test_neumann_laplacian_cosine_modes_and_constants():
    n, L = 12, 2.0
    dx = L / n
    i = np.arange(n) + 0.5
    for kx, ky in [(0, 0), (1, 0), (3, 5), (11, 7)]:
        U = np.outer(np.cos(math.pi * ky * i / n), np.cos(math.pi * kx * i / n))
        lam = -(4.0 / dx ** 2) * (math.sin(math.pi * kx / (2 * n)) ** 2 + math.sin(math.pi * ky / (2 * n)) ** 2)
        assert np.allclose(problems.lap_n(U, dx, dx), lam * U, atol=1e-9 * max(1.0, abs(lam)))
    # diffusion conserves the total (no flux through the walls)
    U = np.random.default_rng(1).random((n, n))
    assert abs(problems.lap_n(U, dx, dx).sum()) < 1e-9


@pytest.mark.parametrize("kind", ["adr", "allen_cahn", "brusselator"])
def test_jacobian_is_the_derivative_of_f(kind):
    n = 10
    rng = np.random.default_rng(2)
    if kind == "adr":
        op, u = problems.ADR(n, 0.1, -10.0, 100.0), synth.adr_state(n)
    elif kind == "allen_cahn":
        op, u = problems.AllenCahn(n, 0.01), synth.allen_cahn_state(n)
    else:
        op, u = problems.Brusselator(n, 0.01), synth.brusselator_state(n)
    u = u + 0.05 * rng.standard_normal(u.size)
    w = rng.standard_normal(u.size)
    jw = problems.with_state(op, u).jv(w)
    e = 1e-5
    cd = (op.f(u + e * w) - op.f(u - e * w)) / (2 * e)  # central difference, O(e^2)
    assert np.linalg.norm(cd - jw) <= 1e-7 * np.linalg.norm(jw)


def test_fd_jacobian_product():
    n = 12
    rng = np.random.default_rng(3)
    # linear operator: the finite difference is exact up to rounding / eps
    op = AdvDiff(n, 0.5, 3.0, 2.0)
    u = rng.random(n * n)
    w = rng.standard_normal(n * n)
    assert np.linalg.norm(variants.fd_jv(op.f, u)(w) - op.jv(w)) <= 1e-6 * np.linalg.norm(op.jv(w))
    # nonlinear: truncation O(eps), eps ~ 1.5e-8 (1 + ||u||) / ||w||
    gs = GrayScott(n, 1e-3, 5e-4, 0.04, 0.06)
    x = np.concatenate([1 - 0.3 * rng.random(n * n), 0.3 * rng.random(n * n)])
    v = rng.standard_normal(2 * n * n)
    ja = GrayScott(n, 1e-3, 5e-4, 0.04, 0.06, state=x).jv(v)
    jf = variants.fd_jv(gs.f, x)(v)
    assert np.linalg.norm(jf - ja) <= 1e-6 * np.linalg.norm(ja)
    assert np.linalg.norm(jf - ja) > 0.0


@pytest.mark.parametrize("p", [1, 3])
def test_augmented_leja_vs_dense_and_kiops(p):
    n = 8
    op = AdvDiff(n, 0.5, 3.0, 2.0)
    rng = np.random.default_rng(4)
    bs = [rng.standard_normal(n * n) for _ in range(p + 1)]
    bs[1] = None if p > 1 else bs[1]
    h = 0.01
    A = exact.dense_matrix(lambda x: h * op.jv(x), n * n)
    ref = exact.augmented_phi_sum(A, bs)
    got, m = variants.leja_combination_augmented(op.jv, bs, h, -8 * 0.5 * n * n, 0.0, 1e-12)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    kv, _ = kiops.kiops(lambda x: h * op.jv(x), bs, [1.0], 1e-12)
    assert np.linalg.norm(got - kv[0]) <= 1e-9 * np.linalg.norm(ref)
