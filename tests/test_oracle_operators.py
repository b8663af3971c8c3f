"""Pins for oracle.operators and oracle.exact: closed-form stencil eigenvalues,
finite-difference Jacobians, FFT sign convention, augmented-matrix theorem."""
import math

import numpy as np
import pytest

import synth
from oracle import exact
from oracle.operators import AdvDiff, GrayScott, Burgers, remainder
from oracle.phi import phi_scalar


def test_laplacian_and_advection_on_fourier_mode():
    n = 20
    X, Y = synth.grid_xy(n)
    k = 3
    u = np.sin(2 * np.pi * k * X).reshape(-1)
    dx = 1.0 / n
    lap_eig = (2 * np.cos(2 * np.pi * k * dx) - 2) / dx ** 2
    op = AdvDiff(n, 1.0, 0.0, 0.0)
    assert np.allclose(op.f(u), lap_eig * u, atol=1e-9 * abs(lap_eig))
    op = AdvDiff(n, 0.0, 1.0, 0.0)
    ref = (np.sin(2 * np.pi * k * dx) / dx) * np.cos(2 * np.pi * k * X).reshape(-1)
    assert np.allclose(op.f(u), ref, atol=1e-10)
    opy = AdvDiff(n, 0.0, 0.0, 1.0)
    uy = np.sin(2 * np.pi * k * Y).reshape(-1)
    refy = (np.sin(2 * np.pi * k * dx) / dx) * np.cos(2 * np.pi * k * Y).reshape(-1)
    assert np.allclose(opy.f(uy), refy, atol=1e-10)


def test_fft_eigenvalues_match_stencil():
    n, D, ax, ay = 12, 0.3, 4.0, -2.5
    op = AdvDiff(n, D, ax, ay)
    v = np.random.default_rng(0).standard_normal(n * n)
    lam = exact.advdiff_eigenvalues(n, D, ax, ay)
    via_fft = np.fft.ifft2(np.fft.fft2(v.reshape(n, n)) * lam).real.reshape(-1)
    assert np.allclose(via_fft, op.jv(v), rtol=1e-12, atol=1e-9)


def test_grayscott_uniform_state_reaction_values():
    n = 4
    u = np.concatenate([np.full(n * n, 0.8), np.full(n * n, 0.25)])
    op = GrayScott(n, 1.0, 0.5, 0.04, 0.06)
    f = op.f(u)
    # no diffusion on a uniform state: f_u = -u v^2 + F(1-u), f_v = u v^2 - (F+k) v
    assert np.allclose(f[: n * n], -0.8 * 0.0625 + 0.04 * 0.2)
    assert np.allclose(f[n * n:], 0.8 * 0.0625 - 0.1 * 0.25)


@pytest.mark.parametrize("kind", ["gs", "burgers", "advdiff"])
def test_jacobian_is_derivative_of_f(kind):
    rng = np.random.default_rng(1)
    n = 9
    if kind == "gs":
        op = GrayScott(n, 2e-3, 1e-3, 0.04, 0.06)
        u = 0.5 + 0.3 * rng.random(2 * n * n)
    elif kind == "burgers":
        op = Burgers(n, 1e-2)
        u = rng.standard_normal(n * n)
    else:
        op = AdvDiff(n, 0.2, 3.0, 1.0)
        u = rng.standard_normal(n * n)
    op.state = u
    w = rng.standard_normal(u.size)
    eps = 1e-6
    fd = (op.f(u + eps * w) - op.f(u - eps * w)) / (2 * eps)
    assert np.linalg.norm(op.jv(w) - fd) <= 1e-7 * np.linalg.norm(fd)


def test_remainder_linear_is_zero_and_quadratic():
    rng = np.random.default_rng(2)
    n = 8
    lin = AdvDiff(n, 0.1, 1.0, 2.0)
    u = rng.standard_normal(n * n)
    a = u + rng.standard_normal(n * n)
    assert np.linalg.norm(remainder(lin, u, a)) <= 1e-12 * np.linalg.norm(lin.f(a))
    gs = GrayScott(n, 1e-3, 5e-4, 0.04, 0.06)
    U = 0.5 + 0.3 * rng.random(2 * n * n)
    gs.state = U
    d = rng.standard_normal(U.size)
    r1 = np.linalg.norm(remainder(gs, U, U + 1e-2 * d))
    r2 = np.linalg.norm(remainder(gs, U, U + 5e-3 * d))
    assert r1 / r2 == pytest.approx(4.0, rel=0.05)


def test_augmented_theorem_scalar_case():
    # 1x1 A = [a]: sum_j phi_j(a) b_j with scalar phi (pinned against mpmath)
    a = -3.7
    bs = [np.array([0.4]), np.array([-1.1]), np.array([2.0]), np.array([0.3])]
    got = exact.augmented_phi_sum(np.array([[a]]), bs)[0]
    ref = sum(phi_scalar(j, a) * b[0] for j, b in enumerate(bs))
    assert got == pytest.approx(ref, rel=1e-13)


def test_fft_phi_matches_dense_augmented():
    n, D, ax, ay, t = 6, 0.05, 1.0, 0.7, 0.8
    op = AdvDiff(n, D, ax, ay)
    A = exact.dense_matrix(op.jv, n * n)
    v = np.random.default_rng(4).standard_normal(n * n)
    for l in range(4):
        f = exact.advdiff_phi_fft(n, D, ax, ay, t, v, l)
        d = exact.dense_phi(t * A, l, v)
        assert np.linalg.norm(f - d) <= 1e-11 * np.linalg.norm(d)


def test_dense_phi_taylor_small_matrix():
    rng = np.random.default_rng(6)
    A = 1e-3 * rng.standard_normal((5, 5))
    v = rng.standard_normal(5)
    for l in range(4):
        # phi_l(A) v = sum_k A^k v / (k+l)!  (converges in a few terms for ||A|| ~ 1e-3)
        ref = np.zeros(5)
        t = v.copy()
        for k in range(12):
            ref += t / math.factorial(k + l)
            t = A @ t
        assert np.allclose(exact.dense_phi(A, l, v), ref, rtol=1e-13, atol=1e-15)


def test_rectangular_grid_modes():
    # on an nx x ny grid, sin(2 pi kx x) sin(2 pi ky y) is an eigenvector of the
    # centred Laplacian with eigenvalue (2cos(2pi kx dx)-2)/dx^2 + (2cos(2pi ky dy)-2)/dy^2
    nx, ny, kx, ky = 12, 7, 2, 3
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    u = (np.sin(2 * np.pi * kx * X) * np.sin(2 * np.pi * ky * Y)).reshape(-1)
    lam = (2 * np.cos(2 * np.pi * kx / nx) - 2) * nx * nx + (2 * np.cos(2 * np.pi * ky / ny) - 2) * ny * ny
    op = AdvDiff(nx, 1.0, 0.0, 0.0, ny=ny)
    assert np.allclose(op.f(u), lam * u, atol=1e-9 * abs(lam))
    gs = GrayScott(nx, 1.0, 1.0, 0.0, 0.0, ny=ny)
    z = np.zeros(nx * ny)
    f = gs.f(np.concatenate([u, z]))
    assert np.allclose(f[: nx * ny], lam * u, atol=1e-9 * abs(lam))


def test_remainder_is_the_nonlinear_remainder():
    """The linear terms of f cancel in R(a) = f(a) - f(u) - J(u)(a - u) (Sec. 1):
    Gray-Scott keeps dv (a_u dv + 2 v du) with sign -/+ per species, Burgers
    keeps -d (D_x d + D_y d) with the central differences of f, advection-
    diffusion keeps 0.  The GPU stage kernel evaluates these forms; here they
    are compared with the definition, on a rectangular grid."""
    rng = np.random.default_rng(11)
    nx, ny = 24, 17
    N = nx * ny
    gs = GrayScott(nx, 2e-5, 1e-5, 0.04, 0.06, ny=ny)
    u = np.concatenate([1.0 - 0.3 * rng.random(N), 0.3 * rng.random(N)])
    a = u + 0.05 * rng.standard_normal(2 * N)
    R = remainder(GrayScott(nx, 2e-5, 1e-5, 0.04, 0.06, u, ny=ny), u, a)
    du, dv = a[:N] - u[:N], a[N:] - u[N:]
    r = dv * (a[:N] * dv + 2.0 * u[N:] * du)
    scale = np.linalg.norm(gs.f(a))
    assert np.max(np.abs(R - np.concatenate([-r, r]))) <= 1e-13 * scale
    assert np.linalg.norm(r) > 1e-4  # the remainder itself is not negligible here

    bu = Burgers(nx, 1e-3, ny=ny)
    ub = rng.standard_normal(N)
    ab = ub + 0.05 * rng.standard_normal(N)
    Rb = remainder(Burgers(nx, 1e-3, ub, ny=ny), ub, ab)
    d = (ab - ub).reshape(ny, nx)
    ddx = (np.roll(d, -1, 1) - np.roll(d, 1, 1)) * (0.5 * nx)
    ddy = (np.roll(d, -1, 0) - np.roll(d, 1, 0)) * (0.5 * ny)
    rb = (-d * (ddx + ddy)).reshape(-1)
    assert np.max(np.abs(Rb - rb)) <= 1e-13 * np.linalg.norm(bu.f(ab))
    assert np.linalg.norm(rb) > 1e-3

    ad = AdvDiff(nx, 1e-3, 0.3, -0.2, ny=ny)
    ua = rng.standard_normal(N)
    assert np.max(np.abs(remainder(ad, ua, ua + rng.standard_normal(N)))) <= 1e-12 * np.linalg.norm(ad.f(ua))
