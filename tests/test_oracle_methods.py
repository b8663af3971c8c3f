"""Pins for the oracle's Leja and KIOPS phi-actions and integrators against the
exact references (FFT diagonalisation, dense augmented expm)."""
import numpy as np
import pytest

import synth
from oracle import exact, kiops, leja, integrators
from oracle.operators import AdvDiff, GrayScott, Burgers, with_state


def _advdiff_case(n=32):
    prm = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    op = AdvDiff(n, prm["D"], prm["ax"], prm["ay"])
    return n, prm, v, op


def test_leja_advdiff_vs_fft_small():
    n, prm, v, op = _advdiff_case(32)
    h = prm["h"]
    alpha = -8 * prm["D"] * n * n
    res, info = leja.leja_phi(op.jv, v, h, alpha, 0.0, [(0, 1), (1, 1), (2, 1), (3, 1)], 1e-10, m_max=300)
    assert info["status"] == 0
    for l in range(4):
        ex = exact.advdiff_phi_fft(n, prm["D"], prm["ax"], prm["ay"], h, v, l)
        assert np.linalg.norm(res[l] - ex) <= 10 * 1e-10 * np.linalg.norm(ex)


def test_leja_vertical_equals_individual():
    n = 16
    D, ax, ay = 1.0, 1.0, 2.0
    op = AdvDiff(n, D, ax, ay)
    v = synth.advdiff_gaussian(n)
    h = 50.0 / (4 * D * n * n)
    alpha = -8 * D * n * n
    outs = [(1, 1.0 / 8), (1, 1.0 / 9), (1, 1.0)]
    res, info = leja.leja_phi(op.jv, v, h, alpha, 0.0, outs, 1e-12, m_max=300)
    assert info["status"] == 0 and info["substeps"] == 1
    for o, r in zip(outs, res):
        ex = exact.advdiff_phi_fft(n, D, ax, ay, o[1] * h, v, o[0])
        assert np.linalg.norm(r - ex) <= 1e-10 * np.linalg.norm(ex)
        single, _ = leja.leja_phi(op.jv, v, h, alpha, 0.0, [o], 1e-12, m_max=300)
        assert np.linalg.norm(r - single[0]) <= 1e-11 * np.linalg.norm(ex)


def test_leja_advection_heavy_needs_imaginary_substeps():
    n = 16
    D, ax, ay = 1.0, 10.0, 10.0
    op = AdvDiff(n, D, ax, ay)
    v = synth.advdiff_gaussian(n)
    h = 50.0 / (4 * D * n * n)
    alpha = -8 * D * n * n
    rho_im = (ax + ay) * n      # |Im lambda| <= (|ax| + |ay|) / dx
    outs = [(1, 1.0 / 8), (1, 1.0 / 9), (1, 1.0)]
    res, info = leja.leja_phi(op.jv, v, h, alpha, 0.0, outs, 1e-12, m_max=300,
                              rho_im=rho_im, iota_cap=4.0)
    assert info["status"] == 0 and info["substeps"] > 3
    for o, r in zip(outs, res):
        ex = exact.advdiff_phi_fft(n, D, ax, ay, o[1] * h, v, o[0])
        assert np.linalg.norm(r - ex) <= 1e-10 * np.linalg.norm(ex)


@pytest.mark.parametrize("kind", ["gs", "burgers"])
def test_leja_nonlinear_jacobian_vs_dense(kind):
    rng = np.random.default_rng(7)
    n = 8
    if kind == "gs":
        op = GrayScott(n, 2e-3, 1e-3, 0.04, 0.06)
        u = np.concatenate([1 - 0.3 * rng.random(n * n), 0.3 * rng.random(n * n)])
        h = 2.0
    else:
        op = Burgers(n, 5e-2)
        X, Y = synth.grid_xy(n)
        u = 0.5 * (np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)).reshape(-1) + 0.05 * rng.standard_normal(n * n)
        h = 0.2
    opu = with_state(op, u)
    A = exact.dense_matrix(opu.jv, u.size)
    lam = np.linalg.eigvals(A)
    rho = np.max(np.abs(lam))
    beta = max(0.0, 1.05 * np.max(lam.real))   # Burgers' reaction term can push Re(lambda) above 0
    v = rng.standard_normal(u.size)
    res, info = leja.leja_phi(opu.jv, v, h, -1.05 * rho, beta, [(0, 1), (1, 1), (3, 1)], 1e-11, m_max=300)
    assert info["status"] == 0
    for (l, _), r in zip([(0, 1), (1, 1), (3, 1)], res):
        ex = exact.dense_phi(h * A, l, v)
        assert np.linalg.norm(r - ex) <= 1e-9 * np.linalg.norm(ex)


def test_leja_substeps_vs_fft():
    n, prm, v, op = _advdiff_case(16)
    h = 4 * prm["h"]
    alpha = -8 * prm["D"] * n * n
    res, info = leja.leja_phi(op.jv, v, h, alpha, 0.0, [(0, 1), (2, 0.5)], 1e-11, m_max=300, gamma_cap=12.0)
    assert info["substeps"] > 2
    for (l, s), r in zip([(0, 1), (2, 0.5)], res):
        ex = exact.advdiff_phi_fft(n, prm["D"], prm["ax"], prm["ay"], s * h, v, l)
        assert np.linalg.norm(r - ex) <= 1e-9 * np.linalg.norm(ex)


def test_kiops_vs_fft_and_output_times():
    n, prm, v, op = _advdiff_case(32)
    h = prm["h"]
    A = lambda x: h * op.jv(x)
    tol = 1e-10
    outs = [(1, 0.5), (1, 1.0), (0, 1.0), (3, 1.0)]
    res, infos = kiops.kiops_phi(A, v, outs, tol)
    for (l, s), r in zip(outs, res):
        ex = exact.advdiff_phi_fft(n, prm["D"], prm["ax"], prm["ay"], s * h, v, l)
        assert np.linalg.norm(r - ex) <= 10 * tol * np.linalg.norm(v)


def test_kiops_phi_sum_vs_dense_augmented():
    rng = np.random.default_rng(8)
    n = 6
    op = GrayScott(n, 3e-3, 1e-3, 0.04, 0.06)
    u = np.concatenate([1 - 0.3 * rng.random(n * n), 0.3 * rng.random(n * n)])
    opu = with_state(op, u)
    Am = exact.dense_matrix(opu.jv, u.size)
    h = 3.0
    bs = [rng.standard_normal(u.size), None, rng.standard_normal(u.size), 0.1 * rng.standard_normal(u.size)]
    outs, info = kiops.kiops(lambda x: h * opu.jv(x), bs, [0.3, 1.0], 1e-11, m_init=8, m_max=24)
    for t, o in zip([0.3, 1.0], outs):
        ref = exact.augmented_phi_sum(t * h * Am, [b if b is None else b * t ** j for j, b in enumerate(bs)])
        assert np.linalg.norm(o - ref) <= 1e-9 * np.linalg.norm(ref)
    assert info["substeps"] >= 2


def test_kiops_substeps_small_m_max():
    n, prm, v, op = _advdiff_case(16)
    h = prm["h"]
    res, infos = kiops.kiops_phi(lambda x: h * op.jv(x), v, [(1, 1.0)], 1e-10, m_init=8, m_max=12)
    ex = exact.advdiff_phi_fft(n, prm["D"], prm["ax"], prm["ay"], h, v, 1)
    assert infos[0]["substeps"] > 1
    assert np.linalg.norm(res[0] - ex) <= 1e-9 * np.linalg.norm(v)


STEP_METHODS = [("exprb43", "leja"), ("exprb43", "kiops"), ("epirk4s3", "leja"), ("epirk4s3", "kiops"),
                ("epirk4s3", "lekry"), ("epirk4s3a", "leja"), ("epirk4s3a", "kiops"), ("epirk4s3a", "lekry"),
                ("exprb53s3", "leja"), ("exprb53s3", "kiops"), ("exprb53s3", "lekry"), ("epirk5p1", "leja"),
                ("epirk5p1", "kiops")]


@pytest.mark.parametrize("scheme,method", STEP_METHODS)
def test_integrator_linear_problem_is_exact(scheme, method):
    # linear f: R == 0 so both solutions are exp(hA) u
    n = 16
    op = AdvDiff(n, 0.5, 3.0, 2.0)
    u = synth.advdiff_gaussian(n)
    h = 20.0 / (4 * 0.5 * n * n)
    spec = (-8 * 0.5 * n * n, 0.0)
    u4, u3, st = integrators.STEPS[scheme](op, u, h, method=method, tol=1e-12,
                                           spec=spec if method != "kiops" else None)
    ex = exact.advdiff_phi_fft(n, 0.5, 3.0, 2.0, h, u, 0)
    assert np.linalg.norm(u4 - ex) <= 1e-10 * np.linalg.norm(ex)
    assert np.linalg.norm(u3 - ex) <= 1e-10 * np.linalg.norm(ex)


def test_methods_agree_on_a_nonlinear_step():
    """Leja, KIOPS and LeKry evaluate the same stages; each result is within
    ~tol of the exact stage values, so the three steps agree to a few tol."""
    n = 16
    rng = np.random.default_rng(5)
    op = GrayScott(n, 2e-3, 1e-3, 0.04, 0.06)
    u0 = np.concatenate([1 - 0.3 * rng.random(n * n), 0.3 * rng.random(n * n)])
    h = 20.0 * (1.0 / n) ** 2 / (4 * 2e-3)
    for scheme in ["epirk4s3", "epirk4s3a", "exprb53s3"]:
        res = {m: integrators.STEPS[scheme](op, u0, h, method=m, tol=1e-11)[0] for m in ["leja", "kiops", "lekry"]}
        d = res["leja"] - u0
        for m in ["kiops", "lekry"]:
            assert np.linalg.norm(res[m] - res["leja"]) <= 1e-8 * np.linalg.norm(d), (scheme, m)


@pytest.mark.slow
@pytest.mark.parametrize("scheme,orders", [("exprb43", (4, 3)), ("epirk4s3", (4, 3)), ("epirk4s3a", (4, 3)),
                                           ("exprb53s3", (5, 3)), ("epirk5p1", (5, 4))])
def test_integrator_order(scheme, orders):
    # global error at T after N and 2N steps: ratio ~ 2^p for an order-p solution
    step = integrators.STEPS[scheme]
    n = 8
    rng = np.random.default_rng(9)
    op = GrayScott(n, 1e-2, 5e-3, 0.04, 0.06)
    u0 = np.concatenate([1 - 0.2 * rng.random(n * n), 0.04 * rng.random(n * n)])
    T = 8.0

    def run(N, which=0):
        u = u0.copy()
        for _ in range(N):
            opu = with_state(op, u)
            A = exact.dense_matrix(opu.jv, u.size)
            lam = np.linalg.eigvals(A)
            spec = (1.1 * min(0.0, np.min(lam.real)) - 1e-3, 1.1 * max(0.0, np.max(lam.real)))
            u = step(op, u, T / N, tol=1e-14, spec=spec, leja_kw=dict(m_max=300))[which]
        return u

    ref = run(256)
    for which, p in enumerate(orders):
        e1 = np.linalg.norm(run(16, which) - ref)
        e2 = np.linalg.norm(run(32, which) - ref)
        print(scheme, which, "ratio", e1 / e2, "expected ~", 2 ** p)
        assert 0.75 * 2 ** p < e1 / e2 < 1.5 * 2 ** p or (which == 1 and e1 / e2 > 0.75 * 2 ** p)
