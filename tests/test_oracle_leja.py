"""Pins for oracle.leja: Leja points, divided differences, SplitMix64, power
iteration and the Newton interpolation of Sec. 2.2."""
import math

import numpy as np
import pytest

from oracle import leja
from oracle.phi import phi_scalar

mp = pytest.importorskip("mpmath")
from mp_ref import phi_mp  # noqa: E402


def test_leja_first_points_closed_form():
    x = leja.leja_points(5)
    assert x[0] == 2.0 and x[1] == -2.0 and x[2] == 0.0
    # argmax |x(x^2-4)| on [-2,2] is +-2/sqrt(3); the tie goes to the smaller x
    assert x[3] == pytest.approx(-2.0 / math.sqrt(3.0), abs=1e-15)


def test_leja_points_max_product_brute_force():
    x = leja.leja_points(60)
    g = np.linspace(-2.0, 2.0, 4_000_001)
    lp = np.zeros_like(g)
    for j in range(1, 60):
        lp += np.log(np.abs(g - x[j - 1]) + 1e-300)
        Lx = np.sum(np.log(np.abs(x[j] - x[:j])))
        # no grid point beats the chosen point (up to grid resolution effects)
        assert np.max(lp) <= Lx + 1e-9
        assert np.all(np.abs(x[j] - x[:j]) > 0)
    assert np.all(np.abs(x) <= 2.0)


def test_leja_points_distinct_and_prefix_stable():
    a = leja.leja_points(120)
    b = leja.leja_points(60)
    assert np.array_equal(a[:60], b)
    assert len(np.unique(a)) == 120


def test_divided_differences_against_mpmath():
    mp.mp.dps = 60
    x = leja.leja_points(40)
    for hg, l in [(3.0, 0), (20.0, 1), (60.0, 3)]:
        c = -2.0 * hg
        f = [phi_scalar(l, c + hg * xx) for xx in x]
        d = leja.divided_differences(x, f)
        # 60-digit recursion on the same nodes, fed with 60-digit function values
        fm = [phi_mp(l, mp.mpf(c) + mp.mpf(hg) * mp.mpf(xx)) for xx in x]
        dm = list(fm)
        X = [mp.mpf(v) for v in x]
        for j in range(1, len(x)):
            for i in range(len(x) - 1, j - 1, -1):
                dm[i] = (dm[i] - dm[i - 1]) / (X[i] - X[i - j])
        # error weighted by the Newton basis magnitude w_m = max_[-2,2] prod|t - x_i|
        t = np.linspace(-2, 2, 4001)
        w = np.ones_like(t)
        for m in range(len(x)):
            err = abs(d[m] - float(dm[m])) * np.max(np.abs(w))
            assert err <= 1e-13, (hg, l, m, err)
            w = w * (t - x[m])


def test_divided_differences_polynomial():
    x = leja.leja_points(8)
    f = 3.0 * x ** 3 - 2.0 * x + 5.0
    d = leja.divided_differences(x, f)
    assert d[3] == pytest.approx(3.0, rel=1e-13)
    assert np.all(np.abs(d[4:]) < 1e-12)
    # Newton form reproduces f at an arbitrary point
    t = 0.37
    val, w = 0.0, 1.0
    for m in range(8):
        val += d[m] * w
        w *= t - x[m]
    assert val == pytest.approx(3 * t ** 3 - 2 * t + 5, rel=1e-13)


def test_splitmix64_published_vectors():
    # SplitMix64 with seed 0: the reference sequence of Steele, Lea & Flood's generator
    z = leja.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = leja.splitmix64_uniform(0, 1000)
    assert np.all((u >= -0.5) & (u < 0.5))
    assert abs(np.mean(u)) < 0.05


def test_power_iteration_diffusion_bound():
    from oracle.operators import AdvDiff
    n = 32
    op = AdvDiff(n, 0.7, 0.0, 0.0)
    rho_exact = 8 * 0.7 * n * n  # symmetric, even n: |lambda|max = 8D/dx^2
    rho, mv = leja.power_iteration(op.jv, n * n, max_it=200, rel=1e-6)
    assert rho <= rho_exact * (1 + 1e-12)
    assert rho >= 0.97 * rho_exact
    rho2, mv2 = leja.power_iteration(op.jv, n * n)
    assert 0.5 * rho_exact < rho2 <= rho_exact * (1 + 1e-12) and mv2 <= 50


def test_newton_leja_diagonal_matrix():
    # J = diag(lam) with lam in [alpha, 0]: phi_l(s h J) v is phi_l(s h lam_i) v_i
    rng = np.random.default_rng(3)
    lam = -rng.uniform(0, 100.0, 200)
    lam[0], lam[1] = 0.0, -100.0
    v = rng.standard_normal(200)
    h = 0.9
    outs = [(0, 1.0), (1, 0.5), (2, 1.0), (4, 1.0)]
    res, info = leja.leja_phi(lambda w: lam * w, v, h, -100.0, 0.0, outs, 1e-12, m_max=300)
    assert info["status"] == 0
    for (l, s), r in zip(outs, res):
        ref = np.array([phi_scalar(l, s * h * li) for li in lam]) * v
        assert np.linalg.norm(r - ref) <= 1e-11 * np.linalg.norm(ref)


def test_leja_substeps_match_single_pass():
    rng = np.random.default_rng(5)
    lam = -rng.uniform(0, 80.0, 100)
    v = rng.standard_normal(100)
    for l in [0, 1, 3]:
        ref = np.array([phi_scalar(l, li) for li in lam]) * v
        res, info = leja.leja_phi(lambda w: lam * w, v, 1.0, -80.0, 0.0, [(l, 1.0)], 1e-12,
                                  m_max=300, gamma_cap=5.0)
        assert info["substeps"] == 4
        assert np.linalg.norm(res[0] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_leja_nonconvergence_reported():
    lam = -np.linspace(0, 100, 50)
    v = np.ones(50)
    res, info = leja.leja_phi(lambda w: lam * w, v, 1.0, -100.0, 0.0, [(1, 1.0)], 1e-12, m_max=10)
    assert info["status"] == leja.ENOTCONV
