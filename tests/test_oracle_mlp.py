"""Pins for oracle.mlp: bf16 rounding, forward pass, gradient, Adam, features."""
import math

import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def _params(seed=0, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.NPARAM) * scale


def test_bf16_round_matches_torch():
    x = np.concatenate([np.random.default_rng(1).standard_normal(2000) * 10.0 ** np.random.default_rng(2).uniform(-5, 5, 2000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0]]).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_forward_matches_torch_module():
    p = _params()
    X = np.random.default_rng(3).standard_normal((50, 16))
    y, _ = mlp.forward(p, X)
    layers = mlp.unpack(p)
    net = torch.nn.Sequential(torch.nn.Linear(16, 64), torch.nn.GELU(), torch.nn.Linear(64, 64), torch.nn.GELU(),
                              torch.nn.Linear(64, 3)).double()
    with torch.no_grad():
        for lin, (W, b) in zip([net[0], net[2], net[4]], layers):
            lin.weight.copy_(torch.tensor(mlp.bf16_round(W)))
            lin.bias.copy_(torch.tensor(b))
        ref = net(torch.tensor(X)).numpy()
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_gradient_finite_differences():
    rng = np.random.default_rng(4)
    p = _params(5)
    X = rng.standard_normal((20, 16))
    T = rng.standard_normal((20, 3))
    # differentiate the model at the rounded weights, treated as continuous
    pq = p.copy()
    o = 0
    for (r, c) in mlp.SIZES:
        pq[o:o + r * c] = mlp.bf16_round(p[o:o + r * c])
        o += r * c + r
    loss, g = mlp.loss_and_grad(pq, X, T, round_weights=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = 1e-6
        lp, _ = mlp.loss_and_grad(pq + e, X, T, round_weights=False)
        lm, _ = mlp.loss_and_grad(pq - e, X, T, round_weights=False)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    _, g2 = mlp.loss_and_grad(p, X, T)
    assert np.allclose(g, g2)  # the rounded model's gradient is the same function


def test_adam_matches_torch():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(40)
    m = np.zeros(40)
    v = np.zeros(40)
    tp = torch.nn.Parameter(torch.tensor(p.copy()))
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.standard_normal(40)
        p, m, v = mlp.adam_step(p, m, v, g, step, 1e-2)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_features_closed_forms():
    nx, ny = 16, 8
    # constant Burgers state: no gradients, advection bound max|U| (nx+ny)/rho_diff
    u = np.full(nx * ny, 0.5)
    f = mlp.features(2, nx, ny, [0.01], 0.1, u)
    rho_diff = 4 * 0.01 * (nx * nx + ny * ny)
    assert f[8] == 0 and f[9] == 0 and f[10] == 0
    assert f[12] == pytest.approx(0.5 * (nx + ny) / rho_diff)
    assert f[1] == pytest.approx(math.log(nx * ny) / 10) and f[15] == 1 and f[0] == 0
    # Gray-Scott uniform state: reaction extrema
    s = np.concatenate([np.full(nx * ny, 0.8), np.full(nx * ny, 0.25)])
    f = mlp.features(1, nx, ny, [2e-3, 1e-3, 0.04, 0.06], 1.0, s)
    assert f[10] == pytest.approx(0.0625) and f[11] == pytest.approx(0.4) and f[0] == 1
    assert f[13] == 0.04 and f[14] == 0.06
    # sin(2 pi x) along x: max centred difference 2 sin(2 pi/nx)
    X = np.tile(np.arange(nx) / nx, ny)
    f = mlp.features(2, nx, ny, [0.01], 0.1, np.sin(2 * np.pi * X))
    assert f[8] == pytest.approx(0.5 * 2 * math.sin(2 * math.pi / nx), rel=1e-12)


def test_labels_substeps():
    nx = ny = 32
    u = np.zeros(nx * ny)
    t = mlp.labels(2, nx, ny, [0.01], 0.5, u, rho_power=4 * 0.01 * 2 * nx * nx)
    assert t[0] == pytest.approx(0.0) and t[1] == 0.0 and t[2] == 0.0  # s = 1
    u[:] = 2.0
    t = mlp.labels(2, nx, ny, [0.01], 0.5, u, rho_power=80.0)
    # rho_im = 2 * 64 = 128, h rho_im / 4 = 16 substeps
    assert t[2] == pytest.approx(math.log(16))
