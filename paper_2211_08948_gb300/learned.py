"""Training data and training loop of the learned spectral interval, through
the C-ABI (features, power iteration and training all run in libphix).

Targets per state (what the method itself would use): t0 = log(rho/rho_diff)
with rho the power-iteration estimate of |lambda(J)|max, t1 =
log(1 + rho_im/rho_diff) with rho_im the Bendixson bound of the skew part
(Burgers: max|u| (nx + ny); Gray-Scott: 0), t2 = log(substeps of a phi_1 Leja
action at that interval); rho_diff = 4 Dmax (nx^2 + ny^2).
"""
import math

import numpy as np

from . import phix

NPARAM = phix.PHIX_MLP_NPARAM


def rho_diff_of(kind, nx, ny, params):
    dmax = max(params[0], params[1]) if kind == phix.PHIX_OP_GRAYSCOTT else params[0]
    return 4.0 * dmax * (nx * nx + ny * ny)


def targets(kind, nx, ny, params, h, state_max_abs, rho, safety=1.2, gamma_cap=200.0, iota_cap=4.0):
    rd = rho_diff_of(kind, nx, ny, params)
    rho_im = 0.0 if kind == phix.PHIX_OP_GRAYSCOTT else state_max_abs * (nx + ny)
    gamma = max(0.25 * safety * rho, 2.0 * rho_im)
    s = max(1, int(math.ceil(h * gamma / gamma_cap - 1e-12)))
    if rho_im > 0:
        s = max(s, int(math.ceil(h * rho_im / iota_cap - 1e-12)))
    return [math.log(rho / rd), math.log1p(rho_im / rd), math.log(s)]


def initial_params(seed=0):
    """Weights ~ N(0, 1/fan_in) from numpy's seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM, dtype=np.float32)
    o = 0
    for r, c in [(64, 16), (64, 64), (3, 64)]:
        p[o:o + r * c] = rng.standard_normal(r * c) / math.sqrt(c)
        o += r * c + r
    return p


def make_dataset(ctx, problems, torch):
    """problems: list of (op, h, state_tensor).  Returns (X float32 [n,16], T float32 [n,3],
    power-iteration matvecs spent)."""
    X, T, mv = [], [], 0
    feats = torch.empty(16, dtype=torch.float32, device="cuda")
    for op, h, st in problems:
        phix.phix_features(ctx, op, h, feats)
        rho, s = phix.phix_spectrum(ctx, op, phix.phix_opts_default())
        mv += s.power_mv
        X.append(feats.cpu().numpy().copy())
        T.append(targets(op.kind, op.nx, op.ny, list(op.param)[:4], h,
                         float(torch.max(torch.abs(st[:op.nx * op.ny]))), rho))
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32), mv


def train(ctx, X, T, torch, seed=0, batch=256, schedule=((3e-3, 2000), (1e-3, 2000), (3e-4, 1000))):
    """Adam on the GPU; returns (params tensor, last loss)."""
    n = (len(X) // batch) * batch
    params = torch.tensor(initial_params(seed), device="cuda")
    m = torch.zeros(NPARAM, device="cuda")
    v = torch.zeros(NPARAM, device="cuda")
    Xd = torch.tensor(X[:n], device="cuda")
    Td = torch.tensor(T[:n], device="cuda")
    step, loss = 0, float("nan")
    for lr, nsteps in schedule:
        step, loss = phix.phix_mlp_train(ctx, params, m, v, step, Xd, Td, batch, nsteps, lr)
    return params, loss
