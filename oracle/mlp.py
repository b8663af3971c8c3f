"""Learned spectral interval: state features and the MLP 16 -> 64 -> 64 -> 3.

Not in the paper: the paper estimates the spectrum by power iterations
(Sec. 2.2) every few steps; here a small network predicts that estimate
(and the imaginary extent and substep count derived from it) from cheap state
features, with power iteration as fallback.  This module is the oracle of
the GPU implementation: float64 NumPy, weights rounded to bfloat16 exactly as
the GPU stores them (round to nearest even), everything else float64.

Parameter layout (float32 master copy, 5443 values):
  W1 [64 x 16], b1 [64], W2 [64 x 64], b2 [64], W3 [3 x 64], b3 [3].
Activation: GELU(x) = x/2 (1 + erf(x / sqrt 2)).
Loss per sample: sum_j w_j(yhat_j - t_j)^2 with w_0 = 4 when yhat_0 < t_0
(under-estimating the spectral radius is the dangerous side), else 1; the
batch loss is the mean over samples.
Adam (Kingma & Ba 2015): beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.
"""
import math

import numpy as np
from scipy.special import erf

SIZES = [(64, 16), (64, 64), (3, 64)]
NPARAM = 64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3  # 5443
NFEAT = 16


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out = []
    o = 0
    for (r, c) in SIZES:
        W = p[o:o + r * c].reshape(r, c)
        o += r * c
        b = p[o:o + r]
        o += r
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(params, X, round_weights=True):
    """X [n x 16] -> (Y [n x 3], cache).  Weights (not biases) rounded to bf16."""
    layers = unpack(params)
    Wq = [bf16_round(W) if round_weights else W for (W, _) in layers]
    bs = [b for (_, b) in layers]
    z1 = X @ Wq[0].T + bs[0]
    a1 = gelu(z1)
    z2 = a1 @ Wq[1].T + bs[1]
    a2 = gelu(z2)
    y = a2 @ Wq[2].T + bs[2]
    return y, (X, z1, a1, z2, a2, Wq)


def loss_and_grad(params, X, T, round_weights=True):
    """Mean loss over the batch and its gradient w.r.t. all parameters (the
    gradient of the bf16-weight model, applied to the master weights)."""
    y, (X, z1, a1, z2, a2, Wq) = forward(params, X, round_weights)
    n = X.shape[0]
    w = np.ones_like(y)
    w[:, 0] = np.where(y[:, 0] < T[:, 0], 4.0, 1.0)
    diff = y - T
    loss = np.sum(w * diff * diff) / n
    dy = 2.0 * w * diff / n
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    da2 = dy @ Wq[2]
    dz2 = da2 * gelu_grad(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    da1 = dz2 @ Wq[1]
    dz1 = da1 * gelu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(params, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------------------
# State features and labels
# --------------------------------------------------------------------------------------
def features(kind, nx, ny, params, h, state):
    """16 features of (operator, state, step); kind 1 = Gray-Scott, 2 = Burgers.
    0 kind==GS, 1 log(nx ny)/10, 2 log(Dmax)/10, 3 log(h)/10, 4 log(h rho_diff)/5,
    5 max|s1|, 6 max|s2|, 7 mean|s1|, 8 max g, 9 mean g  (g = (|dE-W| + |dN-S|)/2 of s1),
    10 GS: max V^2 | Burgers: max|U_x+U_y| / rho_diff, 11 GS: max(0, max 2UV) | Burgers: 0,
    12 Burgers: max|U|(nx+ny)/rho_diff | GS: 0, 13 F, 14 k, 15 1.
    rho_diff = 8 Dmax (nx^2 + ny^2)/2 = 4 Dmax (nx^2 + ny^2).
    These features are this project's own choice (the paper defines no
    learned interval).  Feature 11 is the largest positive value of the
    reaction coefficient 2UV, the term of the Gray-Scott Jacobian that can
    push eigenvalues to the right; it is clamped at 0 (a non-positive 2UV
    cannot widen the interval), and 0 is also the identity element both
    implementations start that maximum from.  On the Gray-Scott states of
    the workloads (U, V >= 0) the clamp is never active."""
    f = np.zeros(NFEAT)
    N = nx * ny
    s1 = state[:N].reshape(ny, nx)
    s2 = state[N:2 * N].reshape(ny, nx) if kind == 1 else np.zeros_like(s1)
    Dmax = max(params[0], params[1]) if kind == 1 else params[0]
    rho_diff = 4.0 * Dmax * (nx * nx + ny * ny)
    dx = np.roll(s1, -1, 1) - np.roll(s1, 1, 1)
    dy = np.roll(s1, -1, 0) - np.roll(s1, 1, 0)
    g = 0.5 * (np.abs(dx) + np.abs(dy))
    f[0] = 1.0 if kind == 1 else 0.0
    f[1] = math.log(N) / 10.0
    f[2] = math.log(Dmax) / 10.0
    f[3] = math.log(h) / 10.0
    f[4] = math.log(h * rho_diff) / 5.0
    f[5] = np.max(np.abs(s1))
    f[6] = np.max(np.abs(s2))
    f[7] = np.mean(np.abs(s1))
    f[8] = np.max(g)
    f[9] = np.mean(g)
    if kind == 1:
        f[10] = np.max(s2 * s2)
        f[11] = max(0.0, np.max(2.0 * s1 * s2))
        f[13] = params[2]
        f[14] = params[3]
    else:
        div = 0.5 * (dx * nx + dy * ny)
        f[10] = np.max(np.abs(div)) / rho_diff
        f[12] = np.max(np.abs(s1)) * (nx + ny) / rho_diff
    f[15] = 1.0
    return f


def labels(kind, nx, ny, params, h, state, rho_power, safety=1.2, gamma_cap=200.0, iota_cap=4.0):
    """Targets of the network, the quantities the method would use:
    t0 = log(rho / rho_diff) with rho the power-iteration estimate,
    t1 = log(1 + rho_im / rho_diff) with rho_im the Bendixson bound of the
         skew part (Burgers: max|U| (nx + ny); Gray-Scott: 0),
    t2 = log(s), s the substep count of the Leja phi_1 action at that interval."""
    N = nx * ny
    Dmax = max(params[0], params[1]) if kind == 1 else params[0]
    rho_diff = 4.0 * Dmax * (nx * nx + ny * ny)
    rho_im = 0.0 if kind == 1 else float(np.max(np.abs(state[:N]))) * (nx + ny)
    gamma = max(0.25 * safety * rho_power, 2.0 * rho_im)
    s = 1
    s = max(s, int(math.ceil(h * gamma / gamma_cap - 1e-12)))
    if rho_im > 0:
        s = max(s, int(math.ceil(h * rho_im / iota_cap - 1e-12)))
    return np.array([math.log(rho_power / rho_diff), math.log1p(rho_im / rho_diff), math.log(s)])
