"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the method: it only draws the initial
states, input vectors and problem parameters of the workloads (all from
``numpy.random.default_rng(seed)``), and lays out grid coordinates.
Workload recipes:

* advection-diffusion 64x64 (2D periodic, D=1, a=(10,10)),
  v = exp(-((x-0.6)^2+(y-0.6)^2)/0.01), h = 50 * dx^2/(4D)
* Gray-Scott 1024x1024 two species (D_u=2e-5, D_v=1e-5, F=0.04, k=0.06),
  u=1, v=0 plus U(0,0.1) on the central 64x64 cells of both species,
  h = 100 * dx^2/(4 max D)
* Burgers 2048x2048, nu=1e-3, u0 = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1)
  smoothed by 3 Jacobi sweeps, h = 50 * dx^2/(4 nu)
* batched advection-diffusion problems: side round(exp(U(ln 32, ln 512))),
  D ~ U(0.1,1), a ~ U(0,50)^2, h = U_log(10,200) * dx^2/(4D), v ~ N(0,1)
* learned spectral interval: Gray-Scott and Burgers states alternately, side
  log-uniform (even), diffusion log-uniform, h = U_log(10,100) x the
  explicit step, Gray-Scott u=1, v=0 plus U(0, amp) on a random central
  patch, Burgers amp (sin sin + 0.1 N(0,1)) smoothed by 3 Jacobi sweeps; at
  the full scale (sides 128..1024, 200k states) drawn on the GPU by torch's
  seeded generator (`learned_state_torch`), the same recipe

Vectors are float64, C-contiguous, planar: species-major, then row (y),
then column (x); grid nodes x_j = j/n on the periodic unit square.
"""
import numpy as np


def grid_xy(n):
    """Node coordinates (X, Y) of shape (n, n), X varying along axis 1."""
    x = np.arange(n, dtype=np.float64) / n
    return np.meshgrid(x, x, indexing="xy")


def advdiff_gaussian(n=64):
    X, Y = grid_xy(n)
    return np.exp(-((X - 0.6) ** 2 + (Y - 0.6) ** 2) / 0.01).reshape(-1)


def advdiff_params(n=64, D=1.0, ax=10.0, ay=10.0, mult=50.0):
    dx = 1.0 / n
    h = mult * dx * dx / (4.0 * D)
    return dict(D=D, ax=ax, ay=ay, h=h)


def grayscott_state(n=1024, seed=0, patch=64, amp=0.1):
    """Two planes (u then v) of length n*n each: u=1, v=0 plus a seeded
    uniform(0, amp) perturbation on the central patch x patch cells of both
    species (u drawn first, then v)."""
    rng = np.random.default_rng(seed)
    u = np.ones((n, n))
    v = np.zeros((n, n))
    lo = n // 2 - patch // 2
    hi = lo + patch
    if patch > 0:
        u[lo:hi, lo:hi] += rng.uniform(0.0, amp, size=(patch, patch))
        v[lo:hi, lo:hi] += rng.uniform(0.0, amp, size=(patch, patch))
    return np.concatenate([u.reshape(-1), v.reshape(-1)])


def grayscott_gaussian(n=64):
    """The paper's smooth Gray-Scott initial state (Sec. 3): u = 1 - exp(-150 r_u),
    v = exp(-150 r_v), r_u = (x-1/2)^2 + (y-1/2)^2, r_v = (x-1/2)^2 + 2 (y-1/2)^2."""
    X, Y = grid_xy(n)
    u = 1.0 - np.exp(-150.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
    v = np.exp(-150.0 * ((X - 0.5) ** 2 + 2.0 * (Y - 0.5) ** 2))
    return np.concatenate([u.reshape(-1), v.reshape(-1)])


def cell_xy(n, x0=0.0, L=1.0):
    """Cell-centre coordinates (X, Y), shape (n, n), of [x0, x0 + L]^2 (X along axis 1)."""
    x = x0 + (np.arange(n, dtype=np.float64) + 0.5) * (L / n)
    return np.meshgrid(x, x, indexing="xy")


def adr_state(n=64):
    """The paper's ADR initial state (Sec. 3): 256 (x y (1 - x)(1 - y))^2 + 0.3 on [0, 1]^2."""
    X, Y = cell_xy(n)
    return (256.0 * (X * Y * (1 - X) * (1 - Y)) ** 2 + 0.3).reshape(-1)


def allen_cahn_state(n=64):
    """The paper's Allen-Cahn initial state (Sec. 3): 0.1 + 0.1 cos(2 pi x) cos(2 pi y) on [-1, 1]^2."""
    X, Y = cell_xy(n, -1.0, 2.0)
    return (0.1 + 0.1 * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)).reshape(-1)


def brusselator_state(n=64):
    """The paper's Brusselator initial state (Sec. 3): u = 2 + 0.25 y, v = 1 + 0.8 x on [0, 1]^2."""
    X, Y = cell_xy(n)
    return np.concatenate([(2.0 + 0.25 * Y).reshape(-1), (1.0 + 0.8 * X).reshape(-1)])


def grayscott_params(n=1024, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, mult=100.0):
    dx = 1.0 / n
    h = mult * dx * dx / (4.0 * max(Du, Dv))
    return dict(Du=Du, Dv=Dv, F=F, k=k, h=h)


def burgers_state(n=2048, seed=0, sweeps=3):
    """u0 = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1), then `sweeps` periodic
    Jacobi sweeps u <- (u_E + u_W + u_N + u_S)/4 (a smoothing recipe, not
    part of the method)."""
    rng = np.random.default_rng(seed)
    X, Y = grid_xy(n)
    u = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + 0.1 * rng.standard_normal((n, n))
    for _ in range(sweeps):
        u = 0.25 * (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1))
    return u.reshape(-1)


def burgers_params(n=2048, nu=1e-3, mult=50.0):
    dx = 1.0 / n
    return dict(nu=nu, h=mult * dx * dx / (4.0 * nu))


def random_vector(n, seed=0):
    return np.random.default_rng(seed).standard_normal(n)


def batched_problems(count=4096, seed=0, side_lo=32, side_hi=512, h_lo=10.0, h_hi=200.0):
    """List of dicts (n, D, ax, ay, h, seed_v) for independent periodic
    advection-diffusion problems; each v is random_vector(n*n, seed_v)."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi), size=count))).astype(int)
    D = rng.uniform(0.1, 1.0, size=count)
    a = rng.uniform(0.0, 50.0, size=(count, 2))
    mult = np.exp(rng.uniform(np.log(h_lo), np.log(h_hi), size=count))
    probs = []
    for i in range(count):
        n = int(sides[i])
        dx = 1.0 / n
        probs.append(dict(n=n, D=float(D[i]), ax=float(a[i, 0]), ay=float(a[i, 1]),
                          h=float(mult[i] * dx * dx / (4.0 * D[i])), seed_v=seed * 100003 + i))
    return probs


def learned_state_specs(count, seed=0, n_lo=32, n_hi=128):
    """Specs of Gray-Scott and Burgers states for the learned spectral interval:
    alternating kinds, sides log-uniform in [n_lo, n_hi] (even), diffusion
    coefficients log-uniform, h = 10..100x the explicit step, random
    perturbation amplitude and seed."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))) / 2) * 2)
        mult = float(np.exp(rng.uniform(np.log(10), np.log(100))))
        if i % 2 == 0:
            Du = float(np.exp(rng.uniform(np.log(5e-4), np.log(5e-2))))
            prm = [Du, 0.5 * Du, 0.04, 0.06]
            h = mult / (4.0 * Du * n * n)
            specs.append(dict(kind=1, n=n, params=prm, h=h, amp=float(rng.uniform(0.05, 0.5)),
                              patch=int(rng.integers(2, max(3, n // 2))), seed=int(rng.integers(1 << 30))))
        else:
            nu = float(np.exp(rng.uniform(np.log(1e-3), np.log(5e-2))))
            h = mult / (4.0 * nu * n * n)
            specs.append(dict(kind=2, n=n, params=[nu, 0.0, 0.0, 0.0], h=h, amp=float(rng.uniform(0.2, 2.0)),
                              patch=0, seed=int(rng.integers(1 << 30))))
    return specs


def learned_state(spec):
    """The state vector of a learned_state_specs entry (float64)."""
    if spec["kind"] == 1:
        return grayscott_state(spec["n"], seed=spec["seed"], patch=spec["patch"], amp=spec["amp"])
    return spec["amp"] * burgers_state(spec["n"], seed=spec["seed"])


def learned_state_torch(spec, torch, device="cuda"):
    """The learned_state recipe drawn on the device with torch's generator
    seeded by spec["seed"] (other values than learned_state's numpy draws,
    the same distribution): float64, planar."""
    n = spec["n"]
    g = torch.Generator(device=device).manual_seed(spec["seed"])
    if spec["kind"] == 1:
        u = torch.ones((n, n), dtype=torch.float64, device=device)
        v = torch.zeros((n, n), dtype=torch.float64, device=device)
        pa = spec["patch"]
        lo = n // 2 - pa // 2
        if pa > 0:
            u[lo:lo + pa, lo:lo + pa] += spec["amp"] * torch.rand((pa, pa), dtype=torch.float64, device=device,
                                                                  generator=g)
            v[lo:lo + pa, lo:lo + pa] += spec["amp"] * torch.rand((pa, pa), dtype=torch.float64, device=device,
                                                                  generator=g)
        return torch.cat([u.reshape(-1), v.reshape(-1)])
    x = torch.arange(n, dtype=torch.float64, device=device) / n
    Y, X = torch.meshgrid(x, x, indexing="ij")
    u = torch.sin(2 * np.pi * X) * torch.sin(2 * np.pi * Y) + 0.1 * torch.randn((n, n), dtype=torch.float64,
                                                                             device=device, generator=g)
    for _ in range(3):
        u = 0.25 * (torch.roll(u, 1, 0) + torch.roll(u, -1, 0) + torch.roll(u, 1, 1) + torch.roll(u, -1, 1))
    return (spec["amp"] * u).reshape(-1).contiguous()
