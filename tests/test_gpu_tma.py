"""The TMA-staged Newton-Leja kernel (forced with opts.kernel) against the
single-step kernel and the CPU oracle: every operator and precision,
K = 1, 2, 4 accumulators, and tile geometries that exercise the periodic
halo patches (one tile, a partial last tile in x and in y, grids narrower
than a tile, a 6 x 3 grid) and the fallback for rows that are not 16-byte
multiples."""
import numpy as np
import pytest

from gpu_util import rel, parity_tol
from oracle import leja
from oracle.operators import AdvDiff, GrayScott, Burgers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    from paper_2211_08948_gb300 import build, phix
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ctx = phix.phix_create(torch.cuda.current_stream())
    yield phix, ctx
    phix.phix_destroy(ctx)


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _problem(kind, nx, ny, seed):
    rng = np.random.default_rng(seed)
    if kind == "advdiff":
        D = 1.0
        ax, ay = 0.3 * min(nx, ny), -0.2 * min(nx, ny)
        return AdvDiff(nx, D, ax, ay, ny=ny), [D, ax, ay], None, 4.0 * D * (nx * nx + ny * ny)
    if kind == "grayscott":
        prm = [0.8e-3, 0.4e-3, 0.04, 0.06]
        # v small: the reaction block stays dissipative (2uv < F + k), so the
        # real interval [-rho, 0] holds the spectrum even where diffusion is weak
        u = np.concatenate([1 - 0.4 * rng.random(nx * ny), 0.05 * rng.random(nx * ny)])
        rho = 4.0 * prm[0] * (nx * nx + ny * ny) + 2.0
        return GrayScott(nx, *prm, state=u, ny=ny), prm, u, rho
    nu = 2e-2
    u = 0.5 * rng.standard_normal(nx * ny)
    rho = 4.0 * nu * (nx * nx + ny * ny) + 4.0 * np.max(np.abs(u)) * (nx + ny)
    return Burgers(nx, nu, state=u, ny=ny), [nu], u, rho


KINDS = {"advdiff": 0, "grayscott": 1, "burgers": 2}
OUTS = {1: [(1, 1.0)], 2: [(1, 0.5), (2, 1.0)], 4: [(0, 1.0), (1, 1.0), (2, 1.0), (3, 0.5)]}


def _run(phix, ctx, kind, nx, ny, prm, state, v, h, outs, tol, prec, kernel, rho):
    op = phix.make_jop(KINDS[kind], nx, ny, prm, dev(state) if state is not None else None)
    o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), kernel=kernel, rho_re=rho)
    vd = dev(v)
    od = [torch.empty_like(vd) for _ in outs]
    st = phix.phix_phi_action(ctx, op, h, vd, [l for l, _ in outs], [s for _, s in outs], od, tol,
                              phix.PHIX_LEJA, o)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in od], st


@pytest.mark.parametrize("kind", ["advdiff", "grayscott", "burgers"])
@pytest.mark.parametrize("nx,ny,K", [(128, 4, 1), (256, 6, 2), (130, 7, 4), (4, 4, 2), (6, 3, 1), (300, 17, 2)])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_tma_kernel_matches_single_step_and_oracle(px, kind, nx, ny, K, prec):
    phix, ctx = px
    op, prm, state, rho = _problem(kind, nx, ny, nx * 31 + ny)
    nc = 2 if kind == "grayscott" else 1
    v = np.random.default_rng(7).standard_normal(nc * nx * ny)
    h = 12.0 / rho
    outs = OUTS[K]
    tol = 1e-10
    r_t, s_t = _run(phix, ctx, kind, nx, ny, prm, state, v, h, outs, tol, prec, phix.PHIX_KERNEL_TMA, rho)
    r_s, s_s = _run(phix, ctx, kind, nx, ny, prm, state, v, h, outs, tol, prec, phix.PHIX_KERNEL_SINGLE, rho)
    assert s_t.status == 0 and s_s.status == 0
    assert s_t.tma_passes == 1 and s_s.tma_passes == 0
    ref, info = leja.leja_phi(op.jv, v, h, -rho, 0.0, outs, tol)
    for a, b, o in zip(r_t, r_s, ref):
        assert rel(a, b) <= parity_tol(s_t.iters == s_s.iters, tol)
        assert rel(a, o) <= parity_tol(s_t.iters == info["iters"], tol)


@pytest.mark.parametrize("kind", ["advdiff", "grayscott", "burgers"])
@pytest.mark.parametrize("prec", ["FP32_JV", "FP32"])
@pytest.mark.parametrize("nx,ny,tma", [(256, 8, 1), (130, 8, 0)])
def test_tma_kernel_reduced_precision_and_fallback(px, kind, prec, nx, ny, tma):
    """4-byte state needs nx % 4 == 0 for 16-byte rows: 130 falls back."""
    phix, ctx = px
    op, prm, state, rho = _problem(kind, nx, ny, 3)
    nc = 2 if kind == "grayscott" else 1
    v = np.random.default_rng(8).standard_normal(nc * nx * ny)
    h = 12.0 / rho
    outs = OUTS[2]
    r_t, s_t = _run(phix, ctx, kind, nx, ny, prm, state, v, h, outs, 1e-6, prec, phix.PHIX_KERNEL_TMA, rho)
    r_s, s_s = _run(phix, ctx, kind, nx, ny, prm, state, v, h, outs, 1e-6, prec, phix.PHIX_KERNEL_SINGLE, rho)
    assert s_t.status == 0 and s_s.status == 0
    assert s_t.tma_passes == tma
    ref, _ = leja.leja_phi(op.jv, v, h, -rho, 0.0, outs, 1e-10)
    for a, b, o in zip(r_t, r_s, ref):
        assert rel(a, b) <= 1e-5
        assert rel(a, o) <= 1e-4
