"""The two-iteration Newton kernel (two Leja iterations per launch, the
second iteration's accumulator term deferred to the next launch or to the
output conversion) against one iteration per launch and against the oracle.

Both kernels apply the same stencil and fused multiply-add to the same
operands in the same order, so for the same stop iteration the outputs
agree bit for bit; the stop iteration falls on either member of a pair,
which the tolerance sweep below covers.
"""
import numpy as np
import pytest

import synth
from gpu_util import rel, parity_tol
from oracle import leja
from oracle.operators import GrayScott, with_state

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


def _gs_state(nx, ny):
    """Both species on ny x nx: the seeded square state cut to ny rows."""
    s = synth.grayscott_state(nx, seed=6, patch=16).reshape(2, nx, nx)
    return np.ascontiguousarray(s[:, :ny, :]).reshape(-1)


def _problem(phix, kind, nx, ny):
    rng = np.random.default_rng(11)
    if kind == "advdiff":
        p = synth.advdiff_params(nx)
        op = phix.make_jop(phix.PHIX_OP_ADVDIFF, nx, ny, [p["D"], p["ax"], p["ay"]])
        v = dev(rng.standard_normal(nx * ny))
        return op, v, p["h"], dict(rho_re=4.0 * p["D"] * (nx * nx + ny * ny)), [0, 1, 2, 3], [1.0, 1.0, 0.5, 1.0]
    if kind == "grayscott":
        prm = synth.grayscott_params(nx, Du=2e-3, Dv=1e-3, mult=30.0)
        st = dev(_gs_state(nx, ny))
        op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, nx, ny, [prm["Du"], prm["Dv"], prm["F"], prm["k"]], st)
        return op, dev(rng.standard_normal(2 * nx * ny)), prm["h"], {}, [1, 1], [0.5, 1.0]
    prm = synth.burgers_params(nx, mult=10.0)
    u = synth.burgers_state(nx, seed=6).reshape(nx, nx)[:ny].reshape(-1)
    op = phix.make_jop(phix.PHIX_OP_BURGERS, nx, ny, [prm["nu"]], dev(u))
    kw = dict(rho_im=2.0 * max(nx, ny) * float(np.abs(u).max()))
    return op, dev(rng.standard_normal(nx * ny)), prm["h"], kw, [1], [1.0]


def _action(phix, ctx, op, v, h, ls, ss, tol, prec, kernel, **kw):
    out = [torch.empty_like(v) for _ in ls]
    o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), kernel=kernel,
                               chain=phix.PHIX_CHAIN_GRAPH, **kw)
    st = phix.phix_phi_action(ctx, op, h, v, ls, ss, out, tol, phix.PHIX_LEJA, o, check=False)
    return out, st


@pytest.mark.parametrize("shape", [(128, 64), (192, 48)])
@pytest.mark.parametrize("kind", ["advdiff", "grayscott", "burgers"])
@pytest.mark.parametrize("prec", ["FP64", "DF64", "FP32_JV", "FP32"])
def test_two_iterations_per_launch_equal_one(px, kind, prec, shape):
    phix, ctx = px
    nx, ny = shape
    op, v, h, kw, ls, ss = _problem(phix, kind, nx, ny)
    parities = set()
    sweep = kind == "grayscott" and prec == "DF64"
    tols = np.geomspace(1e-5, 1e-11, 13) if sweep else (1e-6, 3e-8, 1e-8, 3e-10, 1e-10)
    for tol in tols:
        a, sa = _action(phix, ctx, op, v, h, ls, ss, float(tol), prec, phix.PHIX_KERNEL_FUSED2, **kw)
        b, sb = _action(phix, ctx, op, v, h, ls, ss, float(tol), prec, phix.PHIX_KERNEL_SINGLE, **kw)
        assert sa.status == sb.status == 0
        assert sa.iters == sb.iters and sa.substeps == sb.substeps
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        # two iterations per launch: fewer launches for the same chain
        assert sa.launches <= sb.launches
        parities.add(sa.iters % 2)
    if sweep:
        assert parities == {0, 1}, "the sweep should stop on both members of a pair"


@pytest.mark.parametrize("m_max", [7, 8])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_two_iteration_chain_at_m_max(px, prec, m_max):
    """An unconverged chain ends at m_max, odd (the last launch has one
    iteration) or even (the last term is added by the output conversion)."""
    phix, ctx = px
    op, v, h, kw, ls, ss = _problem(phix, "grayscott", 128, 64)
    a, sa = _action(phix, ctx, op, v, h, ls, ss, 1e-30, prec, phix.PHIX_KERNEL_FUSED2, m_max=m_max, **kw)
    b, sb = _action(phix, ctx, op, v, h, ls, ss, 1e-30, prec, phix.PHIX_KERNEL_SINGLE, m_max=m_max, **kw)
    assert sa.status == sb.status == phix.PHIX_ENOTCONV
    assert sa.iters == sb.iters
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_two_iteration_kernel_vs_oracle(px, prec):
    """Gray-Scott 128 x 64, phi_1 at h/2 and h (vertical), the interval
    [-1.2 rho, 0] from the same SplitMix64 power iteration on both sides:
    element-wise against the oracle's Newton-Leja."""
    phix, ctx = px
    nx, ny = 128, 64
    prm = synth.grayscott_params(nx, Du=2e-3, Dv=1e-3, mult=30.0)
    st = _gs_state(nx, ny)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, nx, ny, [prm["Du"], prm["Dv"], prm["F"], prm["k"]], dev(st))
    v = np.random.default_rng(5).standard_normal(2 * nx * ny)
    tol = 1e-10
    out, sa = _action(phix, ctx, op, dev(v), prm["h"], [1, 1], [0.5, 1.0], tol, prec, phix.PHIX_KERNEL_FUSED2)
    assert sa.status == 0
    g = with_state(GrayScott(nx, prm["Du"], prm["Dv"], prm["F"], prm["k"], ny=ny), st)
    rho, mv = leja.power_iteration(g.jv, st.size)
    assert sa.power_mv == mv and abs(sa.rho - rho) <= 1e-12 * rho
    ref, info = leja.leja_phi(g.jv, v, prm["h"], -1.2 * rho, 0.0, [(1, 0.5), (1, 1.0)], tol)
    assert info["status"] == 0
    for o, r in zip(out, ref):
        assert rel(o.cpu().numpy(), r) <= parity_tol(sa.iters == info["iters"], tol)
