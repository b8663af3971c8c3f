"""GPU parity of the EXPRB43 / EPIRK4s3 steps (C-ABI) against the oracle,
on a small Gray-Scott grid and on the full 1024 x 1024 workload."""
import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import integrators
from oracle.operators import GrayScott, AdvDiff
from oracle import exact

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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("scheme", ["exprb43", "epirk4s3"])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_step_grayscott_small(px, scheme, prec):
    phix, ctx = px
    n = 64
    prm = synth.grayscott_params(n)
    prm["Du"] *= 64
    prm["Dv"] *= 64
    u0 = synth.grayscott_state(n, seed=2, patch=16)
    h = 20.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
    tol = 1e-10
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    fn = phix.phix_exprb43_step if scheme == "exprb43" else phix.phix_epirk4s3_step
    st = fn(ctx, op, ud, h, tol, phix.PHIX_LEJA, phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec)))
    ostep = integrators.exprb43_step if scheme == "exprb43" else integrators.epirk4s3_step
    u4, u3, ost = ostep(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0, h, tol=tol)
    got = host(ud)
    # the step increment (u4 - u0) is what the phi-actions produce
    assert rel(got - u0, u4 - u0) <= 1e-9
    assert st.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-6)
    assert st.power_mv == ost["power_mv"]


@pytest.mark.parametrize("scheme", ["exprb43", "epirk4s3"])
def test_step_linear_problem_is_exact(px, scheme):
    phix, ctx = px
    n = 32
    D, ax, ay = 0.5, 3.0, 2.0
    u0 = synth.advdiff_gaussian(n)
    h = 20.0 / (4 * D * n * n)
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay])
    fn = phix.phix_exprb43_step if scheme == "exprb43" else phix.phix_epirk4s3_step
    fn(ctx, op, ud, h, 1e-12, phix.PHIX_LEJA, phix.phix_opts_default(rho_re=8 * D * n * n))
    ex = exact.advdiff_phi_fft(n, D, ax, ay, h, u0, 0)
    assert rel(host(ud), ex) <= 1e-10


@pytest.mark.slow
def test_step_grayscott_1024_full_size(px):
    """The benchmark workload, as the bench times it: Gray-Scott 1024^2 x 2
    species, h = 100x the explicit limit, tol 1e-8, double-float iteration,
    20 EXPRB43 steps from the seeded state, against the oracle's own 20-step
    trajectory (each side estimates its interval by the same SplitMix64 power
    iteration every step).  Every step must take the oracle's power-iteration
    and Newton iteration counts, and the increment u_k - u_0 must agree to
    1e-10 (the float64 parity bound; measured ~1e-13)."""
    phix, ctx = px
    n = 1024
    prm = synth.grayscott_params(n)
    u0 = synth.grayscott_state(n, seed=0)
    tol = 1e-8
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    gs = GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"])
    uo = u0
    worst = 0.0
    for k in range(20):
        st = phix.phix_exprb43_step(ctx, op, ud, prm["h"], tol, phix.PHIX_LEJA, phix.phix_opts_default())
        u4, u3, ost = integrators.exprb43_step(gs, uo, prm["h"], tol=tol)
        assert st.power_mv == ost["power_mv"] and st.iters == ost["iters"], (k, st.as_dict(), ost["iters"])
        assert st.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-8)
        got = host(ud)
        e = rel(got - u0, u4 - u0)
        worst = max(worst, e)
        assert e <= 1e-10, (k, e)
        assert rel(got, u4) <= 1e-12
        uo = u4
    print("worst increment error over 20 steps", worst)


@pytest.mark.parametrize("kind", ["advdiff", "grayscott", "burgers"])
def test_rhs_vs_oracle(px, kind):
    from oracle.operators import Burgers
    phix, ctx = px
    nx, ny = 40, 24
    rng = np.random.default_rng(11)
    if kind == "advdiff":
        prm, ncomp, kd = [0.3, 2.0, -1.0], 1, phix.PHIX_OP_ADVDIFF
        oop = AdvDiff(nx, *prm, ny=ny)
    elif kind == "grayscott":
        prm, ncomp, kd = [2e-3, 1e-3, 0.04, 0.06], 2, phix.PHIX_OP_GRAYSCOTT
        oop = GrayScott(nx, *prm, ny=ny)
    else:
        prm, ncomp, kd = [1e-2], 1, phix.PHIX_OP_BURGERS
        oop = Burgers(nx, *prm, ny=ny)
    u = rng.random(ncomp * nx * ny)
    ud = dev(u)
    fd = torch.empty_like(ud)
    phix.phix_rhs(ctx, phix.make_jop(kd, nx, ny, prm), ud, fd)
    assert rel(host(fd), oop.f(u)) <= 1e-13


def test_entry_smoke_runs(px):
    """The package's smoke entry (one phi-action and one EXPRB43 step, each
    against the oracle) completes on cuda:0."""
    import __graft_entry__
    __graft_entry__.smoke()
