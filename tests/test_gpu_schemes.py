"""GPU parity of every integrator of Sec. 5 (phix_step through the C-ABI)
against the oracle's step, for each method that scheme has: Leja, KIOPS and
LeKry (Sec. 5.1); exactness on a linear problem; and the host-buffer entry
point phix_step_host against the device one."""
import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import integrators, exact
from oracle.operators import GrayScott, Burgers, AdvDiff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(m_init=16, m_max=64, m_step=8)
SCHEMES = {"exprb43": 0, "epirk4s3": 1, "epirk4s3a": 2, "exprb53s3": 3, "epirk5p1": 4}
CASES = [("exprb43", "leja"), ("exprb43", "kiops"), ("epirk4s3", "leja"), ("epirk4s3", "kiops"),
         ("epirk4s3", "lekry"), ("epirk4s3a", "leja"), ("epirk4s3a", "kiops"), ("epirk4s3a", "lekry"),
         ("exprb53s3", "leja"), ("exprb53s3", "kiops"), ("exprb53s3", "lekry"), ("epirk5p1", "leja"),
         ("epirk5p1", "kiops")]


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


def method_of(phix, m):
    return {"leja": phix.PHIX_LEJA, "kiops": phix.PHIX_KIOPS, "lekry": phix.PHIX_LEKRY}[m]


@pytest.mark.parametrize("scheme,method", CASES)
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_scheme_step_grayscott_vs_oracle(px, scheme, method, prec):
    """One step on a 64 x 64 Gray-Scott state (h = 20x explicit, tol 1e-10):
    the increment u_new - u_0 within 1e-9 of the oracle's, the error
    estimate within 1e-6, the same power-iteration count."""
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
    st = phix.phix_step(ctx, SCHEMES[scheme], op, ud, h, tol, method_of(phix, method),
                        phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec)))
    uh, ul, ost = integrators.STEPS[scheme](GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0, h,
                                            method=method, tol=tol, kiops_kw=KW)
    got = ud.cpu().numpy()
    print(scheme, method, prec, "gpu", st.iters, "oracle", ost["iters"], ost["jv"], "err", rel(got - u0, uh - u0))
    assert rel(got - u0, uh - u0) <= 1e-9
    assert st.err_est == pytest.approx(np.linalg.norm(uh - ul), rel=1e-6)
    assert st.power_mv == ost["power_mv"]


@pytest.mark.parametrize("scheme,method", CASES)
def test_scheme_step_burgers_vs_oracle(px, scheme, method):
    """One step on a 96 x 96 Burgers state (imaginary bound from the state,
    substeps by the iota cap on the Leja side), double-float."""
    phix, ctx = px
    n = 96
    prm = synth.burgers_params(n, mult=10.0)
    u0 = synth.burgers_state(n, seed=4)
    rho_im = 2.0 * n * float(np.max(np.abs(u0)))
    tol = 1e-10
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [prm["nu"]])
    st = phix.phix_step(ctx, SCHEMES[scheme], op, ud, prm["h"], tol, method_of(phix, method),
                        phix.phix_opts_default(rho_im=rho_im))
    uh, ul, ost = integrators.STEPS[scheme](Burgers(n, prm["nu"]), u0, prm["h"], method=method, tol=tol,
                                            kiops_kw=KW, leja_kw=dict(rho_im=rho_im, iota_cap=4.0))
    got = ud.cpu().numpy()
    assert rel(got - u0, uh - u0) <= 1e-9
    assert st.err_est == pytest.approx(np.linalg.norm(uh - ul), rel=1e-6)


@pytest.mark.parametrize("scheme,method", CASES)
def test_scheme_linear_problem_is_exact(px, scheme, method):
    """Linear f: every remainder vanishes and the step is exp(hJ) u."""
    phix, ctx = px
    n = 32
    D, ax, ay = 0.5, 3.0, 2.0
    u0 = synth.advdiff_gaussian(n)
    h = 20.0 / (4 * D * n * n)
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay])
    phix.phix_step(ctx, SCHEMES[scheme], op, ud, h, 1e-12, method_of(phix, method),
                   phix.phix_opts_default(rho_re=8 * D * n * n))
    ex = exact.advdiff_phi_fft(n, D, ax, ay, h, u0, 0)
    assert rel(ud.cpu().numpy(), ex) <= 1e-10


def test_lekry_rejects_schemes_without_combinations(px):
    phix, ctx = px
    n = 16
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [1.0, 0.0, 0.0])
    ud = dev(synth.advdiff_gaussian(n))
    for sc in (phix.PHIX_EXPRB43, phix.PHIX_EPIRK5P1):
        st = phix.phix_step(ctx, sc, op, ud, 1e-4, 1e-8, phix.PHIX_LEKRY, None, check=False)
        assert st.status == phix.PHIX_EINVAL
    st = phix.phix_step(ctx, phix.PHIX_EPIRK4S3, op, ud, 1e-4, 1e-8, phix.PHIX_LEKRY,
                        phix.phix_opts_default(prec=phix.PHIX_FP32), check=False)
    assert st.status == phix.PHIX_EINVAL


@pytest.mark.parametrize("scheme", ["exprb43", "epirk5p1"])
def test_step_host_equals_device_step(px, scheme):
    """phix_step_host (state in page-locked host memory, copies inside the
    call) gives the device entry point's result bit for bit."""
    phix, ctx = px
    n = 64
    prm = synth.grayscott_params(n)
    prm["Du"] *= 64
    prm["Dv"] *= 64
    u0 = synth.grayscott_state(n, seed=5, patch=16)
    h = 20.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    ud = dev(u0)
    sd = phix.phix_step(ctx, SCHEMES[scheme], op, ud, h, 1e-9, phix.PHIX_LEJA)
    uh = torch.tensor(u0, dtype=torch.float64).pin_memory()
    sh = phix.phix_step_host(ctx, SCHEMES[scheme], op, uh, h, 1e-9, phix.PHIX_LEJA)
    assert torch.equal(uh, ud.cpu())
    assert sh.err_est == sd.err_est and sh.iters == sd.iters
    # pageable memory works too; a failed step leaves the host state unchanged
    up = torch.tensor(u0, dtype=torch.float64)
    phix.phix_step_host(ctx, SCHEMES[scheme], op, up, h, 1e-9, phix.PHIX_LEJA)
    assert torch.equal(up, ud.cpu())
    bad = torch.tensor(u0, dtype=torch.float64)
    st = phix.phix_step_host(ctx, SCHEMES[scheme], op, bad, h, 1e-9, phix.PHIX_LEJA,
                             phix.phix_opts_default(m_max=2), check=False)
    assert st.status == phix.PHIX_ENOTCONV
    assert torch.equal(bad, torch.tensor(u0, dtype=torch.float64))
