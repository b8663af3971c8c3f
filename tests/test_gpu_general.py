"""The general float64 path through the C-ABI against the oracle: the
paper's no-flow problems (Sec. 3: ADR, Allen-Cahn, Brusselator on
cell-centred Neumann grids) in phi-actions and EXPRB43 steps, the
finite-difference ("numerical") Jacobian of Sec. 4, and the
augmented-matrix Leja combination of Appendix A."""
import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import leja, integrators, variants, problems, kiops
from oracle.operators import GrayScott, AdvDiff

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


def problem(phix, kind, n):
    """(phix kind, params, oracle operator at its state, state, h)."""
    if kind == "adr":
        prm = [0.1, -10.0, 100.0]   # the paper's case (a)
        u = synth.adr_state(n)
        op = problems.ADR(n, *prm, state=u)
        k = phix.PHIX_OP_ADR
        h = 5.0 * (1.0 / n) ** 2 / (4 * prm[0])
    elif kind == "allen_cahn":
        prm = [0.01]
        u = synth.allen_cahn_state(n)
        op = problems.AllenCahn(n, *prm, state=u)
        k = phix.PHIX_OP_ALLEN_CAHN
        h = 50.0 * (2.0 / n) ** 2 / (4 * prm[0])
    else:
        prm = [0.01]
        u = synth.brusselator_state(n)
        op = problems.Brusselator(n, *prm, state=u)
        k = phix.PHIX_OP_BRUSSELATOR
        h = 20.0 * (1.0 / n) ** 2 / (4 * prm[0])
    return k, prm, op, u, h


@pytest.mark.parametrize("kind", ["adr", "allen_cahn", "brusselator"])
def test_rhs_of_no_flow_problems(px, kind):
    phix, ctx = px
    n = 40
    k, prm, op, u, h = problem(phix, kind, n)
    f = torch.empty(u.size, dtype=torch.float64, device="cuda")
    phix.phix_rhs(ctx, phix.make_jop(k, n, n, prm), dev(u), f)
    assert rel(f.cpu().numpy(), op.f(u)) <= 1e-13


@pytest.mark.parametrize("kind", ["adr", "allen_cahn", "brusselator"])
def test_no_flow_phi_actions_vs_oracle(px, kind):
    """Vertical Leja phi_0, phi_1(1/2), phi_1, float64 whatever opts->prec, the
    power iteration (same SplitMix64 start) checked on its own.  Each problem
    needs its spectrum's shape: ADR's centred advection (cell Peclet ~1) the
    imaginary bound 2 |b| / dx, with substeps; Allen-Cahn's reaction term
    1 - 3u^2 ~ 1 the interval's right end at +1."""
    phix, ctx = px
    n = 48
    k, prm, op, u, h = problem(phix, kind, n)
    v = np.random.default_rng(5).standard_normal(u.size)
    outs = [(0, 1.0), (1, 0.5), (1, 1.0)]
    jop = phix.make_jop(k, n, n, prm, dev(u))
    rho_g, sp = phix.phix_spectrum(ctx, jop, phix.phix_opts_default())
    rho, mv = leja.power_iteration(op.jv, u.size)
    assert sp.power_mv == mv and rho_g == pytest.approx(rho, rel=1e-12)
    kw, okw = dict(rho_re=1.2 * rho), {}
    beta = 0.0
    if kind == "adr":
        kw["rho_im"] = 2.0 * abs(prm[1]) * n
        okw = dict(rho_im=kw["rho_im"], iota_cap=4.0)
    elif kind == "allen_cahn":
        kw["rho_hi"] = beta = 1.0
    od = [torch.empty(u.size, dtype=torch.float64, device="cuda") for _ in outs]
    st = phix.phix_phi_action(ctx, jop, h, dev(v), [l for l, _ in outs], [s for _, s in outs], od, 1e-10,
                              phix.PHIX_LEJA, phix.phix_opts_default(**kw))
    ref, info = leja.leja_phi(op.jv, v, h, -1.2 * rho, beta, outs, 1e-10, **okw)
    assert st.iters == info["iters"] and st.substeps == info["substeps"]
    for o, r in zip(od, ref):
        assert rel(o.cpu().numpy(), r) <= 1e-10


@pytest.mark.parametrize("kind", ["adr", "allen_cahn", "brusselator"])
def test_no_flow_exprb43_step_vs_oracle(px, kind):
    """One EXPRB43 step (Leja, interval from the power iteration every step),
    with each problem's spectral shape as in the phi-action test."""
    phix, ctx = px
    n = 32
    k, prm, op, u, h = problem(phix, kind, n)
    ud = dev(u)
    base = problems.ADR(n, *prm) if kind == "adr" else (problems.AllenCahn(n, *prm) if kind == "allen_cahn"
                                                          else problems.Brusselator(n, *prm))
    kw, okw, spec = {}, {}, None
    if kind == "adr":
        kw["rho_im"] = 2.0 * abs(prm[1]) * n
        okw = dict(leja_kw=dict(rho_im=kw["rho_im"], iota_cap=4.0))
    elif kind == "allen_cahn":
        kw["rho_hi"] = 1.0
        rho, _ = leja.power_iteration(op.jv, u.size)
        spec = (-1.2 * rho, 1.0)
    st = phix.phix_step(ctx, phix.PHIX_EXPRB43, phix.make_jop(k, n, n, prm), ud, h, 1e-10, phix.PHIX_LEJA,
                        phix.phix_opts_default(**kw))
    u4, u3, ost = integrators.exprb43_step(base, u, h, tol=1e-10, spec=spec, **okw)
    assert rel(ud.cpu().numpy() - u, u4 - u) <= 1e-9
    assert st.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-6)


@pytest.mark.parametrize("kind", ["adr", "allen_cahn", "brusselator"])
def test_no_flow_kiops_vs_oracle(px, kind):
    """KIOPS on the no-flow problems (float64 general Arnoldi pass): phi_0 and
    phi_1 at output times 1/2, 1 against the oracle's KIOPS-style method."""
    phix, ctx = px
    n = 32
    k, prm, op, u, h = problem(phix, kind, n)
    v = np.random.default_rng(9).standard_normal(u.size)
    outs = [(0, 1.0), (1, 0.5), (1, 1.0)]
    jop = phix.make_jop(k, n, n, prm, dev(u))
    od = [torch.empty(u.size, dtype=torch.float64, device="cuda") for _ in outs]
    kw = dict(m_init=16, m_max=64, m_step=8)
    st = phix.phix_phi_action(ctx, jop, h, dev(v), [l for l, _ in outs], [s for _, s in outs], od, 1e-10,
                              phix.PHIX_KIOPS, phix.phix_opts_default())
    ref, infos = kiops.kiops_phi(lambda x: h * op.jv(x), v, outs, 1e-10, **kw)
    assert st.iters == sum(i["matvecs"] for i in infos)
    for o, r in zip(od, ref):
        assert rel(o.cpu().numpy(), r) <= 1e-10


@pytest.mark.parametrize("kind,scheme,method", [("adr", "epirk4s3", "lekry"), ("brusselator", "exprb53s3", "kiops"),
                                                ("allen_cahn", "epirk5p1", "kiops")])
def test_no_flow_krylov_steps_vs_oracle(px, kind, scheme, method):
    phix, ctx = px
    n = 32
    k, prm, op, u, h = problem(phix, kind, n)
    base = problems.ADR(n, *prm) if kind == "adr" else (problems.AllenCahn(n, *prm) if kind == "allen_cahn"
                                                          else problems.Brusselator(n, *prm))
    kw, okw = {}, {}
    if kind == "adr" and method == "lekry":
        kw["rho_im"] = 2.0 * abs(prm[1]) * n
        okw = dict(leja_kw=dict(rho_im=kw["rho_im"], iota_cap=4.0))
    ud = dev(u)
    sch = {"epirk4s3": phix.PHIX_EPIRK4S3, "exprb53s3": phix.PHIX_EXPRB53S3, "epirk5p1": phix.PHIX_EPIRK5P1}[scheme]
    meth = phix.PHIX_LEKRY if method == "lekry" else phix.PHIX_KIOPS
    st = phix.phix_step(ctx, sch, phix.make_jop(k, n, n, prm), ud, h, 1e-10, meth,
                        phix.phix_opts_default(prec=phix.PHIX_FP64, **kw))
    uh, ul, ost = integrators.STEPS[scheme](base, u, h, method=method, tol=1e-10,
                                            kiops_kw=dict(m_init=16, m_max=64, m_step=8), **okw)
    assert rel(ud.cpu().numpy() - u, uh - u) <= 1e-9
    assert st.err_est == pytest.approx(np.linalg.norm(uh - ul), rel=1e-6)


@pytest.mark.parametrize("kind", ["grayscott", "brusselator"])
def test_finite_difference_jacobian_vs_oracle(px, kind):
    """PHIX_JV_FD: the Newton basis built from (f(u + eps y) - f(u)) / eps.
    Both sides round f(u + eps y) in float64 and divide by eps ~ 1e-8 / ||y||,
    so each product carries ~2^-52 / eps ~ 1e-8 of rounding that differs
    between the two implementations: 1e-7 is the bound on the result."""
    phix, ctx = px
    n = 40
    if kind == "grayscott":
        prm = [2e-3, 1e-3, 0.04, 0.06]
        u = synth.grayscott_state(n, seed=2, patch=12)
        base = GrayScott(n, *prm)
        k = phix.PHIX_OP_GRAYSCOTT
        h = 20.0 * (1.0 / n) ** 2 / (4 * prm[0])
    else:
        k, prm, op, u, h = problem(phix, kind, n)
        base = problems.Brusselator(n, *prm)
    v = np.random.default_rng(6).standard_normal(u.size)
    jop = phix.make_jop(k, n, n, prm, dev(u))
    od = [torch.empty(u.size, dtype=torch.float64, device="cuda") for _ in range(2)]
    st = phix.phix_phi_action(ctx, jop, h, dev(v), [1, 1], [0.5, 1.0], od, 1e-9, phix.PHIX_LEJA,
                              phix.phix_opts_default(jv=phix.PHIX_JV_FD))
    fdjv = variants.fd_jv(base.f, u)
    rho, mv = leja.power_iteration(fdjv, u.size)
    ref, info = leja.leja_phi(fdjv, v, h, -1.2 * rho, 0.0, [(1, 0.5), (1, 1.0)], 1e-9)
    assert abs(st.iters - info["iters"]) <= 1
    for o, r in zip(od, ref):
        assert rel(o.cpu().numpy(), r) <= 1e-7
    # and the finite-difference result stays close to the analytic Jacobian's
    oa = [torch.empty_like(od[0]) for _ in range(2)]
    phix.phix_phi_action(ctx, jop, h, dev(v), [1, 1], [0.5, 1.0], oa, 1e-9, phix.PHIX_LEJA,
                         phix.phix_opts_default(prec=phix.PHIX_FP64))
    assert rel(od[1].cpu().numpy(), oa[1].cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("p", [1, 3, 4])
def test_augmented_leja_combination_vs_oracle(px, p):
    """sum_j phi_j(hJ) b_j as exp of the augmented matrix by one Leja pass
    (Appendix A) against the oracle's augmented Leja and against KIOPS."""
    phix, ctx = px
    n = 32
    D, ax, ay = 0.5, 3.0, 2.0
    op = AdvDiff(n, D, ax, ay)
    rng = np.random.default_rng(7)
    bs = [rng.standard_normal(n * n) for _ in range(p + 1)]
    if p >= 3:
        bs[2] = None
    h = 20.0 / (4 * D * n * n)
    rho = 8.0 * D * n * n
    jop = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay])
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    bd = [dev(b) if b is not None else None for b in bs]
    st = phix.phix_phi_combination(ctx, jop, h, bd, out, 1e-11, phix.PHIX_LEJA,
                                   phix.phix_opts_default(rho_re=rho, leja_augmented=1))
    ref, m = variants.leja_combination_augmented(op.jv, bs, h, -rho, 0.0, 1e-11)
    assert st.iters == m
    got = out.cpu().numpy()
    assert rel(got, ref) <= 1e-10
    kv, _ = kiops.kiops(lambda x: h * op.jv(x), bs, [1.0], 1e-12)
    assert rel(got, kv[0]) <= 1e-8
