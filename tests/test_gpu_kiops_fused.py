"""GPU parity of the fused Arnoldi steps of the KIOPS-style method (one pass
per step on grids of whole 64 x 8 tiles) against the two-pass steps on the
same inputs, against the oracle's KIOPS-style method (Sec. 2.1) and on the
happy-breakdown special case.  Sizes: 64 x 64 (several tiles, periodic halo
ring at every edge), a rectangular 128 x 40 grid, and the augmented
combination with nonzero b-columns."""
import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import kiops, integrators
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


KW = dict(m_init=16, m_max=64, m_step=8)


def _opts(phix, prec, fused, **kw):
    return phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), kiops_fused=fused,
                                  **{"kiops_" + k: v for k, v in kw.items()})


def beta_aug(bs):
    p = len(bs) - 1
    nb = max([np.sum(np.abs(b)) for b in bs[1:] if b is not None], default=0.0)
    eta = 2.0 ** (-np.ceil(np.log2(nb))) if nb > 0 else 1.0
    b0 = bs[0] if bs[0] is not None else 0.0
    return float(np.sqrt(np.sum(np.square(b0)) + (1.0 / eta ** 2 if p > 0 else 0.0)))


def _gs_case(nx, ny, seed):
    rng = np.random.default_rng(seed)
    prm = [3e-3, 1.5e-3, 0.04, 0.06]
    u = np.concatenate([1 - 0.3 * rng.random(nx * ny), 0.3 * rng.random(nx * ny)])
    return prm, u


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 40)])
def test_fused_combination_matches_two_pass_and_oracle(px, prec, nx, ny):
    """The augmented combination sum_l phi_l(hJ) b_l (b_0, b_2, b_3 nonzero:
    two b-columns in every Arnoldi step) on a Gray-Scott Jacobian: the fused
    and two-pass steps take the same accept/reject path and agree to
    rounding; both agree with the oracle within its error control."""
    phix, ctx = px
    prm, u = _gs_case(nx, ny, 4)
    rng = np.random.default_rng(5)
    N = u.size
    bs = [rng.standard_normal(N), None, rng.standard_normal(N), 0.1 * rng.standard_normal(N)]
    h = 2.0 * (1.0 / nx) ** 2 / (4 * prm[0]) * 10
    tol = 1e-10
    sd = dev(u)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, nx, ny, prm, sd)
    bd = [dev(b) if b is not None else None for b in bs]
    outs, stats = [], []
    for fused in (1, 0):
        o = torch.empty(N, dtype=torch.float64, device="cuda")
        stats.append(phix.phix_phi_combination(ctx, op, h, bd, o, tol, phix.PHIX_KIOPS,
                                               _opts(phix, prec, fused, **KW)))
        outs.append(host(o))
    assert stats[0].iters == stats[1].iters and stats[0].substeps == stats[1].substeps
    assert stats[0].launches < stats[1].launches  # one launch per fused step, two otherwise
    # same decisions: the two arithmetic orders differ by rounding of the basis
    bound = 1e-12 if prec == "FP64" else 1e-11
    assert np.linalg.norm(outs[0] - outs[1]) <= bound * beta_aug(bs)
    gop = GrayScott(nx, *prm, state=u, ny=ny)
    ref, info = kiops.kiops(lambda x: h * gop.jv(x), bs, [1.0], tol, **KW)
    assert np.linalg.norm(outs[0] - ref[0]) <= max(1e-10, 2 * tol) * beta_aug(bs)


@pytest.mark.parametrize("scheme", ["exprb43", "epirk4s3"])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_fused_grayscott_step_vs_oracle(px, scheme, prec):
    phix, ctx = px
    n = 64
    prm = synth.grayscott_params(n)
    prm["Du"] *= 64
    prm["Dv"] *= 64
    u0 = synth.grayscott_state(n, seed=3, patch=16)
    h = 20.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
    tol = 1e-10
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    fn = phix.phix_exprb43_step if scheme == "exprb43" else phix.phix_epirk4s3_step
    st = fn(ctx, op, ud, h, tol, phix.PHIX_KIOPS, _opts(phix, prec, 1, **KW))
    ostep = integrators.exprb43_step if scheme == "exprb43" else integrators.epirk4s3_step
    u4, u3, ost = ostep(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0, h, method="kiops",
                        tol=tol, kiops_kw=KW)
    got = host(ud)
    assert rel(got - u0, u4 - u0) <= 1e-8
    assert st.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-6)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_fused_burgers_action_vs_oracle(px, prec):
    phix, ctx = px
    n = 64
    nu = 5e-3
    U = synth.burgers_state(n, seed=1)
    v = np.random.default_rng(2).standard_normal(n * n)
    h = 20.0 * (1.0 / n) ** 2 / (4 * nu)
    tol = 1e-10
    sd = dev(U)
    op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [nu], sd)
    vd = dev(v)
    outs = [torch.empty_like(vd) for _ in range(2)]
    for fused, o in zip((1, 0), outs):
        phix.phix_phi_action(ctx, op, h, vd, [1], [1.0], [o], tol, phix.PHIX_KIOPS, _opts(phix, prec, fused, **KW))
    bop = Burgers(n, nu, state=U)
    ref, infos = kiops.kiops_phi(lambda x: h * bop.jv(x), v, [(1, 1.0)], tol, **KW)
    bs = [None, v]
    assert np.linalg.norm(host(outs[0]) - host(outs[1])) <= (1e-12 if prec == "FP64" else 1e-11) * beta_aug(bs)
    assert np.linalg.norm(host(outs[0]) - ref[0]) <= max(1e-10, 2 * tol) * beta_aug(bs)


def test_fused_happy_breakdown(px):
    """J(const) = 0 (periodic advection-diffusion): the fused step sees the
    zero orthogonalised vector, stops the basis at one vector, and
    exp(hJ) v = v to rounding."""
    phix, ctx = px
    n = 64
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [1.0, 2.0, 3.0])
    vd = torch.full((n * n,), 0.75, dtype=torch.float64, device="cuda")
    out = torch.empty_like(vd)
    st = phix.phix_phi_action(ctx, op, 0.01, vd, [0], [1.0], [out], 1e-10, phix.PHIX_KIOPS,
                              phix.phix_opts_default(kiops_fused=1))
    assert st.iters == 1 and st.substeps == 1
    assert torch.allclose(out, vd, rtol=1e-12, atol=0)


def test_fused_advdiff_vs_oracle_many_substeps(px):
    """A stiff advection-diffusion action that needs several substeps and
    basis growth (rejections): every restart of the fused steps from a new
    start vector, and every continuation after a rejection, reuses the
    scratch vectors correctly."""
    phix, ctx = px
    n = 64
    D, ax, ay = 0.8, 2.0, -3.0
    v = synth.advdiff_gaussian(n)
    h = 200.0 / (4 * D * n * n)
    tol = 1e-9
    kw = dict(m_init=8, m_max=16, m_step=4)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay])
    vd = dev(v)
    od = torch.empty_like(vd)
    st = phix.phix_phi_action(ctx, op, h, vd, [1], [1.0], [od], tol, phix.PHIX_KIOPS,
                              _opts(phix, "DF64", 1, **kw))
    ref, infos = kiops.kiops_phi(lambda x: h * AdvDiff(n, D, ax, ay).jv(x), v, [(1, 1.0)], tol, **kw)
    assert st.substeps > 2 and st.rejections > 0
    assert np.linalg.norm(host(od) - ref[0]) <= max(1e-10, 2 * tol) * beta_aug([None, v])
