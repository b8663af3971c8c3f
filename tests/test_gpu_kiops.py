"""GPU parity of the KIOPS-style Krylov path (C-ABI) against the oracle's
KIOPS-style method (same controller), the FFT-exact result and the dense
augmented exponential (Theorem of Sec. 2.1)."""
import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import exact, kiops, integrators
from oracle.operators import AdvDiff, GrayScott, with_state

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


def beta_aug(bs):
    """Norm of the augmented start vector [b_0; e_p / eta] of the KIOPS-style
    method, eta = 2^-ceil(log2 max_j ||b_j||_1): the scale its error control
    (tol per unit step, relative to this norm) refers to."""
    p = len(bs) - 1
    nb = max([np.sum(np.abs(b)) for b in bs[1:] if b is not None], default=0.0)
    eta = 2.0 ** (-np.ceil(np.log2(nb))) if nb > 0 else 1.0
    b0 = bs[0] if bs[0] is not None else 0.0
    return float(np.sqrt(np.sum(np.square(b0)) + (1.0 / eta ** 2 if p > 0 else 0.0)))


def kiops_parity(got, ref, bs, tol):
    """Both sides satisfy the same error control independently; with the same
    accept/reject path they agree to rounding, and a decision flipped at
    rounding level (omega ~ 1) moves a result by at most ~tol * beta_aug."""
    return np.linalg.norm(got - ref) <= max(1e-10, 2.0 * tol) * beta_aug(bs)


def _opts(phix, prec, **kw):
    return phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), **{"kiops_" + k: v for k, v in kw.items()})


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_kiops_advdiff_64_vs_oracle_and_fft(px, prec):
    phix, ctx = px
    n = 64
    p = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    outs = [(0, 1.0), (1, 1.0), (2, 1.0), (3, 1.0)]
    tol = 1e-10
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
    vd = dev(v)
    od = [torch.empty_like(vd) for _ in outs]
    st = phix.phix_phi_action(ctx, op, p["h"], vd, [l for l, _ in outs], [s for _, s in outs], od, tol,
                              phix.PHIX_KIOPS, _opts(phix, prec, **KW))
    aop = AdvDiff(n, p["D"], p["ax"], p["ay"])
    ref, infos = kiops.kiops_phi(lambda x: p["h"] * aop.jv(x), v, outs, tol, **KW)
    print(prec, "gpu matvecs", st.iters, "oracle", sum(i["matvecs"] for i in infos))
    for (l, s), r, o in zip(outs, od, ref):
        got = host(r)
        bs = [None] * (l + 1)
        bs[l] = v
        assert kiops_parity(got, o, bs, tol), (l, np.linalg.norm(got - o), beta_aug(bs))
        ex = exact.advdiff_phi_fft(n, p["D"], p["ax"], p["ay"], s * p["h"], v, l)
        assert np.linalg.norm(got - ex) <= 10 * tol * beta_aug(bs)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_kiops_output_times_and_small_basis(px, prec):
    phix, ctx = px
    n = 32
    D, ax, ay = 0.8, 2.0, -3.0
    v = synth.advdiff_gaussian(n)
    h = 60.0 / (4 * D * n * n)
    outs = [(1, 0.5), (1, 1.0), (1, 1.0 / 9.0)]
    tol = 1e-9
    kw = dict(m_init=8, m_max=12, m_step=4)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay])
    vd = dev(v)
    od = [torch.empty_like(vd) for _ in outs]
    st = phix.phix_phi_action(ctx, op, h, vd, [l for l, _ in outs], [s for _, s in outs], od, tol,
                              phix.PHIX_KIOPS, _opts(phix, prec, **kw))
    aop = AdvDiff(n, D, ax, ay)
    ref, infos = kiops.kiops_phi(lambda x: h * aop.jv(x), v, outs, tol, **kw)
    assert st.substeps > 2 and st.rejections > 0
    for (l, s), r, o in zip(outs, od, ref):
        assert kiops_parity(host(r), o, [None, v], tol)
        ex = exact.advdiff_phi_fft(n, D, ax, ay, s * h, v, l)
        assert np.linalg.norm(host(r) - ex) <= 10 * tol * beta_aug([None, v])


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_kiops_combination_vs_dense_augmented(px, prec):
    phix, ctx = px
    n = 10
    rng = np.random.default_rng(8)
    prm = [3e-3, 1e-3, 0.04, 0.06]
    u = np.concatenate([1 - 0.3 * rng.random(n * n), 0.3 * rng.random(n * n)])
    gop = GrayScott(n, *prm, state=u)
    A = exact.dense_matrix(gop.jv, u.size)
    h = 3.0
    bs = [rng.standard_normal(u.size), None, rng.standard_normal(u.size), 0.1 * rng.standard_normal(u.size)]
    tol = 1e-11
    sd = dev(u)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, prm, sd)
    bd = [dev(b) if b is not None else None for b in bs]
    out = torch.empty(u.size, dtype=torch.float64, device="cuda")
    st = phix.phix_phi_combination(ctx, op, h, bd, out, tol, phix.PHIX_KIOPS,
                                   _opts(phix, prec, m_init=8, m_max=24, m_step=8))
    ref_o, info = kiops.kiops(lambda x: h * gop.jv(x), bs, [1.0], tol, m_init=8, m_max=24, m_step=8)
    assert kiops_parity(host(out), ref_o[0], bs, tol)
    ref = exact.augmented_phi_sum(h * A, bs)
    assert rel(host(out), ref) <= 1e-9


def test_kiops_happy_breakdown(px):
    # J(const) = 0 for the periodic advection-diffusion operator: the Krylov
    # space of a constant vector is one-dimensional, exp(hJ) v = v
    phix, ctx = px
    n = 16
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [1.0, 2.0, 3.0])
    vd = torch.full((n * n,), 0.75, dtype=torch.float64, device="cuda")
    out = torch.empty_like(vd)
    st = phix.phix_phi_action(ctx, op, 0.01, vd, [0], [1.0], [out], 1e-10, phix.PHIX_KIOPS,
                              phix.phix_opts_default())
    assert st.iters == 1 and st.substeps == 1
    # J v = 0 is a cancellation of stencil products of size ~200: double-float
    # leaves ~2^-47 of that, so exp(hJ) v = v holds to rounding, not exactly
    assert torch.allclose(out, vd, rtol=1e-12, atol=0)
    ref, info = kiops.kiops(lambda x: 0.01 * AdvDiff(n, 1.0, 2.0, 3.0).jv(x), [np.full(n * n, 0.75)], [1.0], 1e-10)
    assert info["matvecs"] == 1


@pytest.mark.parametrize("scheme", ["exprb43", "epirk4s3"])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_kiops_steps_grayscott_small(px, scheme, prec):
    phix, ctx = px
    n = 48
    prm = synth.grayscott_params(n)
    prm["Du"] *= 64
    prm["Dv"] *= 64
    u0 = synth.grayscott_state(n, seed=2, patch=12)
    h = 20.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
    tol = 1e-10
    ud = dev(u0)
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    fn = phix.phix_exprb43_step if scheme == "exprb43" else phix.phix_epirk4s3_step
    st = fn(ctx, op, ud, h, tol, phix.PHIX_KIOPS, _opts(phix, prec, **KW))
    ostep = integrators.exprb43_step if scheme == "exprb43" else integrators.epirk4s3_step
    u4, u3, ost = ostep(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0, h, method="kiops",
                        tol=tol, kiops_kw=KW)
    got = host(ud)
    assert rel(got - u0, u4 - u0) <= 1e-8
    assert st.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-6)


def test_kiops_grayscott_1024_step_vs_oracle(px):
    """Full-size Gray-Scott EXPRB43 step by KIOPS (double-float Arnoldi, the
    bench's KIOPS leg) against the oracle's KIOPS-style step: same controller,
    so the same accept/reject path and Arnoldi step count, and then the
    increment agrees to the float64 parity bound (measured ~1e-13)."""
    phix, ctx = px
    n = 1024
    prm = synth.grayscott_params(n)
    u0 = synth.grayscott_state(n, seed=0)
    tol = 1e-8
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    uk = dev(u0)
    sk = phix.phix_exprb43_step(ctx, op, uk, prm["h"], tol, phix.PHIX_KIOPS, phix.phix_opts_default())
    u4, u3, ost = integrators.exprb43_step(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0,
                                           prm["h"], method="kiops", tol=tol, kiops_kw=KW)
    got = host(uk)
    print("gpu arnoldi steps", sk.iters, "oracle matvecs", ost["jv"])
    assert sk.iters == ost["jv"]
    assert rel(got - u0, u4 - u0) <= 1e-10
    assert sk.err_est == pytest.approx(np.linalg.norm(u4 - u3), rel=1e-8)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
@pytest.mark.parametrize("c", [2.0 ** -90, 2.0 ** 90])
def test_kiops_scales_with_its_input(px, prec, c):
    """phi_l(A)(c v) = c phi_l(A) v.  With c a power of two every rounding of
    the method scales with it, so the results agree to rounding; the Krylov
    basis must stay inside the double-float range however small or large the
    input is (tiny inputs arise in practice: the nonlinear remainders that
    feed phi_3 and phi_4 near a steady state)."""
    phix, ctx = px
    n = 64
    p = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
    outs = [(0, 1.0), (1, 1.0)]
    res = {}
    for scale in (1.0, c):
        vd = dev(scale * v)
        od = [torch.empty_like(vd) for _ in outs]
        st = phix.phix_phi_action(ctx, op, p["h"], vd, [l for l, _ in outs], [s for _, s in outs], od, 1e-10,
                                  phix.PHIX_KIOPS, _opts(phix, prec, **KW))
        assert st.status == 0
        res[scale] = [host(t) / scale for t in od]
    for a, b in zip(res[c], res[1.0]):
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
@pytest.mark.parametrize("case", ["odd_grid", "offset_output"])
def test_kiops_combination_element_and_pair_paths(px, prec, case):
    """The basis combination reads element pairs with 16-byte loads when the
    unknown count is even and the slots and the output are 16-byte aligned,
    and single elements otherwise: an odd grid (45 x 37) and an output view
    one float64 past an aligned address take the element path.  Both against
    the oracle's KIOPS-style method; the offset output also against the same
    action into aligned outputs (pair path), equal to rounding."""
    phix, ctx = px
    nx, ny = (45, 37) if case == "odd_grid" else (48, 40)
    D, ax, ay = 0.5, 1.5, -2.0
    h = 40.0 / (4 * D * (nx * nx + ny * ny))
    v = np.random.default_rng(21).standard_normal(nx * ny)
    outs = [(1, 0.5), (2, 1.0)]
    tol = 1e-9
    kw = dict(m_init=8, m_max=24, m_step=4)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, nx, ny, [D, ax, ay])
    vd = dev(v)
    if case == "offset_output":
        bufs = [torch.empty(nx * ny + 1, dtype=torch.float64, device="cuda") for _ in outs]
        od = [b[1:] for b in bufs]
        assert all(o.data_ptr() % 16 == 8 for o in od)
    else:
        od = [torch.empty_like(vd) for _ in outs]
    st = phix.phix_phi_action(ctx, op, h, vd, [l for l, _ in outs], [s for _, s in outs], od, tol,
                              phix.PHIX_KIOPS, _opts(phix, prec, **kw))
    assert st.status == 0
    aop = AdvDiff(nx, D, ax, ay, ny=ny)
    ref, _ = kiops.kiops_phi(lambda x: h * aop.jv(x), v, outs, tol, **kw)
    for (l, s), r, o in zip(outs, od, ref):
        bs = [None] * (l + 1)
        bs[l] = v
        assert kiops_parity(host(r), o, bs, tol)
    if case == "offset_output":
        od2 = [torch.empty_like(vd) for _ in outs]
        st2 = phix.phix_phi_action(ctx, op, h, vd, [l for l, _ in outs], [s for _, s in outs], od2, tol,
                                   phix.PHIX_KIOPS, _opts(phix, prec, **kw))
        assert st2.iters == st.iters and st2.substeps == st.substeps
        for a, b in zip(od, od2):
            assert rel(host(a), host(b)) <= 1e-13
