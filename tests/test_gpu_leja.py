"""GPU parity of the Leja phi-action (C-ABI) against the CPU oracle.

Same inputs, same spectral interval (given, or from the same SplitMix64
power iteration), element by element, relative 2-norm per output.
"""
import math

import numpy as np
import pytest

import synth
from gpu_util import rel, parity_tol
from oracle import exact, leja
from oracle.operators import AdvDiff, GrayScott, Burgers, with_state

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


PRECS = ["FP64", "DF64"]


def _prec(phix, name):
    return getattr(phix, "PHIX_" + name)


def _run_action(phix, ctx, kind, nx, ny, params, state, v, h, outs, tol, prec, **opt):
    sd = dev(state) if state is not None else None
    op = phix.make_jop(kind, nx, ny, params, sd)
    o = phix.phix_opts_default(prec=_prec(phix, prec), **opt)
    vd = dev(v)
    od = [torch.empty_like(vd) for _ in outs]
    st = phix.phix_phi_action(ctx, op, h, vd, [l for l, _ in outs], [s for _, s in outs], od, tol,
                              phix.PHIX_LEJA, o)
    return [host(t) for t in od], st


@pytest.mark.parametrize("prec", PRECS)
def test_advdiff_64_phi0123_vs_oracle_and_fft(px, prec):
    phix, ctx = px
    n = 64
    p = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    rho = 8.0 * p["D"] * n * n
    outs = [(0, 1.0), (1, 1.0), (2, 1.0), (3, 1.0)]
    tol = 1e-10
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]], None, v,
                          p["h"], outs, tol, prec, rho_re=rho)
    op = AdvDiff(n, p["D"], p["ax"], p["ay"])
    ref, info = leja.leja_phi(op.jv, v, p["h"], -rho, 0.0, outs, tol)
    assert st.status == 0 and info["status"] == 0
    for (l, s), r, o in zip(outs, res, ref):
        assert rel(r, o) <= parity_tol(st.iters == info["iters"], tol), (l, rel(r, o), st.iters, info["iters"])
        ex = exact.advdiff_phi_fft(n, p["D"], p["ax"], p["ay"], s * p["h"], v, l)
        assert rel(r, ex) <= 10 * tol


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nx,ny", [(5, 5), (17, 17), (31, 31), (100, 100), (24, 10), (9, 40), (3, 3)])
def test_ragged_grids_advdiff(px, prec, nx, ny):
    phix, ctx = px
    rng = np.random.default_rng(nx * 100 + ny)
    D = rng.uniform(0.1, 1)
    # keep |Im lambda| below the real extent: advection scaled with D * n
    ax, ay = rng.uniform(-1, 1, 2) * D * min(nx, ny) / 2
    v = rng.standard_normal(nx * ny)
    rho = 4.0 * D * (nx * nx + ny * ny)
    h = 20.0 / rho
    outs = [(0, 1.0), (2, 0.5)]
    tol = 1e-11
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, nx, ny, [D, ax, ay], None, v, h, outs, tol,
                          prec, rho_re=rho)
    op = AdvDiff(nx, D, ax, ay, ny=ny)
    ref, info = leja.leja_phi(op.jv, v, h, -rho, 0.0, outs, tol)
    for r, o in zip(res, ref):
        assert rel(r, o) <= parity_tol(st.iters == info["iters"], tol)


def _gs_state(n, seed=1, ny=None):
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    return np.concatenate([1 - 0.4 * rng.random(n * ny), 0.3 * rng.random(n * ny)])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nx,ny", [(48, 48), (33, 20)])
def test_grayscott_power_iteration_and_vertical(px, prec, nx, ny):
    phix, ctx = px
    prm = [2e-5 * 40, 1e-5 * 40, 0.04, 0.06]
    u = _gs_state(nx, ny=ny)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(u.size)
    op = GrayScott(nx, *prm, state=u, ny=ny)
    h = 30.0 / (8 * prm[0] * nx * nx)
    outs = [(1, 0.5), (1, 1.0)]
    tol = 1e-10
    res, st = _run_action(phix, ctx, phix.PHIX_OP_GRAYSCOTT, nx, ny, prm, u, v, h, outs, tol, prec)
    rho, mv = leja.power_iteration(op.jv, u.size)
    assert st.power_mv == mv
    assert abs(st.rho - rho) <= 1e-12 * rho
    ref, info = leja.leja_phi(op.jv, v, h, -1.2 * rho, 0.0, outs, tol)
    for r, o in zip(res, ref):
        assert rel(r, o) <= parity_tol(st.iters == info["iters"], tol)


@pytest.mark.parametrize("prec", PRECS)
def test_burgers_vs_oracle(px, prec):
    phix, ctx = px
    n = 40
    nu = 2e-2
    X, Y = synth.grid_xy(n)
    u = (np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)).reshape(-1) + 0.05 * np.random.default_rng(3).standard_normal(n * n)
    op = Burgers(n, nu, state=u)
    v = op.f(u)
    h = 10.0 / (8 * nu * n * n)
    outs = [(1, 1.0)]
    tol = 1e-10
    res, st = _run_action(phix, ctx, phix.PHIX_OP_BURGERS, n, n, [nu], u, v, h, outs, tol, prec)
    rho, mv = leja.power_iteration(op.jv, u.size)
    assert abs(st.rho - rho) <= 1e-12 * rho
    ref, info = leja.leja_phi(op.jv, v, h, -1.2 * rho, 0.0, outs, tol)
    assert rel(res[0], ref[0]) <= parity_tol(st.iters == info["iters"], tol)
    A = exact.dense_matrix(op.jv, u.size)
    ex = exact.dense_phi(h * A, 1, v)
    assert rel(res[0], ex) <= 100 * tol


@pytest.mark.parametrize("prec", PRECS)
def test_substeps_gamma_and_imaginary_caps(px, prec):
    phix, ctx = px
    n = 16
    D, ax, ay = 1.0, 10.0, 10.0
    v = synth.advdiff_gaussian(n)
    h = 50.0 / (4 * D * n * n)
    rho = 8 * D * n * n
    outs = [(1, 1.0 / 8), (1, 1.0 / 9), (1, 1.0)]
    tol = 1e-11
    kw = dict(rho_re=rho, rho_im=(ax + ay) * n, iota_cap=4.0, gamma_cap=200.0)
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [D, ax, ay], None, v, h, outs, tol, prec, **kw)
    op = AdvDiff(n, D, ax, ay)
    ref, info = leja.leja_phi(op.jv, v, h, -rho, 0.0, outs, tol, rho_im=(ax + ay) * n, iota_cap=4.0)
    assert st.substeps == info["substeps"] and st.substeps > 3
    for (l, s), r, o in zip(outs, res, ref):
        assert rel(r, o) <= parity_tol(st.iters == info["iters"], tol)
        assert rel(r, exact.advdiff_phi_fft(n, D, ax, ay, s * h, v, l)) <= 1e-9
    # gamma cap: phi_0 and phi_3 substepped
    outs = [(0, 1.0), (3, 1.0)]
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [D, 1.0, 1.0], None, v, 4 * h, outs, tol,
                          prec, rho_re=rho, gamma_cap=12.0)
    op = AdvDiff(n, D, 1.0, 1.0)
    ref, info = leja.leja_phi(op.jv, v, 4 * h, -rho, 0.0, outs, tol, gamma_cap=12.0)
    assert st.substeps == info["substeps"] > 2
    for r, o in zip(res, ref):
        assert rel(r, o) <= parity_tol(st.iters == info["iters"], tol)


@pytest.mark.parametrize("prec", ["FP32_JV", "FP32"])
def test_reduced_precision_meets_1e6_on_advdiff_64(px, prec):
    """Float32 iteration arithmetic on the small advection-diffusion workload
    (64^2, h = 50x the explicit diffusive step, phi_0..phi_3): every output
    within the pure-float32 tolerance 1e-6 of the FFT-exact result."""
    phix, ctx = px
    n = 64
    p = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    rho = 8.0 * p["D"] * n * n
    outs = [(0, 1.0), (1, 1.0), (2, 1.0), (3, 1.0)]
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]], None, v,
                          p["h"], outs, 1e-8, prec, rho_re=rho)
    for (l, _), r in zip(outs, res):
        err = rel(r, exact.advdiff_phi_fft(n, p["D"], p["ax"], p["ay"], p["h"], v, l))
        print(prec, "phi_%d rel err vs exact" % l, err, "iters", st.iters)
        assert err <= 1e-6, (l, err)


def test_reduced_precision_on_burgers_256(px):
    """Burgers (256^2, h = 50x explicit, phi_1 of f(u) h, imaginary bound from
    the state): the double-float form meets the 1e-8 target against the
    float64 path and both float32 forms the pure-float32 tolerance 1e-6.
    (On this grid the advection bound splits the action into ~32 substeps of
    small h gamma, which keeps float32 rounding small; the 2048^2 workload,
    4 substeps of h gamma ~ 32, carries ~2e-5 and is reported by the bench.)"""
    phix, ctx = px
    n = 256
    prm = synth.burgers_params(n)
    u = synth.burgers_state(n, seed=2)
    op = Burgers(n, prm["nu"], state=u)
    v = op.f(u) * prm["h"]
    rho_im = 2.0 * n * float(np.max(np.abs(u)))
    res = {}
    for prec in ["FP64", "DF64", "FP32_JV", "FP32"]:
        r, st = _run_action(phix, ctx, phix.PHIX_OP_BURGERS, n, n, [prm["nu"]], u, v, prm["h"], [(1, 1.0)],
                            1e-8, prec, rho_im=rho_im)
        res[prec] = r[0]
    errs = {p_: rel(res[p_], res["FP64"]) for p_ in res}
    print("errors vs float64", errs)
    assert errs["DF64"] <= 1e-8
    assert errs["FP32_JV"] <= 1e-6 and errs["FP32"] <= 1e-6


def test_zero_vector_and_zero_step(px):
    phix, ctx = px
    n = 32
    v = np.zeros(n * n)
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [1.0, 1.0, 1.0], None, v, 1e-3,
                          [(1, 1.0)], 1e-10, "DF64", rho_re=8.0 * n * n)
    assert np.all(res[0] == 0.0)
    w = np.random.default_rng(0).standard_normal(n * n)
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [1.0, 1.0, 1.0], None, w, 0.0,
                          [(0, 1.0), (3, 1.0)], 1e-10, "DF64")
    assert np.allclose(res[0], w, rtol=0, atol=0) and np.allclose(res[1], w / 6.0, rtol=1e-15)


def test_invalid_arguments_and_nonconvergence(px):
    phix, ctx = px
    n = 16
    vd = dev(np.ones(n * n))
    out = torch.empty_like(vd)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [1.0, 0.0, 0.0])
    o = phix.phix_opts_default(rho_re=8.0 * n * n)
    st = phix.phix_phi_action(ctx, op, 1e-2, vd, [9], [1.0], [out], 1e-10, phix.PHIX_LEJA, o, check=False)
    assert st.status == phix.PHIX_EINVAL
    bad = phix.make_jop(7, n, n, [1.0])
    st = phix.phix_phi_action(ctx, bad, 1e-2, vd, [1], [1.0], [out], 1e-10, phix.PHIX_LEJA, o, check=False)
    assert st.status == phix.PHIX_EINVAL
    gs = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [1e-3, 1e-3, 0.04, 0.06], None)
    st = phix.phix_phi_action(ctx, gs, 1e-2, vd, [1], [1.0], [out], 1e-10, phix.PHIX_LEJA, o, check=False)
    assert st.status == phix.PHIX_EINVAL
    st = phix.phix_phi_action(ctx, op, 1e-2, vd, [1], [1.0], [vd], 1e-10, phix.PHIX_LEJA, o, check=False)
    assert st.status == phix.PHIX_EINVAL
    o2 = phix.phix_opts_default(rho_re=8.0 * n * n, m_max=4)
    w = dev(np.random.default_rng(1).standard_normal(n * n))
    st = phix.phix_phi_action(ctx, op, 1e-2, w, [1], [1.0], [out], 1e-14, phix.PHIX_LEJA, o2, check=False)
    assert st.status == phix.PHIX_ENOTCONV and st.iters == 4
    assert "converge" in phix.phix_last_error(ctx)
    # the context stays usable
    st = phix.phix_phi_action(ctx, op, 1e-2, w, [1], [1.0], [out], 1e-10, phix.PHIX_LEJA, o)
    assert st.status == 0


@pytest.mark.parametrize("prec", PRECS)
def test_chain_past_its_truncated_table_reruns_with_full_table(px, prec):
    """Coefficient tables are sized to about twice the predicted chain length.
    With m_min far above that prediction the chain reaches the end of its
    table unconverged; the call then repeats itself once with full tables and
    must agree with the oracle run under the same m_min."""
    phix, ctx = px
    n = 48
    p = synth.advdiff_params(n)
    v = synth.advdiff_gaussian(n)
    rho = 8.0 * p["D"] * n * n
    h = 10.0 / rho  # h * gamma = 3: the prediction is a few dozen iterations
    outs = [(1, 1.0), (2, 1.0)]
    tol = 1e-10
    m_min = 150
    res, st = _run_action(phix, ctx, phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]], None, v, h, outs,
                          tol, prec, rho_re=rho, m_min=m_min)
    op = AdvDiff(n, p["D"], p["ax"], p["ay"])
    ref, info = leja.leja_phi(op.jv, v, h, -rho, 0.0, outs, tol, m_min=m_min)
    assert st.status == 0 and info["status"] == 0
    assert st.iters == info["iters"] == m_min
    for r, o in zip(res, ref):
        assert rel(r, o) <= 1e-10


@pytest.mark.parametrize("n", [96, 90, 91])
@pytest.mark.parametrize("kind", ["advdiff", "grayscott", "burgers"])
@pytest.mark.parametrize("prec", ["FP64", "DF64", "FP32_JV", "FP32"])
def test_persistent_chain_equals_graph_chain(px, kind, prec, n):
    """The whole Newton pass in one cooperative launch (grid barrier per
    iteration, every block taking the stop decision) against one launch per
    iteration in a conditional graph: the pointwise Newton updates are the
    same code, so with the same iteration count the outputs are identical.
    n = 90: ragged tiles; 91: odd rows (one point per thread)."""
    phix, ctx = px
    if kind == "advdiff":
        p = synth.advdiff_params(n)
        op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
        v = dev(synth.advdiff_gaussian(n))
        h, kw = p["h"], dict(rho_re=8.0 * p["D"] * n * n)
    elif kind == "grayscott":
        prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=30.0)
        st = dev(synth.grayscott_state(n, seed=6, patch=24))
        op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]], st)
        v = dev(np.random.default_rng(3).standard_normal(2 * n * n))
        h, kw = prm["h"], {}
    else:
        prm = synth.burgers_params(n, mult=10.0)
        u = synth.burgers_state(n, seed=6)
        op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [prm["nu"]], dev(u))
        v = dev(np.random.default_rng(3).standard_normal(n * n))
        h, kw = prm["h"], dict(rho_im=2.0 * n * float(np.abs(u).max()))
    ls, ss = [0, 1, 1], [1.0, 0.5, 1.0]
    res = {}
    for chain in (phix.PHIX_CHAIN_PERSISTENT, phix.PHIX_CHAIN_GRAPH):
        out = [torch.empty_like(v) for _ in ls]
        o = phix.phix_opts_default(prec=_prec(phix, prec), chain=chain, **kw)
        st = phix.phix_phi_action(ctx, op, h, v, ls, ss, out, 1e-10, phix.PHIX_LEJA, o)
        res[chain] = (out, st)
    (a, sa), (b, sb) = res[phix.PHIX_CHAIN_PERSISTENT], res[phix.PHIX_CHAIN_GRAPH]
    assert sa.iters == sb.iters and sa.substeps == sb.substeps
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # a persistent pass is one launch; the graph's passes launch once per iteration
    assert sa.launches < sb.launches
