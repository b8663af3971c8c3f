"""GPU check of phix_phi_action_noalloc, the entry point for callers that
cannot allocate device memory (its scratch is a fixed device array of the
library).  Called twice in a row through the C-ABI, it must give what
phix_phi_action gives on the same inputs, in every iteration precision, on
the three operators, at the longest chain it accepts (m_max = power_max_it =
PHIX_NOALLOC_MMAX) and on a zero operator; one case is also checked against
the CPU oracle.  This file is collected last."""
import numpy as np
import pytest

import synth

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


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def problem(phix, case):
    """(op, h, v, opts keyword arguments, l, scale, host state or None)."""
    if case == "advdiff":
        n = 64
        p = synth.advdiff_params(n)
        op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
        return op, p["h"], dev(synth.advdiff_gaussian(n)), dict(rho_re=8.0 * p["D"] * n * n), \
            [0, 1, 2, 3], [1.0] * 4, None
    if case == "grayscott":
        n = 96
        prm = synth.grayscott_params(n)
        prm["Du"] *= 64
        prm["Dv"] *= 64
        st = synth.grayscott_state(n, seed=3, patch=24)
        op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]], dev(st))
        h = 30.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
        v = dev(np.random.default_rng(4).standard_normal(2 * n * n))
        return op, h, v, {}, [1, 1], [0.5, 1.0], st   # power iteration inside the call
    n = 80   # Burgers
    prm = synth.burgers_params(n)
    st = synth.burgers_state(n, seed=5)
    op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [prm["nu"]], dev(st))
    v = dev(np.random.default_rng(6).standard_normal(n * n))
    # h small enough for one pass without substeps (h rho_im <= iota_cap)
    return op, 0.01, v, dict(rho_im=2.0 * n * float(np.abs(st).max())), [1], [1.0], st


def check_twice(phix, ctx, op, h, v, ls, ss, opts, tol, bound, same_iters=True):
    ref = [torch.empty_like(v) for _ in ls]
    st_ref = phix.phix_phi_action(ctx, op, h, v, ls, ss, ref, tol, phix.PHIX_LEJA, opts)
    for call in range(2):
        got = [torch.full_like(v, float("nan")) for _ in ls]
        st = phix.phix_phi_action_noalloc(op, h, v, ls, ss, got, tol, opts, torch.cuda.current_stream())
        assert st.status == phix.PHIX_OK, call
        if same_iters:
            assert st.iters == st_ref.iters and st.power_mv == st_ref.power_mv, (call, st.iters, st_ref.iters)
        else:
            assert abs(st.iters - st_ref.iters) <= 3, (call, st.iters, st_ref.iters)
        for g, r in zip(got, ref):
            assert rel(g, r) <= bound, (call, rel(g, r))
    return ref


@pytest.mark.parametrize("case", ["advdiff", "grayscott", "burgers"])
@pytest.mark.parametrize("prec", ["DF64", "FP64", "FP32_JV", "FP32"])
def test_noalloc_matches_context_entry_point_twice(px, case, prec):
    phix, ctx = px
    op, h, v, kw, ls, ss, _ = problem(phix, case)
    opts = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), **kw)
    # The two entry points launch different grids, so their norm reductions
    # sum in different orders.  The Newton updates are pointwise and identical;
    # where the interval comes from a float32 power iteration, its estimate
    # differs in the float32 rounding of those sums, the coefficient tables
    # differ with it, and the results differ at the float32 rounding level
    # (the float32 iterations' own error against float64 is ~1e-5).
    f32_power = prec in ("FP32", "FP32_JV") and "rho_re" not in kw
    check_twice(phix, ctx, op, h, v, ls, ss, opts, 1e-10, 1e-4 if f32_power else 1e-10,
                same_iters=not f32_power)


def test_noalloc_longest_chain_and_power_limit(px):
    """m_max = power_max_it = PHIX_NOALLOC_MMAX (the largest parameter block
    the static staging holds) on a small grid."""
    phix, ctx = px
    op, h, v, kw, ls, ss, _ = problem(phix, "grayscott")
    opts = phix.phix_opts_default(m_max=phix.PHIX_NOALLOC_MMAX, power_max_it=phix.PHIX_NOALLOC_MMAX,
                                  power_rel=1e-6)
    check_twice(phix, ctx, op, h, v, ls, ss, opts, 1e-12, 1e-10)


def test_noalloc_against_oracle(px):
    """One vertical pass checked against the CPU oracle's Newton-Leja result."""
    from oracle import leja
    from oracle.operators import AdvDiff
    phix, ctx = px
    n = 64
    p = synth.advdiff_params(n)
    rho = 8.0 * p["D"] * n * n
    v = synth.advdiff_gaussian(n)
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
    got = [torch.empty(n * n, dtype=torch.float64, device="cuda") for _ in range(4)]
    st = phix.phix_phi_action_noalloc(op, p["h"], dev(v), [0, 1, 2, 3], [1.0] * 4, got, 1e-10,
                                      phix.phix_opts_default(rho_re=rho), torch.cuda.current_stream())
    assert st.status == phix.PHIX_OK
    ref, info = leja.leja_phi(AdvDiff(n, p["D"], p["ax"], p["ay"]).jv, v, p["h"], -rho, 0.0,
                              [(l, 1.0) for l in range(4)], 1e-10, m_max=500)
    assert info["iters"] == st.iters
    for l in range(4):
        g = got[l].cpu().numpy()
        assert np.linalg.norm(g - ref[l]) <= 1e-10 * np.linalg.norm(ref[l]), l


def test_noalloc_zero_operator_gives_v_over_factorial(px):
    phix, ctx = px
    n = 32
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [0.0, 0.0, 0.0])
    v = dev(np.random.default_rng(7).standard_normal(n * n))
    ls, ss = [0, 1, 3], [1.0, 1.0, 1.0]
    ref = [torch.empty_like(v) for _ in ls]
    phix.phix_phi_action(ctx, op, 0.1, v, ls, ss, ref, 1e-10, phix.PHIX_LEJA, phix.phix_opts_default())
    for call in range(2):
        got = [torch.full_like(v, float("nan")) for _ in ls]
        st = phix.phix_phi_action_noalloc(op, 0.1, v, ls, ss, got, 1e-10, None, torch.cuda.current_stream())
        assert st.status == phix.PHIX_OK
        for g, r, l in zip(got, ref, ls):
            assert torch.equal(g, r)
            assert rel(g, v / [1.0, 1.0, 2.0, 6.0][l]) <= 1e-15


def test_noalloc_rejects_problem_beyond_scratch(px):
    phix, _ = px
    n = 2048   # 2048^2 x 2 species x 8 B x (2 + 1) vectors > 32 MiB
    state = torch.ones(2 * n * n, dtype=torch.float64, device="cuda")
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [2e-5, 1e-5, 0.04, 0.06], state)
    v = torch.ones(2 * n * n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    st = phix.phix_phi_action_noalloc(op, 1.0, v, [1], [1.0], [out], 1e-8, None, None, check=False)
    assert st.status == phix.PHIX_ETOOBIG
