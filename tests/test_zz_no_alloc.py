"""GPU check of phix_phi_action_noalloc, the entry point for callers that
cannot allocate device memory (its scratch is a fixed device array of the
library).  Called twice in a row through the C-ABI, it must give what
phix_phi_action gives on the same inputs.  This file is collected last."""
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


@pytest.mark.parametrize("case", ["advdiff", "grayscott"])
def test_noalloc_matches_context_entry_point_twice(px, case):
    phix, ctx = px
    if case == "advdiff":
        n = 64
        p = synth.advdiff_params(n)
        v = dev(synth.advdiff_gaussian(n))
        op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
        h = p["h"]
        opts = phix.phix_opts_default(rho_re=8.0 * p["D"] * n * n)
        ls, ss = [0, 1, 2, 3], [1.0] * 4
    else:
        n = 96
        prm = synth.grayscott_params(n)
        prm["Du"] *= 64
        prm["Dv"] *= 64
        state = dev(synth.grayscott_state(n, seed=3, patch=24))
        op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]], state)
        v = dev(np.random.default_rng(4).standard_normal(2 * n * n))
        h = 30.0 * (1.0 / n) ** 2 / (4 * prm["Du"])
        opts = phix.phix_opts_default()   # power iteration inside the call
        ls, ss = [1, 1], [0.5, 1.0]
    tol = 1e-10
    ref = [torch.empty_like(v) for _ in ls]
    st_ref = phix.phix_phi_action(ctx, op, h, v, ls, ss, ref, tol, phix.PHIX_LEJA, opts)
    for call in range(2):
        got = [torch.full_like(v, float("nan")) for _ in ls]
        st = phix.phix_phi_action_noalloc(op, h, v, ls, ss, got, tol, opts, torch.cuda.current_stream())
        assert st.status == phix.PHIX_OK, call
        assert st.iters == st_ref.iters and st.power_mv == st_ref.power_mv
        for g, r in zip(got, ref):
            assert rel(g, r) <= 1e-10, (call, rel(g, r))


def test_noalloc_rejects_problem_beyond_scratch(px):
    phix, _ = px
    n = 2048   # 2048^2 x 2 species x 8 B x (2 + 1) vectors > 32 MiB
    state = torch.ones(2 * n * n, dtype=torch.float64, device="cuda")
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [2e-5, 1e-5, 0.04, 0.06], state)
    v = torch.ones(2 * n * n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    st = phix.phix_phi_action_noalloc(op, 1.0, v, [1], [1.0], [out], 1e-8, None, None, check=False)
    assert st.status == phix.PHIX_ETOOBIG
