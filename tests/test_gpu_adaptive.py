"""phix_integrate (automatic step-size control, Sec. 2.3) through the C-ABI
against the oracle's adaptive integrator: the same accepted and rejected
steps, the same step sizes (to the relative size of the error estimates'
rounding), the same final state."""
import math

import numpy as np
import pytest

import synth
from gpu_util import rel
from oracle import adaptive
from oracle.operators import GrayScott

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


SCHEMES = {"exprb43": 0, "epirk4s3": 1, "epirk4s3a": 2, "exprb53s3": 3, "epirk5p1": 4}


@pytest.mark.parametrize("scheme,method,controller", [("exprb43", "leja", "cost"), ("exprb43", "leja", "traditional"),
                                                      ("epirk5p1", "kiops", "cost"), ("exprb53s3", "lekry", "cost")])
def test_integrate_vs_oracle(px, scheme, method, controller):
    phix, ctx = px
    n = 32
    prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=5.0)
    u0 = synth.grayscott_gaussian(n)
    T = 40.0 * prm["h"]
    tol = 1e-6
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    ud = torch.tensor(u0, dtype=torch.float64, device="cuda")
    meth = {"leja": phix.PHIX_LEJA, "kiops": phix.PHIX_KIOPS, "lekry": phix.PHIX_LEKRY}[method]
    ctl = phix.PHIX_CONTROL_COST if controller == "cost" else phix.PHIX_CONTROL_TRADITIONAL
    st, dts = phix.phix_integrate(ctx, SCHEMES[scheme], op, ud, T, 2.0 * prm["h"], tol, meth, ctl, iter_tol=1e-11,
                                  opts=phix.phix_opts_default(prec=phix.PHIX_FP64))
    u, info = adaptive.integrate(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0, T, 2.0 * prm["h"], tol,
                                 scheme=scheme, method=method, controller=controller, iter_tol=1e-11,
                                 kiops_kw=dict(m_init=16, m_max=64, m_step=8))
    print(scheme, method, controller, "gpu", st.accepted, st.rejected, "oracle", info["accepted"], info["rejected"])
    assert st.accepted == info["accepted"] and st.rejected == info["rejected"]
    assert st.t == pytest.approx(T, abs=1e-12 * T)
    assert np.allclose(dts, info["dts"], rtol=1e-6, atol=0)
    assert rel(ud.cpu().numpy(), u) <= 1e-8
    assert st.accepted >= 3
