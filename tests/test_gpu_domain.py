"""The domain-decomposed Newton-Leja pass on the GPU: libphix's block
kernels (phix_block_newton, phix_block_faces, phix_block_start) driven by
paper_2211_08948_gb300.domain with every block in this process (LocalComm,
blocks run one after another on one stream), against the unsplit oracle
element by element.  (Ranks on several GPUs exchange through TorchComm; this
pool gives one GPU per run, and the multi-rank logic is tested on gloo CPU
ranks in test_domain.py.)"""
import numpy as np
import pytest

import synth
from domain_util import oracle_pass
from oracle import leja
from oracle.operators import AdvDiff, GrayScott, Burgers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    from paper_2211_08948_gb300 import build, phix, domain
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ctx = phix.phix_create(torch.cuda.current_stream())
    yield phix, ctx, domain, domain.GpuBackend(phix, ctx, torch)
    phix.phix_destroy(ctx)


@pytest.mark.parametrize("px,py", [(1, 1), (2, 2), (3, 2)])
@pytest.mark.parametrize("lag", [0, 1])
def test_gpu_blocks_advdiff_vs_oracle(gpu, px, py, lag):
    phix, ctx, domain, be = gpu
    n = 48
    p = synth.advdiff_params(n, mult=20.0)
    v = synth.advdiff_gaussian(n)
    dec = domain.Decomposition(n, n, px, py, 1)
    op = domain.BlockedOperator(be, domain.LocalComm(), dec, phix.PHIX_OP_ADVDIFF, [p["D"], p["ax"], p["ay"]])
    outs = [(0, 1.0), (1, 1.0), (3, 0.5)]
    rho = 8.0 * p["D"] * n * n
    res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in range(dec.count)}, p["h"], outs, 1e-10,
                                interval=(-rho, 0.0), lag=lag)
    ref, m = oracle_pass(AdvDiff(n, p["D"], p["ax"], p["ay"]).jv, v, p["h"], -rho, 0.0, outs, 1e-10,
                         iters_extra=lag)
    assert info["status"] == 0 and info["iters"] == m
    for k in range(len(outs)):
        got = dec.assemble({r: res[r][k] for r in res})
        assert np.linalg.norm(got - ref[k]) <= 1e-12 * np.linalg.norm(ref[k])


@pytest.mark.parametrize("kind", ["grayscott", "burgers"])
def test_gpu_blocks_nonlinear_power_iteration_vs_oracle(gpu, kind):
    phix, ctx, domain, be = gpu
    n = 40
    if kind == "grayscott":
        prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=20.0)
        state = synth.grayscott_state(n, seed=3, patch=12)
        params, kd, nc = [prm["Du"], prm["Dv"], prm["F"], prm["k"]], phix.PHIX_OP_GRAYSCOTT, 2
        oop = GrayScott(n, *params, state=state)
    else:
        prm = synth.burgers_params(n, nu=2e-2, mult=5.0)
        state = synth.burgers_state(n, seed=3)
        params, kd, nc = [prm["nu"]], phix.PHIX_OP_BURGERS, 1
        oop = Burgers(n, prm["nu"], state=state)
    dec = domain.Decomposition(n, n, 3, 2, nc)
    op = domain.BlockedOperator(be, domain.LocalComm(), dec, kd, params,
                                {r: dec.interior(r, state) for r in range(dec.count)})
    v = np.random.default_rng(8).standard_normal(nc * n * n)
    outs = [(1, 0.5), (1, 1.0)]
    res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in range(dec.count)}, prm["h"], outs, 1e-10,
                                lag=1)
    rho, mv = leja.power_iteration(oop.jv, v.size)
    assert info["power_mv"] == mv
    ref, m = oracle_pass(oop.jv, v, prm["h"], -1.2 * rho, 0.0, outs, 1e-10, iters_extra=1)
    assert info["iters"] == m
    for k in range(len(outs)):
        got = dec.assemble({r: res[r][k] for r in res})
        assert np.linalg.norm(got - ref[k]) <= 1e-11 * np.linalg.norm(ref[k])


def test_gpu_blocks_match_single_domain_entry_point(gpu):
    """A 2 x 2 blocked pass (lag 0) gives phix_phi_action's float64 result on
    the same interval to rounding."""
    phix, ctx, domain, be = gpu
    n = 64
    prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=20.0)
    state = synth.grayscott_state(n, seed=4, patch=16)
    params = [prm["Du"], prm["Dv"], prm["F"], prm["k"]]
    v = np.random.default_rng(2).standard_normal(2 * n * n)
    rho = 8.0 * 2e-3 * n * n * 2
    dec = domain.Decomposition(n, n, 2, 2, 2)
    op = domain.BlockedOperator(be, domain.LocalComm(), dec, phix.PHIX_OP_GRAYSCOTT, params,
                                {r: dec.interior(r, state) for r in range(dec.count)})
    res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in range(dec.count)}, prm["h"], [(1, 1.0)], 1e-10,
                                interval=(-rho, 0.0), lag=0)
    sd = torch.tensor(state, dtype=torch.float64, device="cuda")
    vd = torch.tensor(v, dtype=torch.float64, device="cuda")
    out = torch.empty_like(vd)
    jop = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, params, sd)
    st = phix.phix_phi_action(ctx, jop, prm["h"], vd, [1], [1.0], [out], 1e-10, phix.PHIX_LEJA,
                              phix.phix_opts_default(prec=phix.PHIX_FP64, rho_re=rho))
    assert st.iters == info["iters"]
    got = dec.assemble({r: res[r][0] for r in res})
    ref = out.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
