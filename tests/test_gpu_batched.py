"""GPU parity of the batched persistent launch (C-ABI) against the oracle's
Leja action per problem and the FFT-exact result."""
import numpy as np
import pytest

import synth
from gpu_util import rel, parity_tol
from oracle import exact, leja
from oracle.operators import AdvDiff

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


def _bounds(nx, ny, D, ax, ay):
    # exact real extent of the centred periodic advection-diffusion spectrum
    # (Gershgorin / Fourier symbol) and the imaginary bound |ax| nx + |ay| ny
    return 4.0 * D * (nx * nx + ny * ny), abs(ax) * nx + abs(ay) * ny


def _small_batch(seed=0, count=40):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        nx = int(rng.integers(8, 80))
        ny = int(rng.integers(8, 80))
        D = float(rng.uniform(0.1, 1.0))
        heavy = i % 5 == 0
        ax, ay = (rng.uniform(0, 10, 2) if heavy else rng.uniform(-1, 1, 2) * D * min(nx, ny) / 2)
        mult = float(np.exp(rng.uniform(np.log(10), np.log(200))))
        h = mult / (4.0 * D * max(nx, ny) ** 2)
        rre, rim = _bounds(nx, ny, D, ax, ay)
        probs.append(dict(nx=nx, ny=ny, D=D, ax=float(ax), ay=float(ay), h=h, rho_re=rre, rho_im=rim,
                          v=rng.standard_normal(nx * ny)))
    return probs


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_batched_vs_oracle_small(px, prec):
    phix, ctx = px
    probs = _small_batch()
    ls = [0, 1, 2]
    tol = 1e-9
    dev = []
    for q in probs:
        v = torch.tensor(q["v"], dtype=torch.float64, device="cuda")
        dev.append(dict(q, v=v, out=[torch.empty_like(v) for _ in ls]))
    o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec))
    st, per = phix.phix_phi_action_batched(ctx, dev, ls, tol, o)
    assert all(s == 0 for s in per)
    nsub = 0
    for q, d in zip(probs, dev):
        op = AdvDiff(q["nx"], q["D"], q["ax"], q["ay"], ny=q["ny"])
        ref, info = leja.leja_phi(op.jv, q["v"], q["h"], -q["rho_re"], 0.0, [(l, 1.0) for l in ls], tol,
                                  rho_im=q["rho_im"], iota_cap=4.0)
        assert info["status"] == 0
        nsub += info["substeps"] > 1
        for k, l in enumerate(ls):
            got = d["out"][k].cpu().numpy()
            assert rel(got, ref[k]) <= parity_tol(False, tol), (q["nx"], q["ny"], l, rel(got, ref[k]))
            if q["nx"] == q["ny"]:
                ex = exact.advdiff_phi_fft(q["nx"], q["D"], q["ax"], q["ay"], q["h"], q["v"], l)
                assert rel(got, ex) <= 100 * tol
    assert nsub >= 4  # the advection-heavy problems took the substep path


def test_batched_fp32_jv_error(px):
    phix, ctx = px
    probs = _small_batch(seed=1, count=16)
    dev = []
    for q in probs:
        v = torch.tensor(q["v"], dtype=torch.float64, device="cuda")
        dev.append(dict(q, v=v, out=[torch.empty_like(v)]))
    o = phix.phix_opts_default(prec=phix.PHIX_FP32_JV)
    st, per = phix.phix_phi_action_batched(ctx, dev, [1], 1e-7, o)
    worst = 0.0
    for q, d in zip(probs, dev):
        op = AdvDiff(q["nx"], q["D"], q["ax"], q["ay"], ny=q["ny"])
        ref, _ = leja.leja_phi(op.jv, q["v"], q["h"], -q["rho_re"], 0.0, [(1, 1.0)], 1e-10,
                               rho_im=q["rho_im"], iota_cap=4.0)
        worst = max(worst, rel(d["out"][0].cpu().numpy(), ref[0]))
    # float32 stencil products in every Newton step of every substep (these
    # advection-heavy problems take up to ~390 substeps); measured 2.1e-6
    print("FP32_JV batched worst rel err", worst)
    assert worst <= 1e-5


def test_batched_full_workload_sampled(px):
    """The 4096-problem workload (sides log-uniform 32..512, D ~ U(0.1, 1),
    a ~ U(0, 50)^2, h = 10..200x explicit, Gaussian v), one launch, double-float;
    a seeded sample of 24 problems checked against the FFT-exact result."""
    phix, ctx = px
    spec = synth.batched_problems(4096, seed=0)
    dev = []
    total = 0
    for q in spec:
        n = q["n"]
        v = torch.tensor(synth.random_vector(n * n, q["seed_v"]), dtype=torch.float64, device="cuda")
        rre, rim = _bounds(n, n, q["D"], q["ax"], q["ay"])
        dev.append(dict(nx=n, ny=n, D=q["D"], ax=q["ax"], ay=q["ay"], h=q["h"], rho_re=rre, rho_im=rim, v=v,
                        out=[torch.empty_like(v) for _ in range(3)]))
        total += n * n
    st, per = phix.phix_phi_action_batched(ctx, dev, [0, 1, 2], 1e-8, phix.phix_opts_default())
    print("unknowns", total, "stats", st.as_dict())
    assert all(s == 0 for s in per)
    rng = np.random.default_rng(7)
    for i in rng.choice(len(spec), 24, replace=False):
        q, d = spec[i], dev[i]
        vv = d["v"].cpu().numpy()
        for k in range(3):
            ex = exact.advdiff_phi_fft(q["n"], q["D"], q["ax"], q["ay"], q["h"], vv, k)
            assert rel(d["out"][k].cpu().numpy(), ex) <= 1e-6, (i, q["n"], k)
