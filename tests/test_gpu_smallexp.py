"""GPU check of the Krylov method's small exponential (phix_small_expm,
exp(tau T) e_1 of a tridiagonal Hessenberg matrix) against scipy.linalg.expm
on diffusion-like, non-normal and strongly non-normal matrices; both code
paths (Chebyshev, shifted Taylor) are exercised.  Accuracy is normwise, like
a dense expm: ||F - exp(tau T) e_1|| <= 1e-13 ||exp(tau T)||_2."""
import numpy as np
import pytest
import scipy.linalg

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


def _case(rng, n, skew_scale):
    d = -rng.uniform(0, 200, n)
    e = rng.uniform(0, 80, n - 1)
    sk = rng.uniform(-1, 1, n - 1) * skew_scale
    return d, e + sk, e - sk


@pytest.mark.parametrize("skew", [0.0, 0.1, 1.0, 5.0, 40.0, 200.0])
def test_small_expm_vs_scipy(px, skew):
    phix, ctx = px
    rng = np.random.default_rng(int(skew * 10) + 1)
    modes = set()
    for trial in range(12):
        n = int(rng.integers(2, 130))
        d, u, l = _case(rng, n, skew)
        tau = float(rng.choice([0.01, 0.2, 1.0]))
        T = np.diag(d) + np.diag(u, 1) + np.diag(l, -1)
        E = scipy.linalg.expm(tau * T)
        ref = E[:, 0]
        dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        mode = phix.phix_small_expm(ctx, dev(d), dev(u), dev(l), tau, F)
        modes.add(mode)
        got = F.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(E, 2)
        # double-float recurrences (~2^-47 per operation, up to 30 S Taylor terms):
        # normwise 1e-12, two orders below the tolerances the result serves
        assert err <= 1e-12, (n, tau, mode, err)
    print("skew", skew, "paths", sorted(modes))


def test_small_expm_scalar_and_zero(px):
    phix, ctx = px
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    phix.phix_small_expm(ctx, dev([-2.5]), dev([0.0]), dev([0.0]), 1.5, F)
    assert F.item() == pytest.approx(np.exp(-3.75), rel=1e-15)
    F = torch.empty(4, dtype=torch.float64, device="cuda")
    z = dev(np.zeros(4))
    phix.phix_small_expm(ctx, z, dev(np.zeros(3)), dev(np.zeros(3)), 1.0, F)
    assert F.cpu().numpy().tolist() == [1.0, 0.0, 0.0, 0.0]
