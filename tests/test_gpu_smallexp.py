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


def _krylov_like(n, r, skew, seed):
    """Tridiagonal with the shape of a window-2 Hessenberg matrix of a
    diffusion-dominated Jacobian: diagonal spread over [-2r, 0], positive
    symmetric off-diagonals of size ~r/4, a skew part `skew` times that."""
    rng = np.random.default_rng(seed)
    d = -r * (1 + np.cos(np.linspace(0, np.pi, n))) * rng.uniform(0.9, 1.0, n)
    s = r / 2 * rng.uniform(0.3, 0.6, n - 1)
    k = skew * s * rng.uniform(-1, 1, n - 1)
    return d, s + k, s - k


@pytest.mark.parametrize("n,r,skew", [(41, 50, 1.0), (65, 100, 0.5), (65, 100, 1.0), (97, 200, 1.0),
                                      (129, 400, 1.0), (129, 400, 0.2)])
def test_small_expm_wide_spectrum_takes_chebyshev_segments(px, n, r, skew):
    """Field-of-values half-widths r ~ 70..550 with iota/r ~ 0.05..0.3 (the
    range of the Krylov method's tau Hbar on stiff diffusion-reaction
    problems): one Chebyshev expansion would amplify rounding by up to 2^16
    or more, so the expansion runs in segments exp(X/S)^S; the result stays
    within the normwise 1e-12 of scipy's dense expm."""
    phix, ctx = px
    d, u, l = _krylov_like(n, r, skew, n + int(r))
    T = np.diag(d) + np.diag(u, 1) + np.diag(l, -1)
    E = scipy.linalg.expm(T)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    mode = phix.phix_small_expm(ctx, dev(d), dev(u), dev(l), 1.0, F)
    got = F.cpu().numpy()
    err = np.linalg.norm(got - E[:, 0]) / np.linalg.norm(E, 2)
    assert mode == 0, "expected the Chebyshev path"
    assert err <= 1e-12, err
