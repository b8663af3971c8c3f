"""Pins for oracle.phi (Sec. 1 definition of the phi-functions)."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle.phi import phi_scalar

mp = pytest.importorskip("mpmath")
from mp_ref import phi_mp  # noqa: E402


ZS = [0.0, 1e-12, -1e-6, 0.3, -0.999, 1.0, -1.0, 2.5, -7.0, -40.0, -300.0, 12.0,
      0.5 + 0.5j, -3.0 + 4.0j, -50.0 + 20.0j, 1e-9j]


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("z", ZS)
def test_phi_against_mpmath(l, z):
    ref = complex(phi_mp(l, z))
    got = complex(phi_scalar(l, z))
    assert abs(got - ref) <= 1e-14 * max(abs(ref), 1e-300) + 1e-300


@pytest.mark.parametrize("l", range(7))
def test_phi_at_zero_is_inverse_factorial(l):
    assert phi_scalar(l, 0.0) == pytest.approx(1.0 / math.factorial(l), rel=1e-16)


@pytest.mark.parametrize("z", [-0.7, 0.9, -12.0, 3.0 - 2.0j])
def test_phi1_doubling_identity(z):
    # phi_1(2z) = phi_1(z) (e^z + 1) / 2
    lhs = phi_scalar(1, 2 * z)
    rhs = phi_scalar(1, z) * (np.exp(z) + 1) / 2
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("z", [-0.3, -25.0, 4.0])
def test_phi_from_small_expm(l, z):
    # exp of [[z, 1, 0..], [0, 0, 1, ..], ..., [0, ..., 0]] ((l+1)x(l+1)): entry (0, l) = phi_l(z)
    M = np.zeros((l + 1, l + 1))
    M[0, 0] = z
    for i in range(l):
        M[i, i + 1] = 1.0
    E = scipy.linalg.expm(M)
    assert E[0, l] == pytest.approx(phi_scalar(l, z), rel=1e-12)


def test_recurrence_holds():
    for l in range(5):
        for z in [-3.3, 2.2, -0.5 + 1j]:
            lhs = phi_scalar(l + 1, z)
            rhs = (phi_scalar(l, z) - 1.0 / math.factorial(l)) / z
            assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
