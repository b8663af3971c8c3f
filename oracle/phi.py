"""Scalar phi-functions, Sec. 1 of the paper.

phi_0(z) = exp(z),  phi_{l+1}(z) = (phi_l(z) - 1/l!) / z.

The paper prints the recurrence with "l >= 1"; it is read as l >= 0 so
that phi_1(z) = (e^z - 1)/z (the standard definition; otherwise phi_1 is
undefined).  Equivalently phi_l(z) = sum_{k>=0} z^k / (k+l)!, which is
used for |z| < l + 1 where the recurrence cancels.
"""
import math
import numpy as np

_SERIES_TERMS = 80  # |z| < l+1 <= 8: term 80 is below 8^80/80! ~ 1e-47


def phi_scalar(l, z):
    """phi_l(z) for a scalar real or complex z (float64 / complex128)."""
    l = int(l)
    if l < 0:
        raise ValueError("l must be >= 0")
    z = complex(z) if isinstance(z, complex) else float(z)
    if l == 0:
        return np.exp(z) if isinstance(z, complex) else (math.exp(z) if z < 709 else float("inf"))
    # the recurrence cancels when |z| is small against l: use the series there
    if abs(z) < l + 1:
        # phi_l(z) = sum_k z^k/(k+l)!  (series form of the Sec. 1 definition)
        s = 0.0
        term = 1.0 / math.factorial(l)
        for k in range(_SERIES_TERMS):
            s += term
            term = term * z / (k + l + 1)
        return s
    # recurrence of Sec. 1, l >= 0 reading
    p = np.exp(z) if isinstance(z, complex) else math.exp(z) if z < 700 else float("inf")
    for j in range(l):
        p = (p - 1.0 / math.factorial(j)) / z
    return p


def phi(l, z):
    """Vectorised phi_l over an array z."""
    z = np.asarray(z)
    out = np.empty(z.shape, dtype=np.complex128 if np.iscomplexobj(z) else np.float64)
    for idx, zz in np.ndenumerate(z):
        out[idx] = phi_scalar(l, zz)
    return out
