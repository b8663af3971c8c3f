"""High-precision phi-function reference for the oracle pins (mpmath)."""
import mpmath as mp


def phi_mp(l, z):
    """phi_l(z) at 50+ digits: the series sum_k z^k/(k+l)! for |z| <= 10, the
    closed form (e^z - sum_{k<l} z^k/k!) / z^l beyond (no cancellation there
    at this precision)."""
    with mp.workdps(80):
        z = mp.mpmathify(z)
        if abs(z) > 10:
            s = mp.e ** z
            for k in range(l):
                s -= z ** k / mp.factorial(k)
            return s / z ** l
        s = mp.mpf(0)
        term = 1 / mp.factorial(l)
        k = 0
        while abs(term) > mp.mpf(10) ** -70 or k < 5:
            s += term
            term = term * z / (k + l + 1)
            k += 1
        return s
