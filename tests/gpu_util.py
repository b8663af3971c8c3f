"""Helpers of the GPU parity tests (device arrays via torch, comparisons)."""
import numpy as np


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def parity_tol(same_iters, tol, base=1e-10):
    """Same iteration count: rounding-level agreement (base).  A stop decision
    that flipped by one iteration moves the result by at most ~tol."""
    return base if same_iters else max(base, 10.0 * tol)
