"""Exact references for phi-function actions (no iteration, no tolerance).

* FFT diagonalisation of the periodic constant-coefficient advection-
  diffusion operator: each Fourier mode is an eigenvector, so
  phi_l(s h J) v is phi_l(s h lambda) applied mode by mode.
* Dense augmented-matrix exponential, the Theorem of Sec. 2.1:
  for A (N x N), B = [b_p, ..., b_1], K the p x p shift, and
  v = [b_0; e_p], the first N entries of exp(A~) v, A~ = [[A, B], [0, K]],
  equal sum_{j=0}^{p} phi_j(A) b_j.  scipy.linalg.expm is the library
  primitive for exp.
"""
import numpy as np
import scipy.linalg


def advdiff_eigenvalues(n, D, ax, ay):
    """Eigenvalue of the centred-difference operator
    D lap + ax d/dx + ay d/dy on the Fourier mode exp(2 pi i (kx x + ky y))
    (x along axis 1), laid out like numpy.fft.fft2 output [ky, kx]."""
    dx = 1.0 / n
    k = np.fft.fftfreq(n, d=1.0 / n)
    th = 2.0 * np.pi * k / n
    thy, thx = np.meshgrid(th, th, indexing="ij")
    lam = D * (2.0 * np.cos(thx) + 2.0 * np.cos(thy) - 4.0) / (dx * dx) \
        + 1j * (ax * np.sin(thx) + ay * np.sin(thy)) / dx
    return lam


def advdiff_phi_fft(n, D, ax, ay, t, v, l):
    """phi_l(t J) v for the periodic advection-diffusion J (exact up to FFT rounding)."""
    from .phi import phi
    lam = advdiff_eigenvalues(n, D, ax, ay)
    vh = np.fft.fft2(np.asarray(v, dtype=np.float64).reshape(n, n))
    out = np.fft.ifft2(vh * phi(l, t * lam))
    return out.real.reshape(-1)


def dense_matrix(jv, N):
    """Assemble the N x N matrix of a linear map given as a matvec (tiny N only)."""
    M = np.empty((N, N))
    e = np.zeros(N)
    for i in range(N):
        e[i] = 1.0
        M[:, i] = jv(e)
        e[i] = 0.0
    return M


def augmented_phi_sum(A, bs):
    """sum_{j=0}^{p} phi_j(A) b_j via the Theorem of Sec. 2.1 (bs = [b_0, ..., b_p],
    None meaning a zero vector)."""
    N = A.shape[0]
    p = len(bs) - 1
    bs = [np.zeros(N) if b is None else np.asarray(b, dtype=np.float64) for b in bs]
    if p == 0:
        return scipy.linalg.expm(A) @ bs[0]
    At = np.zeros((N + p, N + p))
    At[:N, :N] = A
    for i in range(p):                 # columns of B are b_p, ..., b_1
        At[:N, N + i] = bs[p - i]
    for i in range(p - 1):             # K = [[0, I_{p-1}], [0, 0]]
        At[N + i, N + i + 1] = 1.0
    v = np.zeros(N + p)
    v[:N] = bs[0]
    v[N + p - 1] = 1.0                 # e_p
    return (scipy.linalg.expm(At) @ v)[:N]


def dense_phi(A, l, v):
    """phi_l(A) v by the augmented theorem with b_l = v and all other b_j = 0."""
    bs = [None] * (l + 1)
    bs[l] = v
    return augmented_phi_sum(A, bs)
