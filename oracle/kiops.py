"""KIOPS-style Krylov evaluation of sum_j tau^j phi_j(tau A) b_j, Sec. 2.1.

What the paper fixes (Sec. 2.1): the linear combination is written as the
exponential of the augmented matrix A~ = [[A, B], [0, K]] (Theorem), the
exponential of A~ is projected on a Krylov subspace built by Arnoldi with
incomplete orthogonalisation ("as few as two" inner products per
iteration), the step is split into substeps, and the substep length and
the Krylov dimension are adapted from an error estimate.  The KIOPS paper
itself is not reproduced; the concrete rules below are this project's
reading, followed alike by this module and by the CUDA library:

* B and the tail are balanced by eta = 2^-ceil(log2 max_j ||b_j||_1):
  A~ uses eta*B, the start vector is [b_0; e_p / eta].
* window-2 incomplete orthogonalisation, classical Gram-Schmidt form:
  h_ij = <V_i, A~ V_j> for i in {j-1, j} on the unmodified product,
  then z = A~ V_j - sum_i h_ij V_i, h_{j+1,j} = ||z||.
* error estimate of the corrected Krylov approximation:
  F = exp(tau Hbar) e_1 with Hbar = [[H_m, 0], [h_{m+1,m} e_m^T, 0]],
  err = beta |F_{m+1}|, omega = (tau_end / tau) err / (tol beta).
* omega <= 1: accept w <- beta [V_m, v_{m+1}] F, t += tau,
  tau <- tau * clip(0.8 omega^(-1/m), 1, 2).
  omega > 1: if m < m_max extend the basis by m_step vectors, else
  tau <- tau * clip(0.8 omega^(-1/m), 0.1, 0.9) (same basis, new F).
* happy breakdown when h_{j+1,j} <= 1e-12 ||A~ V_j|| (exact subspace).
* substeps land exactly on every requested output time.
"""
import math
import numpy as np
import scipy.linalg

OK, ENOTCONV, ENAN = 0, 2, 3


def kiops(apply_A, bs, tau_out, tol, m_init=16, m_max=64, m_step=8, iop=2, max_substeps=10000):
    """Outputs w(tau) = sum_{j=0}^{p} tau^j phi_j(tau A) b_j for each tau in tau_out.

    apply_A: x -> A x on R^N.  bs = [b_0, ..., b_p] (None = zero vector).
    Returns (list of outputs ordered like tau_out, info dict).
    """
    p = len(bs) - 1
    N = next(len(b) for b in bs if b is not None)
    bs = [np.zeros(N) if b is None else np.asarray(b, dtype=np.float64) for b in bs]
    nb = max([np.sum(np.abs(b)) for b in bs[1:]], default=0.0)
    eta = 2.0 ** (-math.ceil(math.log2(nb))) if nb > 0 else 1.0

    def apply_aug(x):
        y = np.empty_like(x)
        y[:N] = apply_A(x[:N])
        for i in range(1, p + 1):          # B z = sum_i b_{p+1-i} z_i  (1-based z_i)
            y[:N] += eta * bs[p + 1 - i] * x[N + i - 1]
        y[N:N + p - 1] = x[N + 1:N + p]    # K z: shift up
        if p > 0:
            y[N + p - 1] = 0.0
        return y

    w = np.zeros(N + p)
    w[:N] = bs[0]
    if p > 0:
        w[N + p - 1] = 1.0 / eta
    times = sorted(set(float(t) for t in tau_out))
    tau_end = times[-1]
    results = {}
    info = dict(substeps=0, matvecs=0, rejections=0, expm=0, status=OK, m=m_init)
    if not np.any(w):
        return [np.zeros(N) for _ in tau_out], info
    t = 0.0
    tau = tau_end
    m = min(m_init, m_max)
    ti = 0
    while ti < len(times):
        if info["substeps"] >= max_substeps:
            info["status"] = ENOTCONV
            break
        next_out = times[ti]
        tau = min(tau, next_out - t)
        beta = np.linalg.norm(w)
        V = [w / beta]
        H = np.zeros((m_max + 2, m_max + 2))
        built = 0
        happy = False
        while True:
            while built < m and not happy:
                j = built
                z = apply_aug(V[j])
                info["matvecs"] += 1
                win = range(max(0, j - iop + 1), j + 1)
                for i in win:
                    H[i, j] = np.dot(V[i], z)
                z0 = np.linalg.norm(z)
                for i in win:
                    z = z - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(z)
                built += 1
                if not np.isfinite(H[j + 1, j]):
                    info["status"] = ENAN
                    return [np.zeros(N) for _ in tau_out], info
                if H[j + 1, j] <= 1e-12 * z0:
                    happy = True
                    m = built
                    break
                V.append(z / H[j + 1, j])
            if happy:
                F = scipy.linalg.expm(tau * H[:m, :m])[:, 0]
                omega = 0.0
            else:
                Hbar = np.zeros((m + 1, m + 1))
                Hbar[:m, :m] = H[:m, :m]
                Hbar[m, m - 1] = H[m, m - 1]
                F = scipy.linalg.expm(tau * Hbar)[:, 0]
                err = beta * abs(F[m])
                omega = (tau_end / tau) * err / (tol * beta)
            info["expm"] += 1
            if not np.isfinite(omega):
                info["status"] = ENAN
                return [np.zeros(N) for _ in tau_out], info
            if omega <= 1.0:
                w = beta * sum(F[i] * V[i] for i in range(len(F)))
                t = t + tau
                info["substeps"] += 1
                if abs(t - next_out) <= 1e-13 * max(1.0, next_out):
                    t = next_out
                    results[next_out] = w[:N].copy()
                    ti += 1
                g = 2.0 if omega == 0.0 else min(2.0, max(1.0, 0.8 * omega ** (-1.0 / m)))
                tau = tau * g
                break
            info["rejections"] += 1
            if m < m_max:
                m = min(m_max, m + m_step)
            else:
                tau = tau * min(0.9, max(0.1, 0.8 * omega ** (-1.0 / m)))
    info["m"] = m
    return [results.get(float(t), np.zeros(N)) for t in tau_out], info


def kiops_phi(apply_A, v, outputs, tol, **kw):
    """phi_{l_k}(s_k A) v for outputs [(l_k, s_k)] by KIOPS: for each distinct l,
    one run with b_l = v and output times s_k, divided by s_k^l."""
    res = [None] * len(outputs)
    infos = []
    for l in sorted(set(l for l, _ in outputs)):
        idx = [i for i, (ll, _) in enumerate(outputs) if ll == l]
        bs = [None] * (l + 1)
        bs[l] = v
        outs, info = kiops(apply_A, bs, [outputs[i][1] for i in idx], tol, **kw)
        infos.append(info)
        for i, o in zip(idx, outs):
            res[i] = o / (outputs[i][1] ** l)
    return res, infos
