"""Real Leja-point interpolation of phi_l(hJ)v: Sec. 2.2 (Newton form, stop
test, spectrum by power iteration, divided differences) and Sec. 4 (the
"vertical" form: one Newton basis shared by several phi-functions /
scales).

Readings of the paper where it is silent or ambiguous (this module follows
them, and the CUDA library follows the same readings):
* spectrum: alpha <= Re sigma(J) <= beta <= 0; c = (alpha+beta)/2 and
  gamma = (beta-alpha)/4 map [alpha, beta] onto the Leja domain [-2, 2];
  the interpolated function is phi_l(s h (c + gamma xi)) where s is the
  vertical scale (1/2, 1/8, 1/9, 1 ...).
* Newton form: y_0 = v, p_0 = d_0 y_0,
  y_{m+1} = ((J - c)/gamma - xi_m) y_m,  p_{m+1} = p_m + d_{m+1} y_{m+1}.
* stop test |d_m| ||y_m|| <= tol ||p_m|| (relative 2-norm, every output),
  applied from m >= 3; non-convergence at m_max is an error.
* Leja sequence on [-2, 2]: xi_0 = 2, xi_1 = -2, xi_2 = 0, then
  xi_j = argmax prod_{i<j} |x - xi_i| (exact ties: the smaller x).
* power iteration (Sec. 2.2 "power iterations", Sec. 5.1): start vector
  from the SplitMix64 counter generator, rho_k = ||J v_k|| / ||v_k||,
  stop at relative change <= 1e-2 or 50 matvecs; alpha = -safety*rho.
* complex spectra: the interval rule above assumes a real spectrum; with an
  imaginary extent rho_im the half-width is enlarged to
  gamma = max((beta - alpha)/4, 2 rho_im) and the interval kept anchored at
  its right end, c = beta - 2 gamma (the scaled imaginary extent stays
  <= 1/2 and the interpolated function stays bounded on the interval).
  With rho_im = 0 this is the paper's rule.
* substepping: the paper substeps only the exponential; for phi_l the
  exact ODE identity below is used, one phi_l Leja pass plus l Jacobian
  actions per substep, when s h gamma exceeds gamma_cap (or s h rho_im
  exceeds iota_cap).
"""
import math
import numpy as np

from .phi import phi_scalar

# --------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): x_i = seed + (i+1) * 0x9E3779B97F4A7C15,
# then the 64-bit finaliser z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
# z *= 0x94D049BB133111EB; z ^= z>>31.  Mapped to [-0.5, 0.5) via the top 53 bits.
# --------------------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(seed, count):
    """`count` uint64 outputs of SplitMix64 for stream `seed` (pure Python ints)."""
    out = np.empty(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    out[:] = z
    return out


def splitmix64_uniform(seed, count):
    """Doubles in [-0.5, 0.5): (z >> 11) * 2^-53 - 0.5."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5


# --------------------------------------------------------------------------------------
# Leja points on [-2, 2]
# --------------------------------------------------------------------------------------
_LEJA_CACHE = {}


def leja_points(m):
    """First m real Leja points on [-2, 2] (greedy max-product sequence).

    Each new point maximises L(x) = sum_i log|x - xi_i|.  Between two
    consecutive existing points L has exactly one stationary point, the root
    of L'(x) = sum_i 1/(x - xi_i) (strictly decreasing from +inf to -inf on
    the gap); it is found by bracketed Newton iteration in every gap, and the
    best gap wins.
    """
    m = int(m)
    if m in _LEJA_CACHE:
        return _LEJA_CACHE[m].copy()
    pts = [2.0, -2.0, 0.0][:m]
    while len(pts) < m:
        P = np.array(pts)
        s = np.sort(P)
        lo = s[:-1].copy()
        hi = s[1:].copy()
        x = 0.5 * (lo + hi)
        # bracketed Newton on L'(x) = 0 in every gap: keep [lo, hi] around the
        # root, take the Newton step when it stays inside, else bisect; a gap
        # stops once its step is below 2 ulp.
        act = np.arange(len(x))
        for _ in range(200):
            xa = x[act]
            r = 1.0 / (xa[:, None] - P[None, :])
            g = np.sum(r, axis=1)
            dg = -np.sum(r * r, axis=1)
            lo[act] = np.where(g > 0.0, xa, lo[act])
            hi[act] = np.where(g > 0.0, hi[act], xa)
            xn = xa - g / dg
            bad = ~((xn > lo[act]) & (xn < hi[act]))
            xn = np.where(bad, 0.5 * (lo[act] + hi[act]), xn)
            done = np.abs(xn - xa) <= 2.0 * np.spacing(np.abs(xa))
            x[act] = xn
            act = act[~done]
            if act.size == 0:
                break
        cand = x
        L = np.sum(np.log(np.abs(cand[:, None] - P[None, :])), axis=1)
        best = np.max(L)
        tie = L >= best - 1e-12 * max(1.0, abs(best))
        pts.append(float(np.min(cand[tie])))
    out = np.array(pts[:m])
    _LEJA_CACHE[m] = out
    return out.copy()


def divided_differences(x, f):
    """Newton divided differences d_j = f[x_0, ..., x_j] (standard recursion)."""
    x = np.asarray(x, dtype=np.float64)
    d = np.array(f, dtype=np.float64, copy=True)
    n = len(x)
    for j in range(1, n):
        d[j:] = (d[j:] - d[j - 1:-1]) / (x[j:] - x[: n - j])
    return d


def phi_coefficients(xi, l, scale, c, gamma):
    """DD table of xi -> phi_l(scale * (c + gamma xi)) on the Leja points."""
    f = np.array([phi_scalar(l, scale * (c + gamma * x)) for x in xi])
    return divided_differences(xi, f)


# --------------------------------------------------------------------------------------
# Spectrum estimate
# --------------------------------------------------------------------------------------
def power_iteration(jv, n, seed=0x5EED, max_it=50, rel=1e-2):
    """Largest |eigenvalue| estimate of J by power iteration.

    Returns (rho, matvecs).  rho_k = ||J v_k|| / ||v_k||; v_{k+1} = J v_k.
    Stops when |rho_k - rho_{k-1}| <= rel * rho_k (k >= 2) or after max_it.
    """
    v = splitmix64_uniform(seed, n)
    v = v / np.linalg.norm(v)
    rho_prev = 0.0
    rho = 0.0
    for k in range(1, max_it + 1):
        w = jv(v)
        nw = np.linalg.norm(w)
        rho = nw  # ||v|| == 1
        if nw == 0.0 or not np.isfinite(nw):
            return rho, k
        if k >= 2 and abs(rho - rho_prev) <= rel * rho:
            return rho, k
        rho_prev = rho
        v = w / nw
    return rho, max_it


# --------------------------------------------------------------------------------------
# Newton interpolation (Sec. 2.2) with shared basis (Sec. 4, vertical)
# --------------------------------------------------------------------------------------
OK, ENOTCONV, ENAN = 0, 2, 3


def leja_pass(jv, v, xi, coeffs, c, gamma, tol, m_max, m_min=3):
    """One Newton-Leja pass: p^(k) = sum_m d^(k)_m y_m for every coefficient
    table d^(k) in `coeffs`, sharing y_m.  Returns (p_list, m, status)."""
    K = len(coeffs)
    y = np.array(v, dtype=np.float64, copy=True)
    p = [coeffs[k][0] * y for k in range(K)]
    ny = np.linalg.norm(y)
    for m in range(0, m_max + 1):
        npk = [np.linalg.norm(pk) for pk in p]
        if not (np.isfinite(ny) and all(np.isfinite(npk))):
            return p, m, ENAN
        if m >= m_min and all(abs(coeffs[k][m]) * ny <= tol * npk[k] for k in range(K)):
            return p, m, OK
        if m == m_max:
            break
        # y_{m+1} = ((J - c)/gamma - xi_m) y_m
        y = (jv(y) - c * y) / gamma - xi[m] * y
        for k in range(K):
            p[k] = p[k] + coeffs[k][m + 1] * y
        ny = np.linalg.norm(y)
    return p, m_max, ENOTCONV


def substep_count(h, scale, gamma, rho_im, gamma_cap, iota_cap):
    s = 1
    if gamma_cap > 0:
        s = max(s, int(math.ceil(scale * h * gamma / gamma_cap - 1e-12)))
    if iota_cap > 0 and rho_im > 0:
        s = max(s, int(math.ceil(scale * h * rho_im / iota_cap - 1e-12)))
    return s


def leja_phi(jv, v, h, alpha, beta, outputs, tol, m_max=500, rho_im=0.0,
             gamma_cap=200.0, iota_cap=0.0, m_min=3):
    """phi_{l_k}(s_k h J) v for outputs = [(l_k, s_k), ...].

    Returns (list of vectors, info dict with iters, jv, substeps, status).
    If no output needs substeps they share one Newton basis (vertical form);
    otherwise each output is integrated separately with the substep identity
      u(t+tau) = sum_{j<l} tau^j/j! w_j + tau^l phi_l(tau B) w_l,
      w_0 = u(t), w_j = B w_{j-1} + v t^(l-j)/(l-j)!   (B = s_k h J).
    """
    gamma = max(0.25 * (beta - alpha), 2.0 * rho_im)
    c = beta - 2.0 * gamma   # = (alpha + beta)/2 unless enlarged
    xi = leja_points(m_max + 1)
    info = dict(iters=0, jv=0, substeps=0, status=OK)
    subs = [substep_count(h, s, gamma, rho_im, gamma_cap, iota_cap) for (_, s) in outputs]
    if gamma == 0.0:  # J has a zero spectrum: phi_l(0) v = v / l!
        return [v / math.factorial(l) for (l, _) in outputs], info
    if max(subs) == 1:
        coeffs = [phi_coefficients(xi, l, s * h, c, gamma) for (l, s) in outputs]
        p, m, st = leja_pass(jv, v, xi, coeffs, c, gamma, tol, m_max, m_min)
        info.update(iters=m, jv=m, substeps=1, status=st)
        return p, info
    results = []
    for (l, s), ns in zip(outputs, subs):
        tau = 1.0 / ns
        B = lambda w, s=s: s * h * jv(w)
        coeff = phi_coefficients(xi, l, tau * s * h, c, gamma)
        u = np.array(v, dtype=np.float64, copy=True) if l == 0 else np.zeros_like(v)
        for i in range(ns):
            t = i * tau
            w = [u]
            for j in range(1, l + 1):
                w.append(B(w[-1]) + v * (t ** (l - j)) / math.factorial(l - j))
                info["jv"] += 1
            pl, m, st = leja_pass(jv, w[l], xi, [coeff], c, gamma, tol, m_max, m_min)
            info["iters"] += m
            info["jv"] += m
            if st != OK:
                info["status"] = st
            unew = (tau ** l) * pl[0]
            for j in range(l):
                unew = unew + (tau ** j) / math.factorial(j) * w[j]
            u = unew
        info["substeps"] += ns
        results.append(u)
    return results, info
