"""Independent numpy restatements used to pin the oracle.

Nothing here is shared with ``oracle/oracle.c`` or with the CUDA library:
the integrand is written from the direct definitions (Fermi functions and the
divided difference, not the tanh identities the oracle uses), the brute-force
quadratures are dense periodic trapezoid and tensor Gauss-Legendre grids, and
the form-factor shift matrix is derived by hand from the angle-addition
formulas.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import expit

PH, PP, MONOMIAL, OVERLAP = 0, 1, 2, 3
R2 = math.sqrt(2.0)

# inversion parity p_n: f_n(-k) = p_n f_n(k)
PARITY = np.array([1, 1, 1, -1, -1, 1, 1, -1, -1], dtype=np.float64)
# sign under k -> k + (pi, pi): f_n(k + Q) = s_n f_n(k)
SHIFT_Q = np.array([1, -1, -1, -1, -1, 1, 1, 1, 1], dtype=np.float64)


def disp(kx, ky, lat):
    t, tp, mu = lat
    return -2.0 * t * (np.cos(kx) + np.cos(ky)) - 4.0 * tp * np.cos(kx) * np.cos(ky) - mu


def ff(n, kx, ky):
    cx, cy, sx, sy = np.cos(kx), np.cos(ky), np.sin(kx), np.sin(ky)
    return [np.ones_like(cx), cx + cy, cx - cy, R2 * sx, R2 * sy,
            2 * cx * cy, 2 * sx * sy, 2 * sx * cy, 2 * cx * sy][n]


def nF(e, T):
    return expit(-e / T)


def minus_dnF(e, T):
    f = nF(e, T)
    return f * (1.0 - f) / T


def kernel_direct(kind, e1, e2, T, eps=1e-7):
    """ph: [nF(e2) - nF(e1)]/(e1 - e2); pp: [1 - nF(e1) - nF(e2)]/(e1 + e2);
    the derivative limit where the denominator is below eps."""
    if kind == PH:
        num = nF(e2, T) - nF(e1, T)
        den = e1 - e2
    else:
        num = 1.0 - nF(e1, T) - nF(e2, T)
        den = e1 + e2
    small = np.abs(den) < eps
    safe = np.where(small, 1.0, den)
    return np.where(small, minus_dnF(e1, T), num / safe)


def integrand(kind, q, l, m, T, lat, kx, ky):
    pref = 1.0 / (4.0 * math.pi ** 2)
    qx, qy = q
    if kind == PH:
        return pref * ff(l, kx, ky) * ff(m, kx + qx, ky + qy) * \
            kernel_direct(PH, disp(kx, ky, lat), disp(kx + qx, ky + qy, lat), T)
    if kind == PP:
        return pref * ff(l, kx, ky) * ff(m, qx - kx, qy - ky) * \
            kernel_direct(PP, disp(kx, ky, lat), disp(qx - kx, qy - ky, lat), T)
    if kind == OVERLAP:
        return pref * ff(l, kx, ky) * ff(m, kx + qx, ky + qy)
    if kind == MONOMIAL:
        return pref * (kx / math.pi) ** l * (ky / math.pi) ** m
    raise ValueError(kind)


def trapezoid(kind, q, l, m, T, lat, M, chunk=1 << 20):
    """Dense periodic trapezoid rule on an M x M grid of [-pi, pi)^2 (spectrally
    convergent for analytic periodic integrands)."""
    g = -math.pi + 2.0 * math.pi * np.arange(M) / M
    rows = max(1, chunk // M)
    total = 0.0
    for i0 in range(0, M, rows):
        KX, KY = np.meshgrid(g[i0:i0 + rows], g, indexing="ij")
        total += float(np.sum(integrand(kind, q, l, m, T, lat, KX, KY)))
    return total * (2.0 * math.pi / M) ** 2


def gauss_legendre(kind, q, l, m, T, lat, n):
    """Tensor n x n Gauss-Legendre rule on [-pi, pi]^2."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = math.pi * x
    w = math.pi * w
    KX, KY = np.meshgrid(x, x, indexing="ij")
    return float(np.sum(w[:, None] * w[None, :] * integrand(kind, q, l, m, T, lat, KX, KY)))


def shift_matrix(q):
    """S(q) with f_m(k + q) = sum_n S[m, n] f_n(k) for the 9 form factors,
    from cos(k+a) = cos k cos a - sin k sin a and sin(k+a) = sin k cos a + cos k sin a
    with cx = (f1+f2)/2, cy = (f1-f2)/2, sx = f3/sqrt2, sy = f4/sqrt2."""
    a, b = q
    ca, sa, cb, sb = math.cos(a), math.sin(a), math.cos(b), math.sin(b)
    S = np.zeros((9, 9))
    S[0, 0] = 1.0
    S[1, 1], S[1, 2], S[1, 3], S[1, 4] = (ca + cb) / 2, (ca - cb) / 2, -sa / R2, -sb / R2
    S[2, 1], S[2, 2], S[2, 3], S[2, 4] = (ca - cb) / 2, (ca + cb) / 2, -sa / R2, sb / R2
    S[3, 1], S[3, 2], S[3, 3] = sa / R2, sa / R2, ca
    S[4, 1], S[4, 2], S[4, 4] = sb / R2, -sb / R2, cb
    S[5, 5], S[5, 8], S[5, 7], S[5, 6] = ca * cb, -ca * sb, -sa * cb, sa * sb
    S[6, 6], S[6, 7], S[6, 8], S[6, 5] = ca * cb, ca * sb, sa * cb, sa * sb
    S[7, 7], S[7, 6], S[7, 5], S[7, 8] = ca * cb, -ca * sb, sa * cb, -sa * sb
    S[8, 8], S[8, 5], S[8, 6], S[8, 7] = ca * cb, ca * sb, -sa * cb, -sa * sb
    return S


def c4v_ops():
    """The 8 point-group operations as 2x2 integer matrices g (k -> g k)."""
    ops = []
    for sxx in (1, -1):
        for syy in (1, -1):
            ops.append(np.array([[sxx, 0], [0, syy]]))
            ops.append(np.array([[0, sxx], [syy, 0]]))
    return ops


def ff_rep(g, npts=64, seed=7):
    """D(g) with f_n(g k) = sum_a D[n, a] f_a(k), fitted at random k by least
    squares (the form factors are closed under C4v, so the fit is exact)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(-math.pi, math.pi, size=(npts, 2))
    gk = k @ np.asarray(g, dtype=np.float64).T
    A = np.stack([ff(a, k[:, 0], k[:, 1]) for a in range(9)], axis=1)
    D = np.zeros((9, 9))
    for n in range(9):
        y = ff(n, gk[:, 0], gk[:, 1])
        D[n], *_ = np.linalg.lstsq(A, y, rcond=None)
    return np.round(D, 12)
