"""Spherical-harmonic pieces of the method, FP64 (TEST INFRASTRUCTURE ONLY).

Paper Section 2.1: the Laplace Green's function G(X;Y) = 1/|X-Y| (Eq. (6)),
its spectral expansion in spherical coordinates (Eq. (7)), the series
truncated at index M (Eq. (8)) and the error bound of Theorem 2.1 (Eq. (9)),
whose proof uses the addition theorem for Legendre polynomials.

The associated Legendre functions P_n^m are taken WITHOUT the Condon-Shortley
phase; Eq. (7) multiplies two of them with equal (n, m), so the phase
convention does not change it.  They follow the textbook recurrences

    P_m^m(x)     = (2m-1)!! (1-x^2)^{m/2}
    P_{m+1}^m(x) = (2m+1) x P_m^m(x)
    (n-m) P_n^m  = (2n-1) x P_{n-1}^m - (n+m-1) P_{n-2}^m.

For the FMM reference (a builder's extension after Greengard-Rokhlin, the
paper's ref. on the fast multipole method) the same functions give complex
solid harmonics, for m >= 0

    regular    U_n^m(v) = r^n P_n^m(cos th) e^{i m om} / (n+m)!
    irregular  T_n^m(v) = (n-m)! P_n^m(cos th) e^{i m om} / r^{n+1}

and U_n^{-m} = (-1)^m conj(U_n^m), T_n^{-m} = (-1)^m conj(T_n^m).  With these
normalisations the three identities the translations rest on carry no phase
factors:

    1/|x - y|  = sum_{n,m} conj(U_n^m(y)) T_n^m(x)                (|y| < |x|)
    U_n^m(a+b) = sum_{k,l} U_k^l(a) U_{n-k}^{m-l}(b)
    T_n^m(x-y) = sum_{k,l} conj(U_k^l(y)) T_{n+k}^{m+l}(x)         (|y| < |x|)

The first is Eq. (7) rewritten; tests check all three against direct
evaluation.  Arrays of harmonics are indexed [..., n, m + p] for |m| <= n <= p
and hold zero for |m| > n.
"""
from __future__ import annotations

import math

import numpy as np


def neumann(m: int) -> float:
    """Neumann factor: eps_0 = 1, eps_m = 2 for m > 0 (below Eq. (7))."""
    return 1.0 if m == 0 else 2.0


def legendre_table(nmax: int, x) -> np.ndarray:
    """P_n^m(x) for 0 <= m <= n <= nmax (no Condon-Shortley phase).

    x may be a scalar or an array; the result has shape x.shape + (nmax+1, nmax+1)
    with entry [..., n, m] (zero for m > n).
    """
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros(x.shape + (nmax + 1, nmax + 1))
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P[..., 0, 0] = 1.0
    for m in range(1, nmax + 1):
        P[..., m, m] = P[..., m - 1, m - 1] * (2 * m - 1) * s
    for m in range(0, nmax):
        P[..., m + 1, m] = (2 * m + 1) * x * P[..., m, m]
    for m in range(0, nmax + 1):
        for n in range(m + 2, nmax + 1):
            P[..., n, m] = ((2 * n - 1) * x * P[..., n - 1, m]
                            - (n + m - 1) * P[..., n - 2, m]) / (n - m)
    return P


def legendre_poly(n: int, x) -> np.ndarray:
    """Legendre polynomial P_n(x) by Bonnet's three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def spherical(v) -> tuple:
    """(rho, theta, omega) of 3-vectors v[..., 3]: theta in [0, pi], omega in (-pi, pi]."""
    v = np.asarray(v, dtype=np.float64)
    rho = np.sqrt(v[..., 0] ** 2 + v[..., 1] ** 2 + v[..., 2] ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(rho > 0, v[..., 2] / np.where(rho > 0, rho, 1.0), 1.0)
    theta = np.arccos(np.clip(ct, -1.0, 1.0))
    omega = np.arctan2(v[..., 1], v[..., 0])
    return rho, theta, omega


def truncated_series(X, Y, M: int) -> np.ndarray:
    """Eq. (8): the spectral series of 1/|X-Y| truncated at n <= M.

    sum_{n<=M} sum_{m<=n} eps_m (n-m)!/(n+m)! P_n^m(cos th_y) P_n^m(cos th_x)
        cos(m (om_x - om_y)) * rho_<^n / rho_>^{n+1}
    Requires rho_x != rho_y.
    """
    rx, tx, ox = spherical(X)
    ry, ty, oy = spherical(Y)
    Px = legendre_table(M, np.cos(tx))
    Py = legendre_table(M, np.cos(ty))
    rlo = np.minimum(rx, ry)
    rhi = np.maximum(rx, ry)
    out = np.zeros(np.shape(rx))
    for n in range(M + 1):
        radial = rlo ** n / rhi ** (n + 1)
        for m in range(n + 1):
            d = neumann(m) * math.factorial(n - m) / math.factorial(n + m)
            out = out + d * Py[..., n, m] * Px[..., n, m] * np.cos(m * (ox - oy)) * radial
    return out


def addition_theorem_sum(n: int, tx, ty, ox, oy) -> np.ndarray:
    """Right-hand side of the addition theorem used in the proof of Theorem 2.1:
    sum_{m<=n} eps_m (n-m)!/(n+m)! P_n^m(cos th_y) P_n^m(cos th_x) cos(m (om_x-om_y))."""
    Px = legendre_table(n, np.cos(tx))
    Py = legendre_table(n, np.cos(ty))
    out = np.zeros(np.shape(tx))
    for m in range(n + 1):
        d = neumann(m) * math.factorial(n - m) / math.factorial(n + m)
        out = out + d * Py[..., n, m] * Px[..., n, m] * np.cos(m * (np.asarray(ox) - np.asarray(oy)))
    return out


def thm21_bound(rho_x, rho_y, M: int):
    """Theorem 2.1, Eq. (9): E <= (1/rho_>) r^{M+1}/(1-r), r = rho_</rho_> < 1."""
    rho_x = np.asarray(rho_x, dtype=np.float64)
    rho_y = np.asarray(rho_y, dtype=np.float64)
    rhi = np.maximum(rho_x, rho_y)
    r = np.minimum(rho_x, rho_y) / rhi
    return r ** (M + 1) / ((1.0 - r) * rhi)


def _solid(p: int, v, irregular: bool) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    rho, th, om = spherical(v)
    P = legendre_table(p, np.cos(th))
    H = np.zeros(v.shape[:-1] + (p + 1, 2 * p + 1), dtype=np.complex128)
    for n in range(p + 1):
        if irregular:
            with np.errstate(divide="ignore"):
                radial = 1.0 / rho ** (n + 1)
        else:
            radial = rho ** n
        for m in range(n + 1):
            if irregular:
                coef = math.factorial(n - m)
            else:
                coef = 1.0 / math.factorial(n + m)
            val = coef * radial * P[..., n, m] * np.exp(1j * m * om)
            H[..., n, p + m] = val
            if m > 0:
                H[..., n, p - m] = (-1) ** m * np.conj(val)
    return H


def regular(p: int, v) -> np.ndarray:
    """Regular solid harmonics U_n^m(v), shape v.shape[:-1] + (p+1, 2p+1)."""
    return _solid(p, v, irregular=False)


def irregular(p: int, v) -> np.ndarray:
    """Irregular solid harmonics T_n^m(v), shape v.shape[:-1] + (p+1, 2p+1)."""
    return _solid(p, v, irregular=True)


def laplace_pair(p: int, X, Y) -> np.ndarray:
    """sum_{n<=p, |m|<=n} conj(U_n^m(Y)) T_n^m(X): Eq. (8) in solid-harmonic form."""
    U = regular(p, Y)
    T = irregular(p, X)
    return np.real(np.sum(np.conj(U) * T, axis=(-2, -1)))
