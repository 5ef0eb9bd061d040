"""Karhunen-Loeve expansion of the random input field (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

The paper parameterizes the random coefficient field by a KL expansion
(Section 1; Section 2 assumes i.i.d. entries of xi) but never states the
covariance.  The workloads use the exponential covariance
C(x, y) = sigma^2 exp(-|x - y| / ell) on [0, 1] (1D) and its separable product
on [0, 1]^2 (2D), with the log-normal coefficient a = exp(g),
g(x; xi) = sum_m sqrt(lambda_m) phi_m(x) xi_m.

Eigenpairs of the exponential kernel are the textbook closed forms
(Ghanem & Spanos, the paper's reference R.G): on the centred interval
[-1/2, 1/2] with c = 1/ell,

  even modes   c - w tan(w/2) = 0,   phi = cos(w t) / sqrt(1/2 + sin(w)/(2w))
  odd modes    w + c tan(w/2) = 0,   phi = sin(w t) / sqrt(1/2 - sin(w)/(2w))
  lambda = 2 c sigma^2 / (w^2 + c^2),         t = x - 1/2.

Each equation has exactly one root per half period of tan(w/2); the roots are
found by bracketed Brent iteration.  Modes are ordered by decreasing lambda.
2D: pairs (i, j) of unit-variance 1D modes, lambda = sigma^2 l_i l_j,
phi = phi_i(x1) phi_j(x2); ordered by decreasing lambda, ties broken by
(i + j, i) ascending.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.optimize import brentq


def exp_cov_modes_1d(corr_len: float, count: int, sigma: float = 1.0):
    """First ``count`` KL modes of sigma^2 exp(-|x-y|/corr_len) on [0,1].

    Returns (lam[count], omega[count], parity[count]) with parity 0 = even
    (cosine) mode and 1 = odd (sine) mode, sorted by decreasing lam.
    """
    c = 1.0 / corr_len
    cands = []
    k = 0
    while len(cands) < 2 * count + 2:
        # even root on w in (2k pi, 2k pi + pi)
        lo, hi = 2 * k * math.pi, 2 * k * math.pi + math.pi
        off = 1e-10 * max(1.0, hi)      # stay clear of the pole of tan(w/2)
        fe = lambda w: c - w * math.tan(w / 2)
        w = brentq(fe, lo + (1e-14 if k == 0 else off), hi - off,
                   xtol=1e-15, rtol=8.9e-16, maxiter=500)
        cands.append((w, 0))
        # odd root on w in (2k pi + pi, 2k pi + 2 pi)
        lo, hi = 2 * k * math.pi + math.pi, 2 * k * math.pi + 2 * math.pi
        fo = lambda w: w + c * math.tan(w / 2)
        off = 1e-10 * max(1.0, hi)
        w = brentq(fo, lo + off, hi - off, xtol=1e-15, rtol=8.9e-16,
                   maxiter=500)
        cands.append((w, 1))
        k += 1
    cands.sort(key=lambda t: t[0])
    cands = cands[:count]
    omega = np.array([t[0] for t in cands])
    parity = np.array([t[1] for t in cands], dtype=np.int64)
    lam = 2.0 * c * sigma ** 2 / (omega ** 2 + c ** 2)
    return lam, omega, parity


def exp_cov_phi_1d(x, omega: float, parity: int):
    """Normalized eigenfunction on [0,1] for root ``omega``."""
    t = np.asarray(x, dtype=np.float64) - 0.5
    if parity == 0:
        return np.cos(omega * t) / math.sqrt(0.5 + math.sin(omega) / (2 * omega))
    return np.sin(omega * t) / math.sqrt(0.5 - math.sin(omega) / (2 * omega))


def transcendental_residual(omega: float, parity: int, corr_len: float) -> float:
    c = 1.0 / corr_len
    if parity == 0:
        return c - omega * math.tan(omega / 2)
    return omega + c * math.tan(omega / 2)


def field_basis_1d(sigma: float, corr_len: float, M: int, x) -> np.ndarray:
    """Rows sqrt(lambda_m) phi_m(x) for m = 1..M evaluated at points x: [M, len(x)]."""
    lam, om, par = exp_cov_modes_1d(corr_len, M, sigma)
    return np.stack([math.sqrt(lam[m]) * exp_cov_phi_1d(x, om[m], par[m])
                     for m in range(M)])


def modes_2d(sigma: float, corr_len: float, M: int):
    """Top-M separable 2D modes: list of (lam, i, j) with 1D mode indices i, j."""
    n1 = M + 2
    lam1, om1, par1 = exp_cov_modes_1d(corr_len, n1, 1.0)
    pairs = []
    for i in range(n1):
        for j in range(n1):
            pairs.append((sigma ** 2 * (lam1[i] * lam1[j]), i, j))   # (i,j), (j,i) tie exactly
    pairs.sort(key=lambda t: (-t[0], t[1] + t[2], t[1]))
    return pairs[:M], (lam1, om1, par1)


def log_coefficient_1d(xi: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """g(x; xi) = sum_m sqrt(lambda_m) phi_m(x) xi_m for each row of xi."""
    return np.asarray(xi, dtype=np.float64) @ basis
