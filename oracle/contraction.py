"""Convergence factors of parareal with diagonalized CGC (oracle), Section 4.1.
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

For one-step methods with stability functions R_g (coarse, step dT) and R_f
(fine, step dT/J), Theorem linearthm gives the per-eigenvalue contraction

  K(z, J, alpha) = max{ |alpha R_g(z)| (1 + K_cla(z, J)), K_cla(z, J) }
  K_cla(z, J)    = |R_f(z/J)^J - R_g(z)| / (1 - |R_g(z)|)

with z in the spectrum of dT A.  Backward Euler has R(z) = 1 / (1 + z).
Also returns the Lemma lem1 iteration matrix G(z)^{-1}(G(z) - F(z)) for the
scalar test problem.
"""
from __future__ import annotations

import numpy as np


def r_be(z):
    return 1.0 / (1.0 + np.asarray(z, dtype=np.float64))


def k_cla(z, J: int):
    z = np.asarray(z, dtype=np.float64)
    return np.abs(r_be(z / J) ** J - r_be(z)) / (1.0 - np.abs(r_be(z)))


def k_alpha(z, J: int, alpha: float):
    kc = k_cla(z, J)
    return np.maximum(np.abs(alpha * r_be(z)) * (1.0 + kc), kc)


def lemma_matrices(z: float, J: int, N: int, alpha: float):
    """Scalar G(z), F(z) of Lemma lem1 (N x N)."""
    Gm = np.eye(N) - r_be(z) * np.eye(N, k=-1)
    Gm[0, N - 1] = -alpha * r_be(z)
    Fm = np.eye(N) - (r_be(z / J) ** J) * np.eye(N, k=-1)
    return Gm, Fm
