"""Offline part of Algorithm 3: snapshot KL + gPC least squares (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

Steps (Section 2.1, eqs. KLE basis, KLE parameter, KLE Snapshots, least
square A/F/problem; Algorithm 3 steps 1-6):
  1  snapshots u(xi_j), j = 1..n_t, at the N coarse times, flattened over
     (n, x); mean ubar, fluctuations utilde_j; C_{nm} = (utilde_n, utilde_m)/n_t
  2  eigenpairs (lambda_k, e_k) of C, decreasing; M_Q by the energy rule
  3  B_{jp} = psi_p(xi_j)
  4  g_k = (lambda_k n_t)^{-1/2} sum_j e_k^j utilde_j;
     D_k = [zeta_k(xi_j)]_j with zeta_k(xi) = lambda_k^{-1/2} (utilde(xi), g_k)
  5  h_k = argmin ||B h - D_k||_2 for each k
  6  U^0(xi) = ubar + sum_k sqrt(lambda_k) (sum_p h_{kp} psi_p(xi)) g_k

Readings:
 * Step 2 prints "<= 1 - eps"; the energy rule is read as the smallest M_Q
   whose captured fraction is >= 1 - eps_KL, capped at n_t - 1 (the rank of
   the mean-removed snapshot set).
 * (., .)_X is the unweighted Euclidean product over all (n, x) values;
   a uniform weight cancels in step 6.
 * Snapshots are the sequential fine solution U* of each training sample
   (the paper's reference solution; the paper generates its library with the
   parallel-CGC solver, whose converged result equals U* within tolerance).
"""
from __future__ import annotations

import numpy as np

from .gpc import psi_matrix


class Surrogate:
    def __init__(self, ubar, G, H, lam, p):
        self.ubar = ubar      # [N*n]
        self.G = G            # [M_Q, N*n] orthonormal modes g_k
        self.H = H            # [P, M_Q] gPC coefficients h_k (columns)
        self.lam = lam        # [M_Q]
        self.p = p

    @property
    def MQ(self) -> int:
        return self.G.shape[0]

    def guess(self, xi: np.ndarray) -> np.ndarray:
        """Step 6 for each row of xi: [S, N*n]."""
        B = psi_matrix(xi, self.p)                  # [S, P]
        zeta = B @ self.H                            # [S, M_Q]  zeta_k(xi)
        return self.ubar[None, :] + (zeta * np.sqrt(self.lam)[None, :]) @ self.G


def build_surrogate(snapshots: np.ndarray, xi_train: np.ndarray, p: int,
                    eps_kl: float, eig: str = "eigh") -> Surrogate:
    """snapshots: [n_t, N*n] flattened U*(xi_j).  eig="svd" takes the
    eigenpairs of C from the singular value decomposition of the
    fluctuations instead (C = Ut Ut^T / n_t = U_s (Sigma^2 / n_t) U_s^T): the
    same quantities along another rounding path, used to measure how much
    the guess depends on the rounding of the small retained modes."""
    Y = np.asarray(snapshots, dtype=np.float64)
    nt = Y.shape[0]
    ubar = Y.mean(axis=0)
    Ut = Y - ubar[None, :]
    if eig == "svd":
        E, sv, _ = np.linalg.svd(Ut, full_matrices=False)
        lam = sv ** 2 / nt
    else:
        C = (Ut @ Ut.T) / nt
        lam, E = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, E = lam[order], E[:, order]
    total = np.sum(lam)
    frac = np.cumsum(lam) / total
    MQ = int(np.searchsorted(frac, 1.0 - eps_kl) + 1)
    MQ = max(1, min(MQ, nt - 1))
    lam, E = lam[:MQ], E[:, :MQ]
    G = (E.T @ Ut) / np.sqrt(lam * nt)[:, None]
    D = (Ut @ G.T) / np.sqrt(lam)[None, :]          # zeta_k(xi_j)
    B = psi_matrix(xi_train, p)
    H = np.linalg.lstsq(B, D, rcond=None)[0]         # [P, M_Q]
    return Surrogate(ubar, G, H, lam, p)
