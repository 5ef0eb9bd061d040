"""Parareal with sequential and with diagonalized coarse grid correction (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

Storage: an iterate u^k holds U^k_1..U^k_N as rows of an [N, n] array
(Section 3.2, the stacked vector u^k).  Index n-1 of the array is U_n.

Algorithm 2 (parallel CGC), one iteration from U^k:
  Step 1  Utilde_{n,J} = F(Utilde_{n,0}) with Utilde_{1,0} = u0 and
          Utilde_{n,0} = U^k_{n-1} for n >= 2 (eq. PGC_step1 and the cases
          that follow it).
  Step 2  b_1 = Utilde_{1,J} - G(alpha U^k_N), b_n = Utilde_{n,J} - G(U^k_{n-1})
          (definition of b^k); the CGC system (eq. matrix_NT) is solved by one
          simplified-Newton step (eq. Newton2) started from u_0 = u^k.  For
          the linear f(u) = -A u + f0 the Jacobian -A is constant, so its
          average is exact and one step solves eq. matrix_NT exactly.
          The step is applied by the three-step diagonalization
          (eq. three steps) with a direct O(N^2) DFT over all N frequencies.
  Step 3  stop when max_n ||U^{k+1}_n - U^k_n||_inf <= tol.

Readings (the paper is garbled or silent here):
 * Eigenvector orientation.  The printed V = Lambda_alpha F_N does not
   diagonalize C_alpha (N = 2 gives a counter-example); the eigenvectors are
   the columns of V = Lambda_alpha^{-1} F_N with Lambda_alpha =
   diag(alpha^{(n-1)/N}), for the printed eigenvalues
   lambda_n = 1 - alpha^{1/N} omega^{-(n-1)}.  Hence step (a) scales r by
   alpha^{(n-1)/N} before F_N^*, and step (c) scales by alpha^{-(n-1)/N}
   after F_N.  ``diag_factors(..., printed=True)`` returns the printed form
   so that a test can show it fails.
 * The first eliminated CGC equation lacks its "=" sign; it reads like the
   other rows.
 * Utilde^k_{n,j+1} in Step 2 means the end point Utilde^k_{n,J}.
 * Stopping rule: per-sample absolute increment, as above; the iteration
   count is the number of CGC updates performed.
 * Fine time points are uniform (dt = dT/J), J constant.
"""
from __future__ import annotations

import numpy as np

from .heat1d import F, G


def calpha(N: int, alpha: float) -> np.ndarray:
    """C_alpha of eq. matrix_NT."""
    C = np.eye(N) - np.eye(N, k=-1)
    C[0, N - 1] = -alpha
    return C


def dft_matrix(N: int) -> np.ndarray:
    """F_N with entries omega^{jk} / sqrt(N), omega = exp(2 pi i / N).

    omega^N = 1, so omega^{jk} = omega^{(jk mod N)}: the exponent is reduced
    before the angle is formed, so that every entry is exp of an angle below
    2 pi (for jk up to (N-1)^2 the unreduced angle carries a rounding error of
    eps jk, which step (c)'s alpha^{-(n-1)/N} scaling would amplify)."""
    j = np.arange(N)
    return np.exp(2j * np.pi * (np.outer(j, j) % N) / N) / np.sqrt(N)


def diag_factors(N: int, alpha: float, printed: bool = False):
    """(V, lam) with C_alpha = V diag(lam) V^{-1} (corrected orientation)."""
    n = np.arange(N)
    lam = 1.0 - alpha ** (1.0 / N) * np.exp(-2j * np.pi * n / N)
    scale = alpha ** (n / N)
    Lam = np.diag(scale if printed else 1.0 / scale)
    return Lam @ dft_matrix(N), lam


def cgc_rhs(op, Uk: np.ndarray, b: np.ndarray, dT: float) -> np.ndarray:
    """r^k of eq. three steps at l = 0 (u_0 = u^k), with grad f = -A."""
    Fu = -op.apply(Uk - b) + op.forcing            # F(u_0): f(T_{n-1}, U_n - b_n)
    return dT * op.apply(Uk) + dT * Fu + b         # -dT (I (x) grad f) u_0 + dT F(u_0) + b


def cgc_diagonalized(op, r: np.ndarray, dT: float, alpha: float,
                     fft: bool = False) -> np.ndarray:
    """Solve (C_alpha (x) I + dT I (x) A) u = r by steps (a)-(c), direct DFT.

    fft=True applies F_N and F_N^* with numpy's FFT instead of the explicit
    DFT matrix: the same method along another rounding path, used only to
    measure the method's own rounding floor (the alpha^{-(n-1)/N} scaling of
    step (c) multiplies roundoff by up to 1/alpha).
    """
    N = r.shape[0]
    n = np.arange(N)
    lam = 1.0 - alpha ** (1.0 / N) * np.exp(-2j * np.pi * n / N)
    sr = (alpha ** (n / N))[:, None] * r
    if fft:
        p = np.fft.fft(sr, axis=0) / np.sqrt(N)
    else:
        FN = dft_matrix(N)
        # (a) p = (V^{-1} (x) I) r = (F_N^* (x) I)(Lambda_alpha (x) I) r
        p = FN.conj().T @ sr
    # (b) (lambda_n I + dT A) q_n = p_n for every n (all N frequencies), with
    # iterative refinement where the operator offers it (1D): the plain banded
    # solve loses the smooth modes to pivot cancellation at large dT w, and
    # step (c) amplifies that loss by up to 1/alpha
    solve = getattr(op, "shifted_solve_refined", op.shifted_solve)
    q = np.empty_like(p)
    for k in range(N):
        q[k] = solve(lam[k], dT, p[k])
    # (c) u = (V (x) I) q = (Lambda_alpha^{-1} (x) I)(F_N (x) I) q
    Fq = np.fft.ifft(q, axis=0) * np.sqrt(N) if fft else dft_matrix(N) @ q
    u = (alpha ** (-n / N))[:, None] * Fq
    return u.real


def cgc_dense(op, r: np.ndarray, dT: float, alpha: float) -> np.ndarray:
    """Brute force: dense solve of (C_alpha (x) I + dT I (x) A) u = r."""
    N, nx = r.shape
    K = np.kron(calpha(N, alpha), np.eye(nx)) + dT * np.kron(np.eye(N), op.dense())
    return np.linalg.solve(K, r.reshape(-1)).reshape(N, nx)


def jump_b(op, Fend: np.ndarray, Uk: np.ndarray, dT: float, alpha: float) -> np.ndarray:
    """b^k of Section 3.2: b_1 uses G(alpha U_N), b_n uses G(U_{n-1})."""
    prev = np.empty_like(Uk)
    prev[0] = alpha * Uk[-1]
    prev[1:] = Uk[:-1]
    return Fend - G(op, prev, dT)


def fine_sweep(op, u0: np.ndarray, Uk: np.ndarray, dT: float, J: int) -> np.ndarray:
    """Step 1 of Algorithm 2: F on every subinterval, u0 on the first one."""
    starts = np.empty_like(Uk)
    starts[0] = u0
    starts[1:] = Uk[:-1]
    return F(op, starts, dT, J)


def pcgc_iteration(op, u0, Uk, dT: float, J: int, alpha: float, cgc: str = "diag") -> np.ndarray:
    """One iteration of Algorithm 2.  cgc selects how eq. matrix_NT is solved:
    "diag" (the three steps with a direct DFT, the paper's method), "fft"
    (the same with numpy's FFT) or "dense" (Kronecker brute force, the exact
    solution of the same system; used to measure the diagonalization's own
    rounding error)."""
    Fend = fine_sweep(op, u0, Uk, dT, J)
    b = jump_b(op, Fend, Uk, dT, alpha)
    r = cgc_rhs(op, Uk, b, dT)
    if cgc == "dense":
        return cgc_dense(op, r, dT, alpha)
    return cgc_diagonalized(op, r, dT, alpha, fft=(cgc == "fft"))


def pcgc_solve(op, u0, U0, dT: float, J: int, alpha: float, tol: float,
               kmax: int, history: bool = False, cgc: str = "diag"):
    """Algorithm 2 from the initial guess U0 ([N, n]).

    Returns (U, iters, hist) where iters = number of CGC updates until the
    increment fell to tol, or -1 when kmax updates did not reach it.
    """
    U = np.array(U0, dtype=np.float64)
    hist = [U.copy()] if history else None
    for k in range(kmax):
        Un = pcgc_iteration(op, u0, U, dT, J, alpha, cgc=cgc)
        delta = np.max(np.abs(Un - U))
        U = Un
        if history:
            hist.append(U.copy())
        if not np.isfinite(delta):
            return U, -2, hist
        if delta <= tol:
            return U, k + 1, hist
    return U, -1, hist


def parareal_classical(op, u0, U0, dT: float, J: int, K: int):
    """Algorithm 1 (sequential CGC, eq. pred_correc) for K iterations.

    Returns the list of iterates [U^0, ..., U^K] ([N, n] arrays, row n-1 = U_n).
    """
    N = U0.shape[0]
    U = np.array(U0, dtype=np.float64)
    out = [U.copy()]
    for _ in range(K):
        starts = np.empty_like(U)
        starts[0] = u0
        starts[1:] = U[:-1]
        Fk = F(op, starts, dT, J)
        Gk = G(op, starts, dT)
        Un = np.empty_like(U)
        prev = np.asarray(u0, dtype=np.float64)
        for n in range(N):
            Un[n] = G(op, prev, dT) + Fk[n] - Gk[n]
            prev = Un[n]
        U = Un
        out.append(U.copy())
    return out


def cgc_sequential(op, r: np.ndarray, dT: float) -> np.ndarray:
    """alpha = 0 limit: forward substitution of (C_0 (x) I + dT I (x) A) u = r."""
    N = r.shape[0]
    u = np.empty_like(r)
    prev = np.zeros(r.shape[1])
    for n in range(N):
        u[n] = op.shifted_solve(1.0, dT, r[n] + prev)
        prev = u[n]
    return u


def coarse_guess(op, u0, N: int, dT: float) -> np.ndarray:
    """U^0_n = G(U^0_{n-1}), U^0_0 = u0: the coarse-sweep guess of Section 3.1."""
    out = np.empty((N, op.n))
    v = np.asarray(u0, dtype=np.float64)
    for n in range(N):
        v = G(op, v, dT)
        out[n] = v
    return out
