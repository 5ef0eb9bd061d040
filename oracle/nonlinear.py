"""Nonlinear problems and the nonlinear coarse grid correction (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

Test infrastructure only (imported by tests/, smoke() and bench.py's CPU
legs); shares no code with the library.

Problems (eq. psys with a nonlinear f), A the 1D flux-form operator of
oracle.heat1d (a at the faces, zero Dirichlet values):

* Allen-Cahn-type reaction (CubicRD1D):
      f(u) = -A u - c (u^3 - u) + f0,   grad f(u) = -A - c diag(3 u^2 - 1).
* Burgers-type convection (BurgersEO1D, Section 5, Burgers equation): the
  convective term (u^2/2)_x in conservative upwind form with the
  Engquist-Osher flux splitting,
      f(u) = -A u - c conv(u) + f0,
      conv(u)_i = (Phi(u_i, u_{i+1}) - Phi(u_{i-1}, u_i)) / h,
      Phi(l, r) = max(l, 0)^2 / 2 + min(r, 0)^2 / 2,   u_0 = u_{nx+1} = 0;
  for u >= 0 this is the backward (upwind) difference (u_i^2 - u_{i-1}^2)/(2h).
  grad conv(u) is tridiagonal: |u_i|/h on the diagonal, min(u_{i+1}, 0)/h
  right of it and -max(u_{i-1}, 0)/h left of it.

Propagators (backward Euler, Section 5): one step of size dt solves
    w - v = dt f(w)   <=>   w + dt A w + dt c (w^3 - w) = v + dt f0
by Newton's method from w = v (tridiagonal Jacobian I + dt A + dt c diag(3w^2 - 1)).

Coarse grid correction (Section 3.2): with the jump b^k (eq. after PGC_step2,
G nonlinear), the CGC solves eq. matrix_NT,
    (C_alpha (x) I) u = dT F(u) + b,   F(u)_n = f(U_n - b_n),
by the simplified Newton iteration eq. Newton2 with the time-averaged
Jacobian (eq. Jac),
    Jbar u_{l+1} = -dT (I (x) gradf_bar) u_l + dT F(u_l) + b,
    gradf_bar = (1/N) sum_n grad f(U_{n,l} - b_n),  Jbar = C_alpha (x) I - dT I (x) gradf_bar,
from u_0 = U^k.  Jbar is diagonalized like the linear case: the three steps
with A replaced by -gradf_bar (a different shifted tridiagonal per l).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded

from .heat1d import Heat1D


class CubicRD1D(Heat1D):
    """Heat1D's operator A (with reaction 0) plus the cubic reaction c (u^3 - u)."""

    def __init__(self, a_faces, c: float, forcing: float = 0.0):
        super().__init__(a_faces, 0.0, forcing)
        self.c = float(c)

    def f(self, U):
        U = np.asarray(U, dtype=np.float64)
        return -self.apply(U) - self.c * (U ** 3 - U) + self.forcing

    def jac_diag_extra(self, u):
        """grad f(u) = -A - diag(this)."""
        return self.c * (3.0 * np.asarray(u) ** 2 - 1.0)

    def _banded(self, dt, extra):
        """Banded form of I + dt (A + diag(extra))."""
        ab = np.zeros((3, self.n))
        ab[1] = 1.0 + dt * (self.diag + extra)
        ab[0, 1:] = dt * self.off
        ab[2, :-1] = dt * self.off
        return ab

    def avg_K_dense(self, u, b):
        """-gradf_bar = A + diag(averaged_extra(u, b)) (eq. Jac), dense."""
        return self.dense() + np.diag(averaged_extra(self, u, b))

    def be_step_newton(self, v, dt, tol=1e-14, maxit=50):
        """w with w + dt A w + dt c (w^3 - w) = v + dt f0 (Newton from w = v)."""
        v = np.asarray(v, dtype=np.float64)
        w = v.copy()
        rhs = v + dt * self.forcing
        for _ in range(maxit):
            R = w + dt * self.apply(w) + dt * self.c * (w ** 3 - w) - rhs
            ab = self._banded(dt, self.jac_diag_extra(w))
            d = solve_banded((1, 1), ab, R)
            w = w - d
            if np.max(np.abs(d)) <= tol * max(1.0, np.max(np.abs(w))):
                break
        return w


class BurgersEO1D(Heat1D):
    """Heat1D's operator A (reaction 0) plus the convection c (u^2/2)_x in
    Engquist-Osher upwind form (module docstring)."""

    def __init__(self, a_faces, c: float, forcing: float = 0.0):
        super().__init__(a_faces, 0.0, forcing)
        self.c = float(c)

    def conv(self, U):
        U = np.asarray(U, dtype=np.float64)
        z = np.zeros(U.shape[:-1] + (1,))
        P = np.concatenate([z, U, z], axis=-1)             # boundary zeros
        flux = np.maximum(P[..., :-1], 0.0) ** 2 / 2 + np.minimum(P[..., 1:], 0.0) ** 2 / 2
        return (flux[..., 1:] - flux[..., :-1]) / self.h   # faces i+1/2 minus i-1/2

    def f(self, U):
        return -self.apply(U) - self.c * self.conv(U) + self.forcing

    def K_bands(self, w):
        """Bands of K(w) = -grad f(w) = A + c grad conv(w) along the last axis:
        (sub, diag, sup), sub[i] = K[i, i-1] (sub[0] unused), sup[i] = K[i, i+1]
        (sup[-1] unused)."""
        w = np.asarray(w, dtype=np.float64)
        ch = self.c / self.h
        diag = self.diag + ch * np.abs(w)
        sub = np.zeros_like(w)
        sup = np.zeros_like(w)
        sub[..., 1:] = self.off - ch * np.maximum(w[..., :-1], 0.0)
        sup[..., :-1] = self.off + ch * np.minimum(w[..., 1:], 0.0)
        return sub, diag, sup

    @staticmethod
    def _dense(sub, diag, sup):
        return np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)

    def jacobian(self, w):
        """grad f(w), dense."""
        return -self._dense(*self.K_bands(w))

    def avg_K_dense(self, u, b):
        """-gradf_bar = -(1/N) sum_n grad f(U_n - b_n) (eq. Jac), dense: the
        band entries averaged over the N intervals."""
        sub, diag, sup = self.K_bands(np.asarray(u) - np.asarray(b))
        return self._dense(sub.mean(axis=0), diag.mean(axis=0), sup.mean(axis=0))

    def be_step_newton(self, v, dt, tol=1e-14, maxit=50):
        """w with w + dt A w + dt c conv(w) = v + dt f0 (Newton from w = v)."""
        v = np.asarray(v, dtype=np.float64)
        w = v.copy()
        rhs = v + dt * self.forcing
        for _ in range(maxit):
            R = w + dt * self.apply(w) + dt * self.c * self.conv(w) - rhs
            sub, diag, sup = self.K_bands(w)
            ab = np.zeros((3, self.n))
            ab[0, 1:] = dt * sup[:-1]
            ab[1] = 1.0 + dt * diag
            ab[2, :-1] = dt * sub[1:]
            d = solve_banded((1, 1), ab, R)
            w = w - d
            if np.max(np.abs(d)) <= tol * max(1.0, np.max(np.abs(w))):
                break
        return w


def _be_step_rows(op, V, dt):
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        return op.be_step_newton(V, dt)
    return np.stack([op.be_step_newton(v, dt) for v in V])


# the linear oracle's propagators (oracle.pcgc F, G, parareal_classical,
# coarse_guess) call op.be_step: on these problems it is the Newton step
CubicRD1D.be_step = _be_step_rows
BurgersEO1D.be_step = _be_step_rows


def F(op: CubicRD1D, starts, dT: float, J: int):
    out = np.empty_like(np.asarray(starts, dtype=np.float64))
    for n, v in enumerate(starts):
        w = np.array(v, dtype=np.float64)
        for _ in range(J):
            w = op.be_step_newton(w, dT / J)
        out[n] = w
    return out


def G(op: CubicRD1D, V, dT: float):
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        return op.be_step_newton(V, dT)
    return np.stack([op.be_step_newton(v, dT) for v in V])


def fine_sequential(op: CubicRD1D, u0, N: int, J: int, T: float):
    """U*_n, n = 1..N: N*J Newton backward-Euler steps of T/(N J)."""
    dt = T / (N * J)
    w = np.array(u0, dtype=np.float64)
    out = []
    for _ in range(N):
        for _ in range(J):
            w = op.be_step_newton(w, dt)
        out.append(w.copy())
    return np.stack(out)


def jump_b(op, Fend, Uk, dT, alpha):
    """b_1 = F_1 - G(alpha U_N), b_n = F_n - G(U_{n-1})."""
    prev = np.empty_like(Uk)
    prev[0] = alpha * Uk[-1]
    prev[1:] = Uk[:-1]
    return Fend - G(op, prev, dT)


def cgc_residual(op, u, b, dT, alpha):
    """(C_alpha (x) I) u - dT F(u) - b  (eq. matrix_NT; zero at its solution)."""
    Cu = u.copy()
    Cu[0] -= alpha * u[-1]
    Cu[1:] -= u[:-1]
    return Cu - dT * op.f(u - b) - b


def averaged_extra(op, u, b):
    """The diagonal part of -gradf_bar beyond A: mean_n c (3 (U_n - b_n)^2 - 1)."""
    return np.mean(op.jac_diag_extra(u - b), axis=0)


def cgc_newton_step(op, u, b, dT, alpha):
    """One simplified Newton step (eq. Newton2) by the diagonalization (eq.
    three steps) with A replaced by -gradf_bar."""
    N, n = u.shape
    K = op.avg_K_dense(u, b)                        # -gradf_bar
    rhs = dT * (u @ K.T) + dT * op.f(u - b) + b      # -dT(I(x)gradf_bar)u + dT F(u) + b
    j = np.arange(N)
    lam = 1.0 - alpha ** (1.0 / N) * np.exp(-2j * np.pi * j / N)
    sr = (alpha ** (j / N))[:, None] * rhs
    W = np.exp(-2j * np.pi * (np.outer(j, j) % N) / N)  # F_N^* sqrt(N) (omega^N = 1)
    p = W @ sr
    q = np.stack([np.linalg.solve(lam[k] * np.eye(n) + dT * K, p[k]) for k in range(N)])
    u_new = (np.conj(W) @ q) / N
    return ((alpha ** (-j / N))[:, None] * u_new).real


def cgc_newton_dense(op, u, b, dT, alpha):
    """The same step by a dense solve of Jbar (brute force)."""
    N, n = u.shape
    K = op.avg_K_dense(u, b)
    Ca = np.eye(N) - np.eye(N, k=-1)
    Ca[0, -1] = -alpha
    Jbar = np.kron(Ca, np.eye(n)) + dT * np.kron(np.eye(N), K)
    rhs = dT * (u @ K.T) + dT * op.f(u - b) + b
    return np.linalg.solve(Jbar, rhs.reshape(-1)).reshape(N, n)


def pcgc_iteration(op, u0, Uk, dT, J, alpha, L, dense=False):
    """One iteration of Algorithm 2 with the nonlinear CGC: F on all intervals,
    the jump b, then L simplified Newton steps from u_0 = U^k.  dense=True
    solves each step's Jbar system densely (the same method along another
    rounding path, used to measure the diagonalization's rounding floor)."""
    starts = np.empty_like(Uk)
    starts[0] = u0
    starts[1:] = Uk[:-1]
    Fend = F(op, starts, dT, J)
    b = jump_b(op, Fend, Uk, dT, alpha)
    u = Uk.copy()
    step = cgc_newton_dense if dense else cgc_newton_step
    for _ in range(L):
        u = step(op, u, b, dT, alpha)
    return u


def pcgc_solve(op, u0, U0, dT, J, alpha, tol, kmax, L, dense=False):
    U = np.array(U0, dtype=np.float64)
    for k in range(kmax):
        Un = pcgc_iteration(op, u0, U, dT, J, alpha, L, dense)
        delta = np.max(np.abs(Un - U))
        U = Un
        if not np.isfinite(delta):
            return U, -2
        if delta <= tol:
            return U, k + 1
    return U, -1
