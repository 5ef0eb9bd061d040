"""1D random-diffusion problem and backward-Euler propagators (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

PDE (eq. psys with f(u) = (a u_x)_x - c u + f0): on (0, 1) with zero Dirichlet
boundary values, u_t = (a(x; xi) u_x)_x - c u + f0.  Finite differences on
Nx interior points x_i = i h, h = 1/(Nx+1), coefficient sampled at the faces
x_{i+1/2}:

  (A u)_i = -[a_{i+1/2}(u_{i+1} - u_i) - a_{i-1/2}(u_i - u_{i-1})] / h^2 + c u_i

so the semi-discrete system reads u' + A u = f0 (eq. ODE of Section 4.1).

Propagators (Section 3.1, both backward Euler in every experiment of
Section 5):
  G(v)  one step of Delta T:       (I + dT A) v' = v + dT f0
  F(v)  J steps of dt = dT / J:    (I + dt A) v_{j+1} = v_j + dt f0
Every linear solve is a banded LAPACK solve (scipy.linalg.solve_banded).
F_emulated is a precision experiment, not a reference: F with its
substitutions in a chosen float type (direct or increment form).

The reference ("fine-grid") solution of the paper (Section 2, remark after
eq. psys) is the sequential fine solution U*_n, n = 1..N.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded


class Heat1D:
    def __init__(self, a_faces: np.ndarray, reaction: float = 0.0,
                 forcing: float = 0.0):
        a_faces = np.asarray(a_faces, dtype=np.float64)
        self.nx = a_faces.shape[0] - 1
        self.h = 1.0 / (self.nx + 1)
        w = a_faces / self.h ** 2
        self.wf = w                                  # face weights a_{i+1/2} / h^2
        self.diag = w[:-1] + w[1:] + reaction      # A_ii
        self.off = -w[1:-1]                         # A_{i,i+1} = A_{i+1,i}
        self.forcing = float(forcing)
        self.reaction = float(reaction)

    @property
    def n(self) -> int:
        return self.nx

    def grid(self) -> np.ndarray:
        return np.arange(1, self.nx + 1) * self.h

    def apply(self, V: np.ndarray) -> np.ndarray:
        """A V along the last axis."""
        V = np.asarray(V)
        out = self.diag * V
        out[..., :-1] += self.off * V[..., 1:]
        out[..., 1:] += self.off * V[..., :-1]
        return out

    def dense(self) -> np.ndarray:
        return (np.diag(self.diag) + np.diag(self.off, 1) + np.diag(self.off, -1))

    def shifted_solve(self, shift, scale: float, R: np.ndarray) -> np.ndarray:
        """Solve (shift I + scale A) X = R along the last axis of R."""
        R = np.asarray(R)
        dt = np.result_type(R.dtype, np.asarray(shift).dtype, np.float64)
        ab = np.zeros((3, self.nx), dtype=dt)
        ab[0, 1:] = scale * self.off
        ab[1, :] = shift + scale * self.diag
        ab[2, :-1] = scale * self.off
        X = solve_banded((1, 1), ab, np.moveaxis(R, -1, 0))
        return np.moveaxis(X, 0, -1)

    def apply_flux(self, V: np.ndarray) -> np.ndarray:
        """A V along the last axis in flux form: the differences across the
        faces first, then w-weighted, -(w_{i+1/2} (v_{i+1} - v_i) - w_{i-1/2}
        (v_i - v_{i-1})) + c v_i with zero boundary values.  For a smooth V the
        face differences are small, so the rounding error is eps w |V_{i+1} - V_i|
        instead of eps w |V_i| in the diagonal/off-diagonal form."""
        V = np.asarray(V)
        z = np.zeros(V.shape[:-1] + (1,), dtype=V.dtype)
        Vp = np.concatenate([z, V, z], axis=-1)
        q = self.wf * (Vp[..., 1:] - Vp[..., :-1])
        return -(q[..., 1:] - q[..., :-1]) + self.reaction * V

    def shifted_solve_refined(self, shift, scale: float, R: np.ndarray,
                              steps: int = 2) -> np.ndarray:
        """(shift I + scale A) X = R by the banded solve plus `steps` steps of
        iterative refinement, X += solve(R - (shift X + scale A X)), with the
        residual in flux form.

        Why: the pivots of the LU are p_i = d_i - (scale w_i)^2 / p_{i-1}, a
        difference of O(scale w) numbers whose small remainder carries the smooth
        modes; for scale w ~ 1e4 (Nx = 1023, dT = 1/64) the plain FP64 solve keeps
        only ~1e-11 of them, and step (c) of the diagonalized CGC multiplies
        that by up to alpha^{-(N-1)/N} (Section 3.2, the paragraph on choosing
        alpha: the diagonalization's rounding error is governed by alpha).  The
        flux-form residual of a smooth X is accurate to eps times its face
        differences, so one refinement step restores FP64 accuracy."""
        X = self.shifted_solve(shift, scale, R)
        for _ in range(steps):
            res = R - (shift * X + scale * self.apply_flux(X))
            X = X + self.shifted_solve(shift, scale, res)
        return X

    def be_step(self, V: np.ndarray, dt: float) -> np.ndarray:
        """One backward-Euler step (I + dt A) V' = V + dt f0."""
        return self.shifted_solve(1.0, dt, V + dt * self.forcing)


def u0_sine(nx: int) -> np.ndarray:
    h = 1.0 / (nx + 1)
    return np.sin(np.pi * np.arange(1, nx + 1) * h)


def G(op, V: np.ndarray, dT: float) -> np.ndarray:
    """Coarse propagator: one backward-Euler step of size dT."""
    return op.be_step(V, dT)


def F(op, V: np.ndarray, dT: float, J: int) -> np.ndarray:
    """Fine propagator: J backward-Euler steps of size dT/J."""
    dt = dT / J
    for _ in range(J):
        V = op.be_step(V, dt)
    return V


def fine_sequential(op, u0: np.ndarray, N: int, J: int, T: float) -> np.ndarray:
    """Reference solution U*_n at T_n = n T/N, n = 1..N, shape [N, nx]."""
    dT = T / N
    out = np.empty((N, op.n))
    v = np.asarray(u0, dtype=np.float64)
    for n in range(N):
        v = F(op, v, dT, J)
        out[n] = v
    return out


def F_emulated(op, V: np.ndarray, dT: float, J: int, dtype=np.float32,
               form: str = "increment", flux_every: int = 1) -> np.ndarray:
    """F(V) (J backward-Euler steps of dt = dT/J, Section 3.1) with the
    substitutions carried out in `dtype`: a precision experiment for the fine
    propagator, not a reference.  V: [nx] or [cols][nx]; returns FP64.

    M = I + dt A is factored in FP64 (Thomas: pivots p_0 = M_00,
    l_i = M_{i,i-1} / p_{i-1}, p_i = M_ii - l_i M_{i-1,i}); l, M_{i,i+1} and
    1/p are rounded to `dtype`, and every step's forward and back
    substitution runs in `dtype`.
      form "direct":     M v' = v + dt f0
      form "increment":  M d = rhs, v' = v + d, with rhs the defect
                         -dt A v + dt f0 (A v in flux form) on every
                         flux_every-th step (the first included) and the
                         previous increment d on the others.  For a constant
                         f0 both right-hand sides are equal in exact
                         arithmetic: M (v' - v) = v - v_prev.
    A v in flux form: -(w_{i+1/2} (v_{i+1} - v_i) - w_{i-1/2} (v_i - v_{i-1}))
    + c v_i with w = a / h^2 and zero boundary values."""
    dt = dT / J
    n = op.n
    lower = -dt * op.wf[1:-1]                     # M_{i,i-1}, i = 1..n-1 (= M_{i-1,i})
    diag = 1.0 + dt * (op.wf[:-1] + op.wf[1:] + op.reaction)
    piv = np.empty(n)
    lmul = np.zeros(n)
    piv[0] = diag[0]
    for i in range(1, n):
        lmul[i] = lower[i - 1] / piv[i - 1]
        piv[i] = diag[i] - lmul[i] * lower[i - 1]
    l32 = lmul.astype(dtype)
    u32 = np.concatenate([lower, [0.0]]).astype(dtype)   # M_{i,i+1}
    dinv32 = (1.0 / piv).astype(dtype)
    w = np.asarray(op.wf, dtype=dtype)
    c, f0, dtt = dtype(op.reaction), dtype(op.forcing), dtype(dt)

    def solve(rhs):
        y = np.empty_like(rhs)
        y[..., 0] = rhs[..., 0]
        for i in range(1, n):
            y[..., i] = rhs[..., i] - l32[i] * y[..., i - 1]
        x = np.empty_like(rhs)
        x[..., n - 1] = dinv32[n - 1] * y[..., n - 1]
        for i in range(n - 2, -1, -1):
            x[..., i] = dinv32[i] * (y[..., i] - u32[i] * x[..., i + 1])
        return x

    def flux_Av(v):
        z = np.zeros(v.shape[:-1] + (1,), dtype=dtype)
        vp = np.concatenate([z, v, z], axis=-1)
        q = w * (vp[..., 1:] - vp[..., :-1])      # w_f (v_f - v_{f-1}) at the n + 1 faces
        return -(q[..., 1:] - q[..., :-1]) + c * v

    v = np.asarray(V, dtype=dtype)
    d = None
    for m in range(J):
        if form == "direct":
            v = solve(v + dtt * f0)
        else:
            rhs = -dtt * flux_Av(v) + dtt * f0 if d is None or m % flux_every == 0 else d
            d = solve(rhs)
            v = v + d
        assert v.dtype == dtype
    return v.astype(np.float64)

