"""2D random reaction-diffusion problem (oracle).
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

PDE (eq. psys with f(u) = div(a grad u) - c u + f0) on (0,1)^2 with zero
Dirichlet values, five-point finite differences on an nx x nx interior grid,
h = 1/(nx+1), unknown (ix, iy) at (ix+1, iy+1) h stored at index iy*nx + ix.
The coefficient is sampled at the edge midpoints:
  ax[iy][fx], fx = 0..nx, at ((fx + 1/2) h, (iy + 1) h)   (x-faces)
  ay[fy][ix], fy = 0..nx, at ((ix + 1) h, (fy + 1/2) h)   (y-faces)
  (A u) = -[ax_{fx+1}(u_E - u) - ax_fx (u - u_W)]/h^2 - [ay_{fy+1}(u_N - u) - ay_fy (u - u_S)]/h^2 + c u.
a = exp(g), g the KL expansion of the separable exponential covariance
sigma^2 exp(-|x1-y1|/ell) exp(-|x2-y2|/ell) (products of the 1D modes).

Advection-diffusion (Section 5, advection-diffusion equation): the velocity
b(x) = b0 (x2, x1) (the paper's b0 = 0.1), which is >= 0 on the domain, adds
b . grad u by first-order upwind (here backward) differences,
  + b0 x2 (u - u_W)/h + b0 x1 (u - u_S)/h   at the cell (x1, x2),
so A is no longer symmetric.

Every linear solve is a sparse direct solve (SuperLU, scipy.sparse.linalg):
the exact backward-Euler step and the exact shifted CGC solve, which the
GPU approximates by preconditioned Krylov iterations to a tolerance.
This class offers the same methods as heat1d.Heat1D, so the parareal
functions of oracle.pcgc apply unchanged.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from . import kl_input


class RD2D:
    def __init__(self, ax: np.ndarray, ay: np.ndarray, reaction: float = 0.0,
                 forcing: float = 0.0, advection: float = 0.0):
        ax = np.asarray(ax, dtype=np.float64)
        ay = np.asarray(ay, dtype=np.float64)
        self.nx = ax.shape[0]
        nx = self.nx
        assert ax.shape == (nx, nx + 1) and ay.shape == (nx + 1, nx)
        self.h = 1.0 / (nx + 1)
        h2 = self.h ** 2
        n = nx * nx
        rows, cols, vals = [], [], []
        diag = np.full(n, float(reaction))
        for iy in range(nx):
            for ix in range(nx):
                k = iy * nx + ix
                wW, wE = ax[iy, ix] / h2, ax[iy, ix + 1] / h2
                wS, wN = ay[iy, ix] / h2, ay[iy + 1, ix] / h2
                diag[k] += wW + wE + wS + wN
                # upwind convection: b1 = b0 x2 >= 0 takes u_W, b2 = b0 x1 >= 0
                # takes u_S; b1/h = b0 (iy + 1), b2/h = b0 (ix + 1)
                c1 = advection * (iy + 1)
                c2 = advection * (ix + 1)
                diag[k] += c1 + c2
                if ix > 0:
                    rows.append(k); cols.append(k - 1); vals.append(-c1)
                if iy > 0:
                    rows.append(k); cols.append(k - nx); vals.append(-c2)
                if ix > 0:
                    rows.append(k); cols.append(k - 1); vals.append(-wW)
                if ix < nx - 1:
                    rows.append(k); cols.append(k + 1); vals.append(-wE)
                if iy > 0:
                    rows.append(k); cols.append(k - nx); vals.append(-wS)
                if iy < nx - 1:
                    rows.append(k); cols.append(k + nx); vals.append(-wN)
        rows += list(range(n)); cols += list(range(n)); vals += list(diag)
        self.A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
        self.forcing = float(forcing)
        self.reaction = float(reaction)
        self.advection = float(advection)
        self._lu = {}

    @property
    def n(self) -> int:
        return self.nx * self.nx

    def apply(self, V):
        V = np.asarray(V)
        return (self.A @ V.reshape(-1, self.n).T).T.reshape(V.shape)

    def dense(self):
        return self.A.toarray()

    def shifted_solve(self, shift, scale, R):
        key = (complex(shift), float(scale))
        if key not in self._lu:
            M = (shift * sp.identity(self.n, format="csc") + scale * self.A.tocsc())
            self._lu[key] = splu(M.astype(np.result_type(shift, np.float64)).tocsc())
        R = np.asarray(R)
        flat = R.reshape(-1, self.n)
        out = np.stack([self._lu[key].solve(np.ascontiguousarray(r)) for r in flat])
        return out.reshape(R.shape)

    def be_step(self, V, dt):
        return self.shifted_solve(1.0, dt, V + dt * self.forcing)


def face_points(nx: int):
    """(x1, x2) of the x-faces [nx][nx+1] and of the y-faces [nx+1][nx]."""
    h = 1.0 / (nx + 1)
    fx = (np.arange(nx + 1) + 0.5) * h
    iy = (np.arange(nx) + 1) * h
    X1x, X2x = np.meshgrid(fx, iy)              # [nx][nx+1]
    ix = (np.arange(nx) + 1) * h
    fy = (np.arange(nx + 1) + 0.5) * h
    X1y, X2y = np.meshgrid(ix, fy)              # [nx+1][nx]
    return (X1x, X2x), (X1y, X2y)


def field_basis_2d(sigma: float, corr_len: float, M: int, pts):
    """Rows sqrt(lambda_m) phi_i(x1) phi_j(x2) of the top-M separable modes at pts."""
    pairs, (lam1, om1, par1) = kl_input.modes_2d(sigma, corr_len, M)
    X1, X2 = pts
    out = []
    for lam, i, j in pairs:
        out.append(math.sqrt(lam) * kl_input.exp_cov_phi_1d(X1, om1[i], par1[i])
                   * kl_input.exp_cov_phi_1d(X2, om1[j], par1[j]))
    return np.stack(out)
