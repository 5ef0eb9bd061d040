"""End-to-end KLE-PCGC on a workload (oracle): setup + per-sample solves.
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

setup(w, xi_train)  input-KL basis at the faces, sequential fine snapshots of
                    the training set, surrogate (Algorithm 3 offline part)
solve_sample(...)   Algorithm 2 from the surrogate guess (Algorithm 3 online)
error metrics       relative L2 error vs U* per sample; the paper's mean
                    infinity-norm error per coarse point (Section 5).
"""
from __future__ import annotations

import numpy as np

from . import kl_input, heat1d, pcgc
from .surrogate import build_surrogate


def _reference_worker(args):
    w, xi = args
    st = Setup1D(w, build=False)
    return st.reference(xi).reshape(-1)


class Setup1D:
    def __init__(self, w, xi_train=None, build=True, processes=1):
        from synth import draw_train
        self.w = w
        nx = w.nx
        h = 1.0 / (nx + 1)
        self.faces = (np.arange(nx + 1) + 0.5) * h
        self.basis = kl_input.field_basis_1d(w.sigma, w.corr_len, w.M, self.faces)
        self.u0 = heat1d.u0_sine(nx) if w.u0_kind == 0 else np.zeros(nx)
        self.dT = w.T / w.N
        if xi_train is None:
            xi_train = draw_train(w)
        self.xi_train = xi_train
        self.sur = None
        if build:
            snaps = self.references(xi_train, processes)
            self.snaps = snaps.reshape(len(xi_train), -1)
            self.sur = build_surrogate(self.snaps, xi_train, w.gpc_degree, w.eps_kl)

    def surrogate_svd(self):
        """The same surrogate with the snapshot eigenpairs from an SVD."""
        return build_surrogate(self.snaps, self.xi_train, self.w.gpc_degree, self.w.eps_kl,
                               eig="svd")

    def references(self, xis, processes=1) -> np.ndarray:
        """U*(xi) for each row of xis, [S, N, nx]; optional spawn process pool."""
        if processes <= 1 or len(xis) < 2:
            return np.stack([self.reference(x) for x in xis])
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_reference_worker, [(self.w, x) for x in xis],
                              chunksize=max(1, len(xis) // (4 * processes))))
        return np.stack(out).reshape(len(xis), self.w.N, self.w.nx)

    def operator(self, xi, field_ulps: float = 0.0, seed: int = 0) -> heat1d.Heat1D:
        """Operator of sample xi.  field_ulps > 0 multiplies every face value by
        (1 +- field_ulps * 2^-53) with random signs: a model of the rounding of
        an independently computed field, used to measure how strongly a result
        depends on the last bits of a."""
        a = np.exp(kl_input.log_coefficient_1d(xi, self.basis))
        if field_ulps:
            sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=a.shape)
            a = a * (1.0 + field_ulps * 2.0 ** -53 * sgn)
        return heat1d.Heat1D(a, self.w.reaction, self.w.forcing)

    def reference(self, xi) -> np.ndarray:
        """U*(xi): sequential fine solution, [N, nx]."""
        return heat1d.fine_sequential(self.operator(xi), self.u0, self.w.N,
                                      self.w.J, self.w.T)

    def guess(self, xi) -> np.ndarray:
        return self.sur.guess(np.atleast_2d(xi)).reshape(-1, self.w.N, self.w.nx)

    def solve_sample(self, xi, U0=None, kmax=None, history=False, cgc="diag", field_ulps=0.0):
        w = self.w
        if U0 is None:
            U0 = self.guess(xi)[0]
        op = self.operator(xi, field_ulps)
        return pcgc.pcgc_solve(op, self.u0, U0, self.dT, w.J, w.alpha, w.tol,
                               kmax or w.kmax, history=history, cgc=cgc)


def _reference_worker_2d(args):
    w, xi = args
    st = Setup2D(w, build=False)
    return st.reference(xi).reshape(-1)


class Setup2D(Setup1D):
    """Same stages as Setup1D on the 2D reaction-(advection-)diffusion problem
    (rd2d)."""

    def __init__(self, w, xi_train=None, build=True, processes=1):
        from synth import draw_train
        from . import rd2d
        self.w = w
        nx = w.nx
        self.xpts, self.ypts = rd2d.face_points(nx)
        self.bx = rd2d.field_basis_2d(w.sigma, w.corr_len, w.M, self.xpts)
        self.by = rd2d.field_basis_2d(w.sigma, w.corr_len, w.M, self.ypts)
        x = (np.arange(nx) + 1) / (nx + 1)
        if w.u0_kind == 0:
            self.u0 = np.outer(np.sin(np.pi * x), np.sin(np.pi * x)).reshape(-1)
        elif w.u0_kind == 2:
            # sin(pi x1) sin(2 pi x2), index iy*nx + ix (rows are x2)
            self.u0 = np.outer(np.sin(2 * np.pi * x), np.sin(np.pi * x)).reshape(-1)
        else:
            self.u0 = np.zeros(nx * nx)
        self.dT = w.T / w.N
        if xi_train is None:
            xi_train = draw_train(w)
        self.xi_train = xi_train
        self.sur = None
        if build:
            snaps = self.references(xi_train, processes)
            self.sur = build_surrogate(snaps.reshape(len(xi_train), -1), xi_train,
                                       w.gpc_degree, w.eps_kl)

    def operator(self, xi, field_ulps: float = 0.0, seed: int = 0):
        from . import rd2d
        ax = np.exp(np.tensordot(np.asarray(xi, dtype=np.float64), self.bx, axes=1))
        ay = np.exp(np.tensordot(np.asarray(xi, dtype=np.float64), self.by, axes=1))
        if field_ulps:
            rng = np.random.default_rng(seed)
            ax = ax * (1.0 + field_ulps * 2.0 ** -53 * rng.choice([-1.0, 1.0], size=ax.shape))
            ay = ay * (1.0 + field_ulps * 2.0 ** -53 * rng.choice([-1.0, 1.0], size=ay.shape))
        return rd2d.RD2D(ax, ay, self.w.reaction, self.w.forcing,
                         getattr(self.w, "advection", 0.0))

    def references(self, xis, processes=1) -> np.ndarray:
        if processes <= 1 or len(xis) < 2:
            return np.stack([self.reference(x) for x in xis])
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_reference_worker_2d, [(self.w, x) for x in xis]))
        return np.stack(out).reshape(len(xis), self.w.N, -1)

    def guess(self, xi) -> np.ndarray:
        return self.sur.guess(np.atleast_2d(xi)).reshape(-1, self.w.N, self.w.nx * self.w.nx)


def _reference_worker_ac(args):
    w, xi = args
    st = SetupAC1D(w, build=False)
    return st.reference(xi).reshape(-1)


class SetupAC1D(Setup1D):
    """Same stages as Setup1D on the nonlinear problems of oracle.nonlinear
    (w.reaction_kind 1: Allen-Cahn-type reaction, 2: Burgers-type
    convection): Newton backward-Euler propagators and the simplified-Newton
    CGC with w.cgc_newton steps."""

    def operator(self, xi, field_ulps: float = 0.0, seed: int = 0):
        from . import nonlinear
        a = np.exp(kl_input.log_coefficient_1d(xi, self.basis))
        if field_ulps:
            sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=a.shape)
            a = a * (1.0 + field_ulps * 2.0 ** -53 * sgn)
        cls = nonlinear.BurgersEO1D if self.w.reaction_kind == 2 else nonlinear.CubicRD1D
        return cls(a, self.w.reaction, self.w.forcing)

    def reference(self, xi) -> np.ndarray:
        from . import nonlinear
        return nonlinear.fine_sequential(self.operator(xi), self.u0, self.w.N, self.w.J,
                                         self.w.T)

    def references(self, xis, processes=1) -> np.ndarray:
        if processes <= 1 or len(xis) < 2:
            return np.stack([self.reference(x) for x in xis])
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_reference_worker_ac, [(self.w, x) for x in xis]))
        return np.stack(out).reshape(len(xis), self.w.N, self.w.nx)

    def solve_sample(self, xi, U0=None, kmax=None, history=False, cgc="diag", field_ulps=0.0):
        from . import nonlinear
        w = self.w
        if U0 is None:
            U0 = self.guess(xi)[0]
        op = self.operator(xi, field_ulps)
        U, k = nonlinear.pcgc_solve(op, self.u0, U0, self.dT, w.J, w.alpha, w.tol,
                                    kmax or w.kmax, w.cgc_newton, dense=(cgc == "dense"))
        return U, k, None


def rel_l2(U, Uref) -> float:
    return float(np.linalg.norm(np.ravel(U) - np.ravel(Uref)) /
                 np.linalg.norm(np.ravel(Uref)))


def mean_inf_error(Uref_batch, U_batch) -> np.ndarray:
    """e_n = (1/S) sum_i ||u_n(xi_i) - U_n(xi_i)||_inf, n = 1..N (Section 5)."""
    d = np.abs(np.asarray(Uref_batch) - np.asarray(U_batch))
    return d.max(axis=-1).mean(axis=0)
