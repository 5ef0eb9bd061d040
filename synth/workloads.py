"""Workload descriptors and seeded xi draws.

Every random input of the method is a KL coefficient vector xi ~ N(0, I_M)
(the entries of xi are i.i.d., Section 2).  Draws use
``numpy.random.default_rng(seed).standard_normal``; the same bytes feed the
oracle and the CUDA path.  The training set Xi_t of Algorithm 3 comes from a
separate seed so that it never overlaps the evaluation batch.

Workload names describe what they are:

* ``heat1d_nx63``   1D random-diffusion heat equation, Nx=63, N=16, J=16,
                    M=4, total-degree-2 Hermite gPC, alpha=1e-3, 32 samples.
* ``heat1d_nx1023`` same PDE at Nx=1023, N=64, J=64, M=10, degree 3,
                    alpha=1e-4, 4096 samples (FP64 and mixed precision).
* ``rd2d_255``      2D reaction-diffusion on a 255x255 grid, N=32, J=32,
                    M=20 separable KL, degree 2, 1024 samples.
* ``ade2d_nx19``    2D advection-diffusion u_t = div(a grad u) - b . grad u + 1,
                    b = 0.1 (x2, x1) (upwind), u0 = sin(pi x1) sin(2 pi x2),
                    h = 1/20, T=1, N=32, J=50, M=4 separable KL, degree 2,
                    1024 samples (the paper's advection-diffusion set-up,
                    Section 5, with a KL-random diffusion).
* ``heat1d_uneven`` 8192 1D instances with Nx, N, J drawn per instance.
* ``ac1d_nx127``    1D Allen-Cahn-type problem (cubic reaction, random
                    diffusion), Nx=127, N=32, J=16, 256 samples.
* ``burgers1d_nx99`` 1D Burgers-type problem u_t + 25 (u^2/2)_x = (a u_x)_x
                    (upwind convection, random diffusion), Nx=99, T=0.08,
                    N=32, J=40, 256 samples, |Xi_t| = 36 (the paper's Burgers
                    set-up, Section 5, rescaled in time by its mean viscosity).
* ``mlp_guess``     learned-guess workload on the heat1d_nx1023 problem.

Values the paper leaves open are fixed here (training-set size n_t = 2P,
eps_KL = 1e-10 as in every experiment of Section 5, tol = 1e-8).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int            # 1 or 2 space dimensions
    nx: int             # interior points per direction
    T: float
    N: int              # coarse intervals
    J: int              # fine backward-Euler steps per coarse interval
    sigma: float        # std-dev of the Gaussian field g, a = exp(g)
    corr_len: float     # correlation length of exp(-|x-y|/corr_len)
    M: int              # input KL terms kept
    gpc_degree: int     # total degree p of the Hermite gPC basis
    n_train: int        # |Xi_t| = 2P
    eps_kl: float       # snapshot-KL energy tolerance
    alpha: float        # alpha of the twisted coarse problem u(0) = alpha u(T)
    tol: float          # per-sample increment tolerance (stopping rule)
    S: int              # evaluation samples
    seed: int           # seed of the evaluation xi batch
    train_seed: int     # seed of the training set Xi_t
    reaction: float = 0.0   # c in u_t = div(a grad u) - c u + f
    forcing: float = 0.0    # f (constant)
    u0_kind: int = 0        # 0: sin(pi x) (1D) / product of sines (2D); 1: zero;
                            # 2 (2D): sin(pi x1) sin(2 pi x2)
    kmax: int = 60
    extra: dict = field(default_factory=dict)
    reaction_kind: int = 0  # 0: linear c u; 1: cubic c (u^3 - u) (Allen-Cahn type);
                            # 2: convection c (u^2/2)_x (Burgers type)
    cgc_newton: int = 1     # simplified Newton steps per CGC (nonlinear problems)
    advection: float = 0.0  # b0 of the 2D velocity b = b0 (x2, x1) (upwind)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


WORKLOADS = {
    "heat1d_nx63": Workload(
        name="heat1d_nx63", dim=1, nx=63, T=1.0, N=16, J=16, sigma=0.5,
        corr_len=0.5, M=4, gpc_degree=2, n_train=30, eps_kl=1e-10,
        alpha=1e-3, tol=1e-8, S=32, seed=1, train_seed=101),
    "heat1d_nx1023": Workload(
        name="heat1d_nx1023", dim=1, nx=1023, T=1.0, N=64, J=64, sigma=0.5,
        corr_len=0.5, M=10, gpc_degree=3, n_train=572, eps_kl=1e-10,
        alpha=1e-4, tol=1e-8, S=4096, seed=2, train_seed=102),
    "rd2d_255": Workload(
        name="rd2d_255", dim=2, nx=255, T=1.0, N=32, J=32, sigma=0.4,
        corr_len=0.3, M=20, gpc_degree=2, n_train=462, eps_kl=1e-10,
        alpha=1e-3, tol=1e-8, S=1024, seed=3, train_seed=103,
        reaction=1.0, forcing=1.0, u0_kind=1),
    "ade2d_nx19": Workload(
        name="ade2d_nx19", dim=2, nx=19, T=1.0, N=32, J=50, sigma=0.3,
        corr_len=0.3, M=4, gpc_degree=2, n_train=30, eps_kl=1e-10,
        alpha=1e-3, tol=1e-8, S=1024, seed=9, train_seed=109,
        reaction=0.0, forcing=1.0, u0_kind=2, advection=0.1),
    "heat1d_uneven": Workload(
        name="heat1d_uneven", dim=1, nx=1023, T=1.0, N=64, J=64, sigma=0.5,
        corr_len=0.5, M=10, gpc_degree=3, n_train=572, eps_kl=1e-10,
        alpha=1e-4, tol=1e-8, S=8192, seed=4, train_seed=104,
        extra=dict(nx_choices=(127, 255, 511, 1023, 2047),
                   N_choices=(16, 32, 64), J_choices=(8, 16, 32, 64, 128))),
    "ac1d_nx127": Workload(
        name="ac1d_nx127", dim=1, nx=127, T=8.0, N=32, J=16, sigma=0.3,
        corr_len=0.3, M=6, gpc_degree=2, n_train=56, eps_kl=1e-10,
        alpha=1e-3, tol=1e-8, S=256, seed=7, train_seed=107,
        reaction=5.0, forcing=0.0, u0_kind=0, reaction_kind=1, cgc_newton=3),
    "burgers1d_nx99": Workload(
        name="burgers1d_nx99", dim=1, nx=99, T=0.08, N=32, J=40, sigma=0.3,
        corr_len=0.3, M=4, gpc_degree=2, n_train=36, eps_kl=1e-10,
        alpha=1e-3, tol=1e-8, S=256, seed=8, train_seed=108,
        reaction=25.0, forcing=0.0, u0_kind=0, reaction_kind=2, cgc_newton=3),
    "mlp_guess": Workload(
        name="mlp_guess", dim=1, nx=1023, T=1.0, N=64, J=64, sigma=0.5,
        corr_len=0.5, M=10, gpc_degree=3, n_train=572, eps_kl=1e-10,
        alpha=1e-4, tol=1e-8, S=4096, seed=6, train_seed=102,
        extra=dict(mlp_width=256, mlp_out_points=64, mlp_train=16384,
                   mlp_train_seed=5)),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return w.with_(**overrides) if overrides else w


def draw_xi(S: int, M: int, seed: int) -> np.ndarray:
    """S i.i.d. standard-normal KL coefficient vectors, shape [S, M], float64."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((S, M)), dtype=np.float64)


def draw_train(w: Workload) -> np.ndarray:
    """The training set Xi_t of Algorithm 3: n_train draws from train_seed."""
    return draw_xi(w.n_train, w.M, w.train_seed)


def draw_uneven_shapes(w: Workload) -> np.ndarray:
    """Per-instance (Nx, N, J) for the uneven batch, drawn in that order."""
    rng = np.random.default_rng(w.seed)
    e = w.extra
    nx = rng.choice(np.asarray(e["nx_choices"]), size=w.S)
    N = rng.choice(np.asarray(e["N_choices"]), size=w.S)
    J = rng.choice(np.asarray(e["J_choices"]), size=w.S)
    return np.stack([nx, N, J], axis=1).astype(np.int32)
