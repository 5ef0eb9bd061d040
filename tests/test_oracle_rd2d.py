"""Pins of the 2D reaction-diffusion oracle against closed forms and brute force."""
import math

import numpy as np
import pytest

from oracle import pcgc, rd2d


def _op(nx, const=False, reaction=0.0, forcing=0.0, seed=0, advection=0.0):
    rng = np.random.default_rng(seed)
    ax = np.ones((nx, nx + 1)) if const else np.exp(0.4 * rng.standard_normal((nx, nx + 1)))
    ay = np.ones((nx + 1, nx)) if const else np.exp(0.4 * rng.standard_normal((nx + 1, nx)))
    return rd2d.RD2D(ax, ay, reaction, forcing, advection)


def test_five_point_spectrum_and_eigenvector():
    # a == 1: mu_jk = (4/h^2)(sin^2(j pi h/2) + sin^2(k pi h/2)) + c, eigvec sin(j pi x) sin(k pi y)
    nx, c = 9, 0.6
    op = _op(nx, const=True, reaction=c)
    h = op.h
    s = 4 / h ** 2 * np.sin(np.arange(1, nx + 1) * np.pi * h / 2) ** 2
    mu = np.sort((s[:, None] + s[None, :]).ravel() + c)
    assert np.allclose(np.sort(np.linalg.eigvalsh(op.dense())), mu, rtol=1e-12)
    x = (np.arange(nx) + 1) * h
    v = np.outer(np.sin(2 * np.pi * x), np.sin(np.pi * x)).ravel()   # [iy][ix]: y-mode 2, x-mode 1
    lam = s[0] + s[1] + c
    assert np.allclose(op.apply(v), lam * v, rtol=1e-11, atol=1e-9)
    # one backward-Euler step scales it by 1/(1 + dt lam)
    assert np.allclose(op.be_step(v, 0.01), v / (1 + 0.01 * lam), rtol=1e-12)


def test_operator_symmetric_and_matches_stencil_definition():
    op = _op(6, seed=3, reaction=1.0)
    A = op.dense()
    assert np.allclose(A, A.T)
    # row sums: reaction c plus the boundary-face weights (interior faces cancel)
    nx, h2 = op.nx, op.h ** 2
    rng = np.random.default_rng(3)
    ax = np.exp(0.4 * rng.standard_normal((nx, nx + 1)))
    ay = np.exp(0.4 * rng.standard_normal((nx + 1, nx)))
    bnd = np.zeros((nx, nx))
    bnd[:, 0] += ax[:, 0]
    bnd[:, -1] += ax[:, -1]
    bnd[0, :] += ay[0, :]
    bnd[-1, :] += ay[-1, :]
    assert np.allclose(A.sum(1), 1.0 + bnd.ravel() / h2)


@pytest.mark.parametrize("advection", [0.0, 3.0])
def test_three_step_solve_equals_dense_kron_solve_2d(advection):
    op = _op(3, seed=4, reaction=1.0, advection=advection)
    N, alpha, dT = 4, 1e-2, 0.25
    r = np.random.default_rng(1).standard_normal((N, op.n))
    assert np.allclose(pcgc.cgc_diagonalized(op, r, dT, alpha), pcgc.cgc_dense(op, r, dT, alpha),
                       rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("advection", [0.0, 3.0])
def test_pcgc_reaches_fine_solution_2d(advection):
    op = _op(5, seed=5, reaction=1.0, forcing=1.0, advection=advection)
    N, J = 6, 3
    u0 = np.zeros(op.n)
    from oracle import heat1d
    Ustar = heat1d.fine_sequential(op, u0, N, J, 1.0)
    U, its, _ = pcgc.pcgc_solve(op, u0, np.zeros((N, op.n)), 1.0 / N, J, 1e-3, 1e-13, 60)
    assert its > 0 and np.max(np.abs(U - Ustar)) < 1e-12


def test_face_points_and_2d_basis_products():
    (X1x, X2x), (X1y, X2y) = rd2d.face_points(4)
    h = 0.2
    assert np.allclose(X1x[0], (np.arange(5) + 0.5) * h) and np.allclose(X2x[:, 0], (np.arange(4) + 1) * h)
    assert np.allclose(X1y[0], (np.arange(4) + 1) * h) and np.allclose(X2y[:, 0], (np.arange(5) + 0.5) * h)
    B = rd2d.field_basis_2d(0.4, 0.3, 3, (X1x, X2x))
    from oracle import kl_input
    pairs, (lam1, om1, par1) = kl_input.modes_2d(0.4, 0.3, 3)
    lam, i, j = pairs[1]
    ref = math.sqrt(lam) * kl_input.exp_cov_phi_1d(X1x, om1[i], par1[i]) * kl_input.exp_cov_phi_1d(X2x, om1[j], par1[j])
    assert np.allclose(B[1], ref)


def test_upwind_advection_is_exact_on_linear_functions():
    # a = 1, b = b0 (x2, x1): the five-point Laplacian of x1 (x2) vanishes and
    # the backward differences of a linear function are exact, so away from
    # the boundary rows where the zero Dirichlet value differs from it,
    # A x1 = b0 x2 and A x2 = b0 x1.
    nx, b0 = 9, 2.5
    op = _op(nx, const=True, advection=b0)
    x = (np.arange(nx) + 1) * op.h
    X1, X2 = np.meshgrid(x, x)          # [iy][ix]
    A1 = op.apply(X1.ravel()).reshape(nx, nx)
    assert np.allclose(A1[1:-1, :-1], (b0 * X2)[1:-1, :-1], rtol=1e-12, atol=1e-10)
    A2 = op.apply(X2.ravel()).reshape(nx, nx)
    assert np.allclose(A2[:-1, 1:-1], (b0 * X1)[:-1, 1:-1], rtol=1e-12, atol=1e-10)
    # the skew part comes from the convection alone
    A0 = _op(nx, const=True).dense()
    assert np.allclose(A0, A0.T)
    assert not np.allclose(op.dense(), op.dense().T)


def test_advection_diffusion_converges_to_the_manufactured_solution():
    # a = 1: -lap u + b . grad u = f for u = sin(pi x1) sin(2 pi x2); upwind
    # convection is first order, so the error halves with h
    b0, errs = 5.0, []
    from scipy.sparse.linalg import spsolve
    for nx in (15, 31, 63):
        op = _op(nx, const=True, advection=b0)
        x = (np.arange(nx) + 1) * op.h
        X1, X2 = np.meshgrid(x, x)
        u = np.sin(np.pi * X1) * np.sin(2 * np.pi * X2)
        f = (5 * np.pi ** 2 * u + b0 * X2 * np.pi * np.cos(np.pi * X1) * np.sin(2 * np.pi * X2)
             + b0 * X1 * 2 * np.pi * np.sin(np.pi * X1) * np.cos(2 * np.pi * X2))
        errs.append(np.max(np.abs(spsolve(op.A.tocsc(), f.ravel()) - u.ravel())))
    assert errs[0] < 0.1
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.7 < e1 / e2 < 2.3, errs


def test_field_basis_2d_rebuilds_the_separable_covariance():
    # Mercer for the separable kernel sigma^2 exp(-|x1-y1|/ell - |x2-y2|/ell):
    # the top-400 product modes rebuild it to ~4e-5 between distinct points and
    # to the (slower) truncation tail on the diagonal.  A lambda for
    # sqrt(lambda), a dropped sigma or a unit-variance mix-up is off by ~sigma^2.
    from oracle import rd2d
    sigma, ell, M = 0.3, 0.3, 400
    P1 = np.array([0.1, 0.2, 0.5, 0.9, 0.33])
    P2 = np.array([0.7, 0.2, 0.5, 0.1, 0.61])
    B = rd2d.field_basis_2d(sigma, ell, M, (P1[None, :], P2[None, :])).reshape(M, -1)
    C = B.T @ B
    exact = sigma ** 2 * np.exp(-np.abs(P1[:, None] - P1[None, :]) / ell
                                - np.abs(P2[:, None] - P2[None, :]) / ell)
    err = np.abs(C - exact)
    assert err[~np.eye(5, dtype=bool)].max() < 2e-4
    assert err.max() < 0.1 * sigma ** 2


def test_variable_coefficient_2d_operator_is_second_order_consistent():
    # A u against -div(a grad u) for u = sin(pi x1) sin(2 pi x2) and a sample's
    # separable-KL field: with a at the edge midpoints the five-point flux form
    # is O(h^2) (ratio 4 per halving of h); x-faces shifted by h/2 give ~2.
    # Pins the face points of both directions, the index order (rows are x2)
    # and the flux signs with a non-constant coefficient.
    from synth import draw_xi, workload
    from oracle.klecgc import Setup2D
    errs = []
    for nx in (15, 31, 63):
        w = workload("ade2d_nx19", nx=nx, advection=0.0)
        st = Setup2D(w, build=False)
        xi = 2.0 * draw_xi(1, w.M, 6)[0]
        op = st.operator(xi)
        x = (np.arange(nx) + 1) / (nx + 1)
        X1, X2 = np.meshgrid(x, x)
        u = np.sin(np.pi * X1) * np.sin(2 * np.pi * X2)
        Au = (op.apply(u.ravel()) - op.reaction * u.ravel()).reshape(nx, nx)

        def a_of(P1, P2):
            B = rd2d.field_basis_2d(w.sigma, w.corr_len, w.M, (P1, P2))
            return np.exp(np.tensordot(xi, B, axes=1))

        d = 1e-5
        a1 = (a_of(X1 + d, X2) - a_of(X1 - d, X2)) / (2 * d)
        a2 = (a_of(X1, X2 + d) - a_of(X1, X2 - d)) / (2 * d)
        u1 = np.pi * np.cos(np.pi * X1) * np.sin(2 * np.pi * X2)
        u2 = 2 * np.pi * np.sin(np.pi * X1) * np.cos(2 * np.pi * X2)
        exact = -(a1 * u1 + a2 * u2 - 5 * np.pi ** 2 * a_of(X1, X2) * u)
        errs.append(np.abs(Au - exact).max() / np.abs(exact).max())
    assert errs[-1] < 2e-3
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 < e1 / e2 < 4.4, errs
