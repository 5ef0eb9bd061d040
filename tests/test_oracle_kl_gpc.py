"""Pins of the oracle's input KL and gPC basis against closed forms,
independent discretizations and quadrature (no GPU)."""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e, legendre

from oracle import gpc, kl_input


@pytest.mark.parametrize("ell", [0.3, 0.5, 1.0])
def test_kl_roots_solve_transcendental_equations(ell):
    lam, om, par = kl_input.exp_cov_modes_1d(ell, 12, sigma=1.0)
    c = 1.0 / ell
    for w, p in zip(om, par):
        # residual relative to the size of the terms in the equation
        res = kl_input.transcendental_residual(w, p, ell)
        scale = c + w * abs(math.tan(w / 2)) + w
        assert abs(res) <= 1e-12 * scale
    # one root per half period of tan(w/2), alternating even/odd
    assert np.all(np.diff(om) > 0)
    assert list(par[:6]) == [0, 1, 0, 1, 0, 1]
    assert np.all(np.diff(lam) < 0)


@pytest.mark.parametrize("ell,sigma", [(0.5, 0.5), (0.3, 0.4)])
def test_kl_eigenvalues_match_nystrom(ell, sigma):
    # independent discretization: midpoint-rule Nystrom matrix of the kernel
    n = 3000
    x = (np.arange(n) + 0.5) / n
    K = sigma ** 2 * np.exp(-np.abs(x[:, None] - x[None, :]) / ell) / n
    ev = np.sort(np.linalg.eigvalsh(K))[::-1][:8]
    lam, _, _ = kl_input.exp_cov_modes_1d(ell, 8, sigma)
    assert np.allclose(ev, lam, rtol=2e-4, atol=0)


def test_kl_eigenfunctions_orthonormal_and_are_eigenfunctions():
    ell, sigma = 0.5, 0.5
    lam, om, par = kl_input.exp_cov_modes_1d(ell, 6, sigma)
    # split Gauss-Legendre quadrature on [0,1] (smooth integrands)
    g, gw = legendre.leggauss(80)
    xs = 0.5 * (g + 1)
    ws = 0.5 * gw
    Phi = np.stack([kl_input.exp_cov_phi_1d(xs, om[m], par[m]) for m in range(6)])
    Gram = (Phi * ws) @ Phi.T
    assert np.allclose(Gram, np.eye(6), atol=1e-12)
    # integral eigen-equation at a few points, integrand has a kink at y = x0
    for x0 in (0.1, 0.37, 0.8):
        for m in range(3):
            tot = 0.0
            for lo, hi in ((0.0, x0), (x0, 1.0)):
                ys = lo + (hi - lo) * 0.5 * (g + 1)
                wy = (hi - lo) * 0.5 * gw
                k = sigma ** 2 * np.exp(-np.abs(x0 - ys) / ell)
                tot += np.sum(wy * k * kl_input.exp_cov_phi_1d(ys, om[m], par[m]))
            assert abs(tot - lam[m] * kl_input.exp_cov_phi_1d(x0, om[m], par[m])) < 1e-12


def test_kl_trace_equals_variance():
    # sum of all eigenvalues = integral of C(x, x) = sigma^2; tail ~ 2c sigma^2 / (pi^2 K)
    sigma, ell = 0.5, 0.5
    lam, _, _ = kl_input.exp_cov_modes_1d(ell, 4000, sigma)
    c = 1 / ell
    tail = 2 * c * sigma ** 2 / (math.pi ** 2 * 4000)
    gap = sigma ** 2 - lam.sum()
    assert 0 < gap < 1.5 * tail


def test_kl_2d_modes_are_products_sorted():
    pairs, (lam1, _, _) = kl_input.modes_2d(0.4, 0.3, 20)
    lams = [p[0] for p in pairs]
    assert np.all(np.diff(lams) <= 1e-15)
    assert pairs[0][1:] == (0, 0)
    assert math.isclose(pairs[0][0], 0.16 * lam1[0] ** 2, rel_tol=1e-14)
    # ties (i, j) / (j, i) are adjacent with i + j equal and i ascending
    assert pairs[1][1:] == (0, 1) and pairs[2][1:] == (1, 0)


@pytest.mark.parametrize("M,p,P", [(4, 2, 15), (10, 3, 286), (20, 2, 231)])
def test_gpc_basis_count(M, p, P):
    idx = gpc.multi_indices(M, p)
    assert idx.shape == (P, M)
    assert len({tuple(k) for k in idx}) == P
    assert np.all(idx.sum(1) <= p)
    assert np.all(np.diff(idx.sum(1)) >= 0)
    assert math.comb(p + M, M) == P


def test_univariate_hermite_matches_numpy_hermite_e():
    x = np.linspace(-4, 4, 41)
    vals = gpc.hermite_orthonormal(6, x)
    for k in range(7):
        c = np.zeros(k + 1)
        c[k] = 1
        assert np.allclose(vals[k], hermite_e.hermeval(x, c) / math.sqrt(math.factorial(k)),
                           rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M,p", [(3, 4), (4, 2), (2, 5)])
def test_gpc_orthonormal_by_gauss_hermite(M, p):
    # tensor Gauss-Hermite (probabilists') rule exact for degree <= 2q-1 per dim
    q = p + 1
    z, wz = hermite_e.hermegauss(q)
    wz = wz / math.sqrt(2 * math.pi)
    grids = np.meshgrid(*([z] * M), indexing="ij")
    pts = np.stack([g.ravel() for g in grids], axis=1)
    wgrid = np.meshgrid(*([wz] * M), indexing="ij")
    w = np.prod(np.stack([g.ravel() for g in wgrid], axis=1), axis=1)
    B = gpc.psi_matrix(pts, p)
    Gram = (B * w[:, None]).T @ B
    assert np.allclose(Gram, np.eye(B.shape[1]), atol=1e-12)


def test_field_basis_rebuilds_the_covariance_kernel():
    # Mercer: sum_m sqrt(lam_m) phi_m(x) sqrt(lam_m) phi_m(y) -> sigma^2 exp(-|x-y|/ell)
    # uniformly on [0,1]; the truncation error at K modes is at most
    # max|phi|^2 * (tail of sum lam) <= 2 * 2 c sigma^2 / (pi^2 K).  Pins the
    # sqrt(lambda) scaling, the normalization of phi and the [0,1] placement.
    sigma, ell, K = 0.3, 0.3, 2000
    x = np.array([0.0, 0.05, 0.3, 0.5, 0.77, 1.0])
    B = kl_input.field_basis_1d(sigma, ell, K, x)
    C = B.T @ B
    exact = sigma ** 2 * np.exp(-np.abs(x[:, None] - x[None, :]) / ell)
    tail = 2 * 2 * sigma ** 2 / (ell * math.pi ** 2 * K)
    err = np.abs(C - exact)
    assert err.max() < 1.5 * tail
    assert err[~np.eye(len(x), dtype=bool)].max() < 1e-6
