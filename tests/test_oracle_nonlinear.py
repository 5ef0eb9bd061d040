"""Pins of the nonlinear oracle (Allen-Cahn-type reaction, simplified-Newton CGC)."""
import numpy as np

from oracle import heat1d, nonlinear as nl, pcgc


def _op(nx=24, c=5.0, f0=0.0, seed=0):
    a = np.exp(0.3 * np.random.default_rng(seed).standard_normal(nx + 1))
    return nl.CubicRD1D(a, c, f0), a


def test_newton_step_solves_the_backward_euler_equation():
    op, _ = _op(c=5.0, f0=0.7)
    v = np.sin(np.pi * op.grid()) * 1.3
    for dt in (1e-3, 0.05, 0.3):
        w = op.be_step_newton(v, dt)
        res = w + dt * op.apply(w) + dt * op.c * (w ** 3 - w) - v - dt * op.forcing
        assert np.max(np.abs(res)) < 1e-13 * max(1.0, np.max(np.abs(w)))


def test_zero_reaction_reduces_to_the_linear_oracle():
    op, a = _op(c=0.0, f0=0.4, seed=1)
    lin = heat1d.Heat1D(a, 0.0, 0.4)
    u0 = heat1d.u0_sine(op.nx)
    N, J, dT, alpha = 8, 4, 0.125, 1e-2
    U = np.random.default_rng(2).standard_normal((N, op.nx))
    assert np.allclose(nl.G(op, U, dT), heat1d.G(lin, U, dT), rtol=1e-13, atol=1e-14)
    starts = np.vstack([u0, U[:-1]])
    Fn = nl.F(op, starts, dT, J)
    assert np.allclose(Fn, heat1d.F(lin, starts, dT, J), rtol=1e-13, atol=1e-14)
    b = nl.jump_b(op, Fn, U, dT, alpha)
    ref = pcgc.cgc_diagonalized(lin, pcgc.cgc_rhs(lin, U, b, dT), dT, alpha)
    assert np.allclose(nl.cgc_newton_step(op, U, b, dT, alpha), ref, rtol=1e-11, atol=1e-12)


def test_newton_step_diagonalized_equals_dense():
    op, _ = _op(nx=10, c=3.0, f0=0.2, seed=3)
    N, dT, alpha = 4, 0.2, 1e-2
    rng = np.random.default_rng(4)
    u, b = rng.standard_normal((N, op.nx)), 0.1 * rng.standard_normal((N, op.nx))
    assert np.allclose(nl.cgc_newton_step(op, u, b, dT, alpha),
                       nl.cgc_newton_dense(op, u, b, dT, alpha), rtol=1e-10, atol=1e-12)


def test_simplified_newton_converges_to_the_cgc_equation():
    # the l-loop's fixed point solves eq. matrix_NT (residual -> 0)
    op, _ = _op(nx=20, c=5.0, f0=0.0, seed=5)
    N, J, dT, alpha = 8, 4, 0.25, 1e-2
    u0 = heat1d.u0_sine(op.nx)
    U = nl.fine_sequential(op, u0, N, J, N * dT) * 1.05
    starts = np.vstack([u0, U[:-1]])
    b = nl.jump_b(op, nl.F(op, starts, dT, J), U, dT, alpha)
    u = U.copy()
    r0 = np.max(np.abs(nl.cgc_residual(op, u, b, dT, alpha)))
    for _ in range(30):
        u = nl.cgc_newton_step(op, u, b, dT, alpha)
    assert np.max(np.abs(nl.cgc_residual(op, u, b, dT, alpha))) < 1e-11 * max(1.0, r0)


def test_nonlinear_pcgc_reaches_the_fine_solution():
    op, _ = _op(nx=20, c=5.0, f0=0.3, seed=6)
    N, J, T, alpha = 8, 8, 2.0, 1e-3
    u0 = heat1d.u0_sine(op.nx)
    Ustar = nl.fine_sequential(op, u0, N, J, T)
    U, its = nl.pcgc_solve(op, u0, np.zeros_like(Ustar), T / N, J, alpha, 1e-12, 80, 3)
    assert its > 0 and np.max(np.abs(U - Ustar)) < 1e-10


# ---- Burgers-type convection (Engquist-Osher upwind form) ----

def _bop(nx=24, c=8.0, f0=0.0, seed=10, sigma=0.3):
    a = np.exp(sigma * np.random.default_rng(seed).standard_normal(nx + 1))
    return nl.BurgersEO1D(a, c, f0)


def test_burgers_flux_is_upwind_and_conservative():
    op = _bop(nx=16)
    h = op.h
    rng = np.random.default_rng(11)
    up = rng.uniform(0.1, 1.0, op.nx)
    # positive speed: the backward difference of u^2/2 (zero left boundary value)
    assert np.allclose(op.conv(up), (up ** 2 - np.r_[0.0, up[:-1]] ** 2) / (2 * h), rtol=1e-14)
    # negative speed: the forward difference (zero right boundary value)
    un = -up
    assert np.allclose(op.conv(un), (np.r_[un[1:], 0.0] ** 2 - un ** 2) / (2 * h), rtol=1e-14)
    # mixed signs: the interior fluxes telescope to the two boundary fluxes
    u = rng.standard_normal(op.nx)
    total = h * np.sum(op.conv(u))
    assert abs(total - (max(u[-1], 0) ** 2 / 2 - min(u[0], 0) ** 2 / 2)) < 1e-13


def test_burgers_jacobian_matches_finite_differences():
    op = _bop(nx=12, c=5.0, f0=0.3)
    u = np.random.default_rng(12).standard_normal(op.nx)
    u[np.abs(u) < 0.05] = 0.3           # stay off the kink of max(., 0) at 0
    Jd = op.jacobian(u)
    eps = 1e-6
    Jfd = np.stack([(op.f(u + eps * e) - op.f(u - eps * e)) / (2 * eps)
                    for e in np.eye(op.nx)], axis=1)
    assert np.max(np.abs(Jd - Jfd)) < 1e-6 * np.max(np.abs(Jd))


def test_burgers_newton_step_solves_the_backward_euler_equation():
    op = _bop(c=10.0, f0=0.4)
    v = np.sin(2 * np.pi * op.grid()) * 1.2
    for dt in (1e-3, 0.02, 0.2):
        w = op.be_step_newton(v, dt)
        res = w + dt * op.apply(w) + dt * op.c * op.conv(w) - v - dt * op.forcing
        assert np.max(np.abs(res)) < 1e-13 * max(1.0, np.max(np.abs(w)))


def test_burgers_converges_to_the_cole_hopf_solution():
    # a = 1: u_t + c u u_x = u_xx; v = c u solves the viscous Burgers equation
    # with unit viscosity, v = -2 phi_x / phi for phi = 2 + exp(-pi^2 t) cos(pi x)
    # (Cole-Hopf).  Backward Euler and upwind convection are first order: the
    # error halves with h and dt.
    c, T = 10.0, 0.05

    def exact(x, t):
        e = np.exp(-np.pi ** 2 * t)
        return 2 * np.pi * e * np.sin(np.pi * x) / (2 + e * np.cos(np.pi * x)) / c

    errs = []
    for nx, steps in ((49, 40), (99, 80), (199, 160)):
        op = nl.BurgersEO1D(np.ones(nx + 1), c)
        x = op.grid()
        U = nl.fine_sequential(op, exact(x, 0.0), 4, steps // 4, T)
        errs.append(np.max(np.abs(U[-1] - exact(x, T))))
    assert errs[0] < 4e-3 * np.max(exact(np.linspace(0, 1, 101), T))
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.7 < e1 / e2 < 2.3, errs


def test_burgers_cgc_step_diagonalized_equals_dense():
    op = _bop(nx=10, c=6.0, f0=0.2, seed=13)
    N, dT, alpha = 4, 0.05, 1e-2
    rng = np.random.default_rng(14)
    u, b = rng.standard_normal((N, op.nx)), 0.1 * rng.standard_normal((N, op.nx))
    K = op.avg_K_dense(u, b)
    assert not np.allclose(K, K.T)      # the averaged Jacobian is non-symmetric
    assert np.allclose(nl.cgc_newton_step(op, u, b, dT, alpha),
                       nl.cgc_newton_dense(op, u, b, dT, alpha), rtol=1e-10, atol=1e-12)


def test_burgers_parareal_terminates_and_pcgc_converges_to_the_fine_solution():
    op = _bop(nx=20, c=8.0, seed=15)
    N, J, T, alpha = 6, 8, 0.3, 1e-3
    u0 = heat1d.u0_sine(op.nx)
    Ustar = nl.fine_sequential(op, u0, N, J, T)
    # Algorithm 1: after N iterations the first N intervals are fine-exact
    its = pcgc.parareal_classical(op, u0, np.zeros_like(Ustar), T / N, J, N)
    assert np.max(np.abs(its[N] - Ustar)) < 1e-13
    for k in range(1, N):
        assert np.max(np.abs(its[k][:k] - Ustar[:k])) < 1e-13
    U, k = nl.pcgc_solve(op, u0, np.zeros_like(Ustar), T / N, J, alpha, 1e-12, 80, 3)[:2]
    assert k > 0 and np.max(np.abs(U - Ustar)) < 1e-10


def test_nonlinear_contraction_within_theorem_bound():
    # Theorem thm2: under the one-sided Lipschitz condition with constant L
    # (Assumption assump; for f = -A u - c (u^3 - u), L = mu_min(A) - c since
    # u^3 is monotone), the max-over-intervals error contracts per iteration by
    #   rho(alpha) = max{alpha (1 + e^{-x}) / x, (e^{-x} + 1/(1+x)) / (1 - 1/(1+x))},
    # x = L dT.  The CGC is solved to convergence (25 simplified Newton steps).
    rng = np.random.default_rng(21)
    nx = 20
    a = np.exp(0.3 * rng.standard_normal(nx + 1))
    for c, T, N, alpha in ((1.0, 4.0, 4, 0.1), (1.0, 4.0, 8, 0.1), (2.0, 6.0, 6, 0.3)):
        op = nl.CubicRD1D(a, c, 0.0)
        L = np.linalg.eigvalsh(op.dense()).min() - c
        x = L * T / N
        rho = max(alpha * (1 + np.exp(-x)) / x, (np.exp(-x) + 1 / (1 + x)) / (1 - 1 / (1 + x)))
        assert rho < 1
        u0 = heat1d.u0_sine(nx) * 1.5
        J = 8
        Ustar = nl.fine_sequential(op, u0, N, J, T)
        U = np.zeros_like(Ustar)
        err = np.max(np.linalg.norm(U - Ustar, axis=1))
        for _ in range(3):
            U = nl.pcgc_iteration(op, u0, U, T / N, J, alpha, 25)
            e = np.max(np.linalg.norm(U - Ustar, axis=1))
            assert e <= rho * err * (1 + 1e-9), (c, T, N, alpha, e / err, rho)
            err = e
