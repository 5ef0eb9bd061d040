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
