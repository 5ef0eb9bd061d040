"""Pins of the oracle's operator, propagators and parareal iterations against
closed forms, dense brute force and the paper's error-propagation matrices."""
import math

import numpy as np
import pytest

from oracle import contraction, heat1d, pcgc


def _op(nx, seed=0, reaction=0.0, forcing=0.0, const=False):
    rng = np.random.default_rng(seed)
    a = np.ones(nx + 1) if const else np.exp(0.5 * rng.standard_normal(nx + 1))
    return heat1d.Heat1D(a, reaction, forcing)


def test_operator_eigenvalues_constant_coefficient():
    # a == 1: textbook spectrum mu_k = (4/h^2) sin^2(k pi h / 2), eigvecs sin(k pi x)
    nx = 31
    op = _op(nx, const=True, reaction=0.7)
    h = op.h
    mu = 4 / h ** 2 * np.sin(np.arange(1, nx + 1) * np.pi * h / 2) ** 2 + 0.7
    ev = np.sort(np.linalg.eigvalsh(op.dense()))
    assert np.allclose(ev, mu, rtol=1e-12)
    x = op.grid()
    for k in (1, 5):
        v = np.sin(k * np.pi * x)
        assert np.allclose(op.apply(v), mu[k - 1] * v, rtol=1e-11, atol=1e-9)


def test_sequential_fine_solution_closed_form_a_const():
    # a == 1, u0 = sin(pi x): U*_n = (1 + dt mu_1)^(-nJ) sin(pi x_i) exactly
    nx, N, J, T = 63, 16, 16, 1.0
    op = _op(nx, const=True)
    u0 = heat1d.u0_sine(nx)
    U = heat1d.fine_sequential(op, u0, N, J, T)
    mu1 = 4 / op.h ** 2 * math.sin(math.pi * op.h / 2) ** 2
    dt = T / N / J
    n = np.arange(1, N + 1)
    exact = (1 + dt * mu1) ** (-(n * J))[:, None] * u0[None, :]
    assert np.allclose(U, exact, rtol=1e-12, atol=1e-15)
    # coarse propagator multiplies by 1 / (1 + dT mu_1)
    assert np.allclose(heat1d.G(op, u0, T / N), u0 / (1 + T / N * mu1), rtol=1e-13)


def test_forcing_steady_state_is_discrete_parabola():
    # a == 1, f0 = 1: the 3-point scheme is exact on x(1-x)/2, the steady state of BE
    nx = 31
    op = _op(nx, const=True, forcing=1.0)
    v = np.zeros(nx)
    for _ in range(400):
        v = op.be_step(v, 0.05)
    x = op.grid()
    assert np.allclose(v, x * (1 - x) / 2, rtol=1e-10, atol=1e-13)


def test_diagonalization_corrected_and_printed_orientation():
    for N, alpha in ((2, 0.3), (8, 1e-3), (16, 1e-4)):
        C = pcgc.calpha(N, alpha)
        V, lam = pcgc.diag_factors(N, alpha)
        assert np.linalg.norm(C @ V - V @ np.diag(lam)) <= 1e-12 * np.linalg.norm(V)
        Vp, _ = pcgc.diag_factors(N, alpha, printed=True)
        assert np.linalg.norm(C @ Vp - Vp @ np.diag(lam)) > 1e-3 * np.linalg.norm(Vp)
        # eigenvalues printed as 1 - alpha^(1/N) omega^-(n-1) are the true ones
        ev = np.linalg.eigvals(C)
        for l in lam:
            assert np.min(np.abs(ev - l)) < 1e-10


@pytest.mark.parametrize("N,nx,alpha", [(4, 8, 0.1), (6, 5, 1e-3), (8, 7, 1e-2), (2, 1, 0.5),
                                        (2, 2, 1e-4)])
def test_three_step_solve_equals_dense_kron_solve(N, nx, alpha):
    op = _op(nx, seed=N, reaction=0.3)
    r = np.random.default_rng(1).standard_normal((N, nx))
    dT = 1.0 / N
    u1 = pcgc.cgc_diagonalized(op, r, dT, alpha)
    u2 = pcgc.cgc_dense(op, r, dT, alpha)
    assert np.allclose(u1, u2, rtol=1e-11, atol=1e-12 * np.abs(u2).max())


def test_dft_of_real_data_is_hermitian():
    N = 16
    r = np.random.default_rng(3).standard_normal((N, 5))
    p = pcgc.dft_matrix(N).conj().T @ r
    for k in range(1, N):
        assert np.allclose(p[N - k], p[k].conj(), atol=1e-13)


def test_alpha_limit_is_sequential_cgc():
    # CGC_alpha - CGC_seq = O(alpha) (the alpha-system tends to the sequential one)
    N, nx = 8, 9
    op = _op(nx, seed=5)
    r = np.random.default_rng(2).standard_normal((N, nx))
    dT = 1 / N
    useq = pcgc.cgc_sequential(op, r, dT)
    ratios = []
    for alpha in (1e-2, 1e-3, 1e-4, 1e-5):
        ratios.append(np.linalg.norm(pcgc.cgc_diagonalized(op, r, dT, alpha) - useq) / alpha)
    assert max(ratios) / min(ratios) < 1.1
    assert ratios[0] > 1e-8


def test_classical_parareal_terminates_after_N_iterations():
    nx, N, J = 11, 6, 5
    op = _op(nx, seed=7, reaction=0.2, forcing=0.5)
    u0 = heat1d.u0_sine(nx)
    Ustar = heat1d.fine_sequential(op, u0, N, J, 1.0)
    U0 = np.random.default_rng(0).standard_normal((N, nx))
    its = pcgc.parareal_classical(op, u0, U0, 1.0 / N, J, N)
    assert np.allclose(its[N], Ustar, rtol=1e-12, atol=1e-13)
    # and after k iterations the first k points are already exact
    for k in range(1, N):
        assert np.allclose(its[k][:k], Ustar[:k], rtol=1e-12, atol=1e-13)


def test_cgc_rhs_newton_form_equals_jump_form():
    # r of eq. three steps at l=0 equals (I + dT A) b + dT f0 for linear f
    N, nx = 5, 7
    op = _op(nx, seed=9, reaction=0.4, forcing=0.8)
    rng = np.random.default_rng(4)
    Uk, b = rng.standard_normal((2, N, nx))
    dT = 0.2
    r = pcgc.cgc_rhs(op, Uk, b, dT)
    assert np.allclose(r, b + dT * op.apply(b) + dT * 0.8, rtol=1e-13, atol=1e-13)


def _scalar_setup(N=12, J=8, alpha=1e-2, nx=15, T=1.0):
    op = _op(nx, const=True)
    u0 = heat1d.u0_sine(nx)
    mu1 = 4 / op.h ** 2 * math.sin(math.pi * op.h / 2) ** 2
    return op, u0, mu1, N, J, alpha, T


def test_error_propagation_matches_lemma_matrices():
    # a == 1, every iterate is a multiple of sin(pi x); the error vector obeys
    # e^{k+1} = G(z)^{-1} (G(z) - F(z)) e^k exactly (Lemma lem1), z = dT mu_1
    op, u0, mu1, N, J, alpha, T = _scalar_setup()
    dT = T / N
    z = dT * mu1
    Ustar = heat1d.fine_sequential(op, u0, N, J, T)
    rng = np.random.default_rng(0)
    U = rng.standard_normal(N)[:, None] * u0[None, :]
    Gm, Fm = contraction.lemma_matrices(z, J, N, alpha)
    Mit = np.linalg.solve(Gm, Gm - Fm)
    e = (U - Ustar)[:, 0] / u0[0]
    for _ in range(5):
        U = pcgc.pcgc_iteration(op, u0, U, dT, J, alpha)
        e_new = (U - Ustar)[:, 0] / u0[0]
        # alpha-twisted G couples e_1 to alpha e_N; the fixed point is U*
        assert np.allclose(e_new, Mit @ e, rtol=1e-9, atol=1e-12)
        assert np.max(np.abs(e_new)) <= contraction.k_alpha(z, J, alpha) * np.max(np.abs(e)) + 1e-14
        e = e_new


def test_contraction_factor_sup_is_below_one_third():
    # BE/BE: sup_z K_cla(z, J) -> sup (e^-z - 1/(1+z)) (1+z)/z ~ 0.2984 (paper quotes ~1/3)
    z = np.logspace(-3, 3, 20001)
    kc = contraction.k_cla(z, 10 ** 6)
    zz = z
    limit = np.abs(np.exp(-zz) - 1 / (1 + zz)) / (1 - 1 / (1 + zz))
    assert abs(kc.max() - limit.max()) < 1e-5
    assert 0.29 < kc.max() < 1 / 3
    # finite J stays below the J -> infinity envelope
    assert contraction.k_cla(z, 16).max() <= kc.max() + 1e-12


def test_pcgc_converges_to_fine_solution():
    # fixed point of Algorithm 2 is U* (F starts from u0 on the first interval)
    nx, N, J = 15, 8, 6
    op = _op(nx, seed=11, reaction=0.1, forcing=0.3)
    u0 = heat1d.u0_sine(nx)
    Ustar = heat1d.fine_sequential(op, u0, N, J, 1.0)
    U0 = pcgc.coarse_guess(op, u0, N, 1.0 / N)
    U, its, _ = pcgc.pcgc_solve(op, u0, U0, 1.0 / N, J, 1e-3, 1e-12, 60)
    assert its > 0
    assert np.max(np.abs(U - Ustar)) < 1e-11


def test_variable_coefficient_operator_is_second_order_consistent():
    # A u against -(a u')' for u = sin(pi x) and a sample's KL field a = exp(g):
    # with a taken at the faces x_{i+1/2} the flux form is consistent to
    # O(h^2) (error ratio 4 per halving of h); faces shifted by h/2 would give
    # O(h) (ratio 2).  Pins the face placement, the flux-form signs and the
    # 1/h^2 scaling with a non-constant coefficient.
    from synth import draw_xi, workload
    from oracle import kl_input
    from oracle.klecgc import Setup1D
    errs = []
    for nx in (63, 127, 255):
        w = workload("heat1d_nx63", nx=nx)
        st = Setup1D(w, build=False)
        xi = 2.0 * draw_xi(1, w.M, 5)[0]
        op = st.operator(xi)
        x = (np.arange(nx) + 1) / (nx + 1)
        u = np.sin(np.pi * x)
        Au = op.apply(u) - op.reaction * u

        def a_of(y):
            B = kl_input.field_basis_1d(w.sigma, w.corr_len, w.M, y)
            return np.exp(kl_input.log_coefficient_1d(xi, B))

        d = 1e-5
        da = (a_of(x + d) - a_of(x - d)) / (2 * d)
        exact = -(da * np.pi * np.cos(np.pi * x) - a_of(x) * np.pi ** 2 * np.sin(np.pi * x))
        errs.append(np.abs(Au - exact).max() / np.abs(exact).max())
    assert errs[-1] < 1e-4
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 < e1 / e2 < 4.4, errs


def test_emulated_fine_propagator_algebra_in_fp64():
    # in FP64 the emulation is the propagator F itself, in either form and for
    # any refresh period: the increment recurrence M (v' - v) = v - v_prev and
    # the flux-form defect are exact identities of backward Euler
    op = _op(40, seed=3, reaction=0.3, forcing=0.7)
    V = np.random.default_rng(6).standard_normal((3, 40))
    ref = np.stack([heat1d.F(op, v, 0.05, 12) for v in V])
    for form, K in (("direct", 1), ("increment", 1), ("increment", 5), ("increment", 12)):
        got = heat1d.F_emulated(op, V, 0.05, 12, np.float64, form, K)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref)), (form, K)


def test_emulated_fp32_increment_form_keeps_accuracy():
    # FP32 substitutions with FP64-made factors on the Nx = 1023, J = 64 heat
    # workload: the increment form with the flux defect on every step is far
    # more accurate than the direct form, and reusing the previous increment
    # between refreshes costs accuracy monotonically in the refresh period
    from synth import draw_xi, workload
    from oracle.klecgc import Setup1D
    w = workload("heat1d_nx1023")
    st = Setup1D(w, build=False)
    op = st.operator(draw_xi(1, w.M, 5)[0])
    dT = w.T / w.N
    V = np.stack([st.u0, heat1d.F(op, st.u0, 10 * dT, 10 * w.J)])
    ref = np.stack([heat1d.F(op, v, dT, w.J) for v in V])

    def err(form, K):
        got = heat1d.F_emulated(op, V, dT, w.J, np.float32, form, K)
        return np.max(np.abs(got - ref)) / np.max(np.abs(ref))

    direct, e1, e16, e64 = err("direct", 1), err("increment", 1), err("increment", 16), \
        err("increment", 64)
    assert direct > 1e-6 and e1 < 2e-7
    assert e1 < direct / 20 and e16 < direct / 5
    assert e1 < e16 < e64


def test_coarse_guess_closed_form_a_const():
    # a == 1, f0 = 0, u0 = sin(pi x): the coarse sweep U0_n = G(U0_{n-1}) is
    # (1 + dT mu_1)^(-n) sin(pi x_i) (Section 3.1); with f0 = 1 from zero it
    # tends to the discrete steady state x(1-x)/2
    nx, N, T = 31, 16, 1.0
    op = _op(nx, const=True)
    u0 = heat1d.u0_sine(nx)
    U0 = pcgc.coarse_guess(op, u0, N, T / N)
    mu1 = 4 / op.h ** 2 * math.sin(math.pi * op.h / 2) ** 2
    n = np.arange(1, N + 1)
    exact = (1 + T / N * mu1) ** (-n.astype(float))[:, None] * u0[None, :]
    assert U0.shape == (N, nx)
    assert np.allclose(U0, exact, rtol=1e-12, atol=1e-15)
    opf = _op(nx, const=True, forcing=1.0)
    Uf = pcgc.coarse_guess(opf, np.zeros(nx), 400, 0.05)
    x = opf.grid()
    assert np.allclose(Uf[-1], x * (1 - x) / 2, rtol=1e-10, atol=1e-13)


def test_error_metrics_by_construction():
    # Section 5's e_n = (1/S) sum_i ||u_n(xi_i) - U_n(xi_i)||_inf: perturb one
    # entry of each (sample, n) by a chosen t[s, n] and smaller ones elsewhere
    from oracle.klecgc import mean_inf_error, rel_l2
    rng = np.random.default_rng(8)
    S, N, nx = 3, 4, 5
    Uref = rng.standard_normal((S, N, nx))
    t = rng.random((S, N)) + 0.5
    D = rng.uniform(-0.4, 0.4, (S, N, nx))
    pos = rng.integers(0, nx, (S, N))
    for s in range(S):
        for n in range(N):
            D[s, n, pos[s, n]] = -t[s, n] if (s + n) % 2 else t[s, n]
    assert np.allclose(mean_inf_error(Uref, Uref + D), t.mean(axis=0), rtol=1e-14)
    # rel_l2 of a uniform relative scaling is the scaling
    assert abs(rel_l2(1.25 * Uref, Uref) - 0.25) < 1e-14


def _cgc_extended(op, r, dT, alpha):
    """Steps (a)-(c) of the diagonalized CGC carried out in long double
    (x86 80-bit or IEEE quad): the direct DFT with exponents reduced mod N,
    a Thomas solve by divisions, the alpha^{+-j/N} scalings.  A reference for
    the FP64 rounding, not a second oracle: it shares the three steps' algebra
    (pinned by the dense Kronecker test) and differs in precision only."""
    LD = np.longdouble
    N, n = r.shape
    j = np.arange(N)
    two_pi = 2 * LD("3.141592653589793238462643383279502884")
    ang = two_pi * (np.outer(j, j) % N).astype(LD) / LD(N)
    Wr, Wi = np.cos(ang), np.sin(ang)                           # omega^{jk}
    a = LD(alpha)
    sc = a ** (j.astype(LD) / LD(N))
    sr = sc[:, None] * r.astype(LD)
    inv_sqrt_n = LD(1) / np.sqrt(LD(N))
    pr, pi = (Wr.T @ sr) * inv_sqrt_n, -(Wi.T @ sr) * inv_sqrt_n   # F_N^* (Lambda r)
    th = two_pi * j.astype(LD) / LD(N)
    root = a ** (LD(1) / LD(N))
    lr, li = 1 - root * np.cos(th), root * np.sin(th)            # lambda_k = 1 - a^{1/N} e^{-i th}
    w = LD(dT) * op.wf.astype(LD)                                # dT a / h^2 at the n + 1 faces
    c = LD(dT) * LD(op.reaction)
    # Thomas over rows, vectorized over the N frequencies (complex as pairs)
    yr, yi = np.empty((n, N), LD), np.empty((n, N), LD)
    gr, gi = np.empty((n, N), LD), np.empty((n, N), LD)            # pivots
    for i in range(n):
        dr, di = lr + w[i] + w[i + 1] + c, li.copy()
        br, bi = pr[:, i].copy(), pi[:, i].copy()
        if i > 0:
            den = gr[i - 1] ** 2 + gi[i - 1] ** 2
            mr, mi = -w[i] * gr[i - 1] / den, w[i] * gi[i - 1] / den   # l = -w_i / piv_{i-1}
            dr, di = dr + mr * w[i], di + mi * w[i]
            br, bi = br - (mr * yr[i - 1] - mi * yi[i - 1]), bi - (mr * yi[i - 1] + mi * yr[i - 1])
        gr[i], gi[i], yr[i], yi[i] = dr, di, br, bi
    qr, qi = np.empty((n, N), LD), np.empty((n, N), LD)
    xr, xi = np.zeros(N, LD), np.zeros(N, LD)
    for i in range(n - 1, -1, -1):
        tr, ti = yr[i] + w[i + 1] * xr, yi[i] + w[i + 1] * xi         # y_i - M_{i,i+1} x_{i+1}
        if i == n - 1:
            tr, ti = yr[i], yi[i]
        den = gr[i] ** 2 + gi[i] ** 2
        xr, xi = (tr * gr[i] + ti * gi[i]) / den, (ti * gr[i] - tr * gi[i]) / den
        qr[i], qi[i] = xr, xi
    # (c) u = Lambda^{-1} F_N q, real part
    ur = (Wr @ qr.T - Wi @ qi.T) * inv_sqrt_n
    return ((LD(1) / sc)[:, None] * ur).astype(np.float64)


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18,
                    reason="long double is not wider than double on this host")
def test_cgc_fp64_accuracy_at_alpha_1e4_against_extended_precision():
    # Nx = 1023, N = 64, dT = 1/64, alpha = 1e-4: the shifted systems have
    # dT a / h^2 ~ 1e4, and step (c) multiplies rounding by up to alpha^{-63/64}
    # (Section 3.2, the paragraph on choosing alpha).  The oracle's FP64 result
    # must be within 1e-11 (relative L2) of the same three steps in extended
    # precision; without the refinement of step (b) it is off by ~3e-9.
    from oracle import kl_input
    nx, N, alpha = 1023, 64, 1e-4
    dT = 1.0 / N
    faces = (np.arange(nx + 1) + 0.5) / (nx + 1)
    basis = kl_input.field_basis_1d(0.5, 0.5, 10, faces)
    xi = np.random.default_rng(93).standard_normal(10)
    op = heat1d.Heat1D(np.exp(kl_input.log_coefficient_1d(xi, basis)))
    u0 = heat1d.u0_sine(nx)
    U0 = pcgc.coarse_guess(op, u0, N, dT)
    Fend = pcgc.fine_sweep(op, u0, U0, dT, 4)
    r = pcgc.cgc_rhs(op, U0, pcgc.jump_b(op, Fend, U0, dT, alpha), dT)
    ref = _cgc_extended(op, r, dT, alpha)
    got = pcgc.cgc_diagonalized(op, r, dT, alpha)
    d = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert d < 1e-11, d
    # the extended evaluation itself agrees with the FP64 one where rounding is
    # not amplified (the first coarse time), i.e. it computes the same thing
    assert np.linalg.norm(got[0] - ref[0]) / np.linalg.norm(ref[0]) < 1e-14


def test_refined_shifted_solve_residual_and_dense_agreement():
    # the refined solve satisfies the system: dense LU on a small grid agrees,
    # and the flux-form operator equals the matrix form (exact algebra)
    op = _op(40, seed=3, reaction=0.4)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((3, 40)) + 1j * rng.standard_normal((3, 40))
    shift, scale = 0.2 - 0.3j, 0.05
    X = op.shifted_solve_refined(shift, scale, R)
    M = shift * np.eye(40) + scale * op.dense()
    assert np.allclose(X, np.linalg.solve(M, R.T).T, rtol=1e-13, atol=1e-13)
    V = rng.standard_normal((2, 40))
    assert np.allclose(op.apply_flux(V), op.apply(V), rtol=1e-13, atol=1e-12)
