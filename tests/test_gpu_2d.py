"""2D problem on the GPU (five-point operator, Krylov solves) against the
sparse-direct CPU oracle.

The GPU solves every linear system iteratively to a relative residual rtol;
the parity runs use rtol = 1e-14, where the remaining error of a solve is the
rounding of the iteration itself (of order eps times the system's condition
number).  Bars: 1e-12 relative L2, or 4x the oracle's own sensitivity where
that is larger (the distance between oracle results for the coefficient
field and for the field perturbed by 4 ulps, plus, for the CGC, the distance
between the direct-DFT and FFT variants of the diagonalized solve, which
measures the alpha^{-(N-1)/N} amplification of roundoff in step (c)); for
the CGC also eps times the condition number of the shifted systems, scaled
by that amplification (the attainable accuracy of an iterative solve).
Sizes: nx = 15 and 31 keep every system in shared memory (961 unknowns is
ragged against the 256-thread CTA); nx = 63 exceeds it and runs the
global-memory variant of both kernels.
"""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, oracle_setup2d, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-14
SMALL = dict(nx=15, N=8, J=4, M=6, gpc_degree=2, n_train=56)
MID = dict(nx=31, N=8, J=4, M=6, gpc_degree=2, n_train=56)
BIG = dict(nx=63, N=4, J=2, M=4, gpc_degree=1, n_train=10)


def shifted_cond(op, dT, alpha, N):
    from scipy.sparse.linalg import eigsh
    mu_max = eigsh(op.A, k=1, which="LA", return_eigenvectors=False)[0]
    mu_min = eigsh(op.A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    k = np.arange(N // 2 + 1)
    lam = 1.0 - alpha ** (1.0 / N) * np.exp(-2j * np.pi * k / N)
    return float(np.max(np.abs(lam + dT * mu_max) / np.abs(lam + dT * mu_min)))


def dev():
    return torch.device("cuda:0")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def solver2d(over, method=1):
    """method 1: Krylov solves, 2: banded LU (FP64 paths)."""
    solver, w = gpu_solver("rd2d_255", **over)
    solver.set_krylov(RTOL, RTOL, 20000)
    solver.set_2d_method(method)
    return solver, w


METHODS = pytest.mark.parametrize("method", [1, 2], ids=["krylov", "band"])


def test_2d_field_matches_input_kl():
    solver, w = solver2d(SMALL)
    st = oracle_setup2d("rd2d_255", **SMALL)
    S, nx = 4, w.nx
    xi = draw_xi(S, w.M, 31)
    a = torch.empty((S, 2 * nx * (nx + 1)), dtype=torch.float64, device=dev())
    solver.field(T(xi), S, a)
    a = a.cpu().numpy()
    for s in range(S):
        ax = np.exp(np.tensordot(xi[s], st.bx, axes=1))
        ay = np.exp(np.tensordot(xi[s], st.by, axes=1))
        assert rel(a[s, :nx * (nx + 1)], ax.ravel()) < 1e-14
        assert rel(a[s, nx * (nx + 1):], ay.ravel()) < 1e-14


@METHODS
@pytest.mark.parametrize("over", [SMALL, MID, BIG], ids=["nx15", "nx31", "nx63_global"])
def test_2d_reference_matches_sparse_direct(over, method):
    solver, w = solver2d(over, method)
    st = oracle_setup2d("rd2d_255", **over)
    S = 3
    xi = draw_xi(S, w.M, 32)
    U = torch.empty((S, w.N, w.nx * w.nx), dtype=torch.float64, device=dev())
    solver.reference(T(xi), S, w.N, w.J, U)
    its, _ = solver.krylov_stats()
    assert (its > 0) == (method == 1)
    for s in range(S):
        ref = st.reference(xi[s])
        op_p = st.operator(xi[s], 4.0)
        from oracle import heat1d
        floor = rel(heat1d.fine_sequential(op_p, st.u0, w.N, w.J, w.T), ref)
        d = rel(U[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * floor), (s, d, floor)


@METHODS
@pytest.mark.parametrize("over", [SMALL, BIG], ids=["nx15", "nx63_global"])
def test_2d_fine_sweep_matches_oracle(over, method):
    from oracle import pcgc
    solver, w = solver2d(over, method)
    st = oracle_setup2d("rd2d_255", **over)
    S, dT = 3, w.T / w.N
    xi = draw_xi(S, w.M, 33)
    Uin = np.stack([st.reference(x) for x in xi]) * 1.02 + 1e-3
    r = torch.empty_like(T(Uin))
    solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, 0, r)
    for s in range(S):
        op = st.operator(xi[s])
        Fend = pcgc.fine_sweep(op, st.u0, Uin[s], dT, w.J)
        ref = pcgc.cgc_rhs(op, Uin[s], pcgc.jump_b(op, Fend, Uin[s], dT, w.alpha), dT)
        opp = st.operator(xi[s], 4.0)
        Fp = pcgc.fine_sweep(opp, st.u0, Uin[s], dT, w.J)
        refp = pcgc.cgc_rhs(opp, Uin[s], pcgc.jump_b(opp, Fp, Uin[s], dT, w.alpha), dT)
        # r = (I + dT A) F - prev amplifies the rounding of F by ||I + dT A||_inf
        amp = 1.0 + dT * abs(op.A).sum(1).max()
        bar = max(1e-12, 4 * rel(refp, ref), 10 * 2.3e-16 * amp)
        assert rel(r[s].cpu().numpy(), ref) < bar


@pytest.mark.parametrize("over,alpha", [(SMALL, 1e-3), (SMALL, 0.2), (MID, 1e-2),
                                        (BIG, 1e-3)],
                         ids=["nx15_a1e-3", "nx15_a0.2", "nx31", "nx63_global"])
@METHODS
def test_2d_cgc_apply_matches_oracle(over, alpha, method):
    from oracle import pcgc
    solver, w = solver2d(over, method)
    st = oracle_setup2d("rd2d_255", **over)
    S, N, dT = 3, w.N, w.T / w.N
    n = w.nx * w.nx
    xi = draw_xi(S, w.M, 34)
    r = np.random.default_rng(6).standard_normal((S, N, n))
    u = torch.empty_like(T(r))
    solver.cgc_apply(T(xi), S, N, T(r), dT, alpha, 0, u)
    its = solver.krylov_stats()[1]
    assert (its > 0) == (method == 1)
    for s in range(S):
        op = st.operator(xi[s])
        ref = pcgc.cgc_diagonalized(op, r[s], dT, alpha)
        floor = rel(pcgc.cgc_diagonalized(op, r[s], dT, alpha, fft=True), ref)
        floor += rel(pcgc.cgc_diagonalized(st.operator(xi[s], 4.0), r[s], dT, alpha), ref)
        if n * N <= 2000:
            floor += rel(pcgc.cgc_dense(op, r[s], dT, alpha), ref)
        # the Krylov solution of system k carries a forward error up to its
        # condition number times eps, which step (c) scales by up to
        # alpha^{-(N-1)/N}; lambda_k I + dT A is normal, so its condition
        # number is |lambda_k + dT mu_max| / |lambda_k + dT mu_min|
        kry = 4 * 2.2e-16 * shifted_cond(op, dT, alpha, N) * alpha ** (-(N - 1) / N)
        d = rel(u[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * floor, kry), (s, d, floor, kry)


@METHODS
@pytest.mark.parametrize("over", [SMALL, MID], ids=["nx15", "nx31"])
def test_2d_solve_matches_oracle(over, method):
    import paper_2510_26180_gb300 as pkg
    solver, w = solver2d(over, method)
    st = oracle_setup2d("rd2d_255", **over)
    S = 6
    xi = draw_xi(S, w.M, 35)
    n = w.nx * w.nx
    U = torch.empty((S, w.N, n), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    stt = torch.empty(S, dtype=torch.int32, device=dev())
    U0 = torch.empty_like(U)
    solver.guess(T(xi), S, 0, U0)
    assert rel(U0.cpu().numpy(), st.guess(xi)) < 1e-10
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.FP64,
                        pkg.GUESS_GPC, U, it, stt)
    assert code == 0
    U, it, stt = U.cpu().numpy(), it.cpu().numpy(), stt.cpu().numpy()
    assert np.all(stt == 0)
    for s in range(S):
        Uo, ko, _ = st.solve_sample(xi[s])
        Up, _, _ = st.solve_sample(xi[s], field_ulps=4.0)
        Uf, _, _ = st.solve_sample(xi[s], cgc="fft")
        floor = rel(Up, Uo) + rel(Uf, Uo)
        assert it[s] == ko
        d = rel(U[s], Uo)
        assert d < max(1e-12, 4 * floor), (s, d, floor)
        assert rel(U[s], st.reference(xi[s])) < 1e-6


def test_2d_krylov_cap_is_reported():
    import paper_2510_26180_gb300 as pkg
    solver, w = solver2d(SMALL)
    S = 2
    xi = draw_xi(S, w.M, 36)
    U = torch.empty((S, w.N, w.nx * w.nx), dtype=torch.float64, device=dev())
    stt = torch.empty(S, dtype=torch.int32, device=dev())
    try:
        solver.set_krylov(1e-12, 1e-12, 2)
        code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, 3, pkg.FP64,
                            pkg.GUESS_GPC, U, None, stt)
        assert code == pkg.E_NOT_CONVERGED
        assert np.all(stt.cpu().numpy() == pkg.E_NOT_CONVERGED)
        with pytest.raises(pkg.KlecgcError):
            solver.reference(T(xi), S, w.N, w.J, U)
    finally:
        solver.set_krylov(RTOL, RTOL, 20000)


def test_2d_unsupported_modes():
    import paper_2510_26180_gb300 as pkg
    solver, w = solver2d(SMALL)
    S = 2
    xi = T(draw_xi(S, w.M, 37))
    U = torch.empty((S, w.N, w.nx * w.nx), dtype=torch.float64, device=dev())
    with pytest.raises(pkg.KlecgcError) as e:
        solver.solve(xi, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, 5, pkg.MIXED_DEFECT,
                     pkg.GUESS_GPC, U)
    assert e.value.status == pkg.E_UNSUPPORTED
    with pytest.raises(pkg.KlecgcError) as e:
        solver.mlp_set(torch.zeros(solver.mlp_n_params(), dtype=torch.float32, device=dev()))
    assert e.value.status == pkg.E_UNSUPPORTED
    with pytest.raises(pkg.KlecgcError) as e:
        solver.reference_noalloc(xi, S, w.N, w.J, U)
    assert e.value.status == pkg.E_UNSUPPORTED


@pytest.mark.parametrize("over", [SMALL, BIG], ids=["nx15", "nx63"])
def test_2d_fine_sweep_mixed_refinement_matches_oracle(over):
    """The mixed propagator (FP64 refinement around FP32 PCG) meets the same
    FP64 residual test, so it has the FP64 bar."""
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = solver2d(over)
    st = oracle_setup2d("rd2d_255", **over)
    S, dT = 3, w.T / w.N
    xi = draw_xi(S, w.M, 38)
    Uin = np.stack([st.reference(x) for x in xi]) * 0.97 + 2e-3
    r = torch.empty_like(T(Uin))
    solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, pkg.MIXED, r)
    assert solver.krylov_stats()[0] > 0
    for s in range(S):
        op = st.operator(xi[s])
        Fend = pcgc.fine_sweep(op, st.u0, Uin[s], dT, w.J)
        ref = pcgc.cgc_rhs(op, Uin[s], pcgc.jump_b(op, Fend, Uin[s], dT, w.alpha), dT)
        opp = st.operator(xi[s], 4.0)
        Fp = pcgc.fine_sweep(opp, st.u0, Uin[s], dT, w.J)
        refp = pcgc.cgc_rhs(opp, Uin[s], pcgc.jump_b(opp, Fp, Uin[s], dT, w.alpha), dT)
        amp = 1.0 + dT * abs(op.A).sum(1).max()
        bar = max(1e-12, 4 * rel(refp, ref), 10 * 2.3e-16 * amp)
        assert rel(r[s].cpu().numpy(), ref) < bar


@pytest.mark.parametrize("over", [SMALL, MID], ids=["nx15", "nx31"])
def test_2d_solve_mixed_matches_oracle(over):
    import paper_2510_26180_gb300 as pkg
    solver, w = solver2d(over)
    st = oracle_setup2d("rd2d_255", **over)
    S = 6
    xi = draw_xi(S, w.M, 39)
    n = w.nx * w.nx
    U = torch.empty((S, w.N, n), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    stt = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.MIXED,
                        pkg.GUESS_GPC, U, it, stt)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for s in range(S):
        Uo, ko, _ = st.solve_sample(xi[s])
        Up, _, _ = st.solve_sample(xi[s], field_ulps=4.0)
        Uf, _, _ = st.solve_sample(xi[s], cgc="fft")
        floor = rel(Up, Uo) + rel(Uf, Uo)
        assert it[s] == ko
        assert rel(U[s], Uo) < max(1e-12, 4 * floor)


@pytest.mark.parametrize("over,alpha", [(SMALL, 1e-3), (MID, 1e-2), (BIG, 1e-3)],
                         ids=["nx15", "nx31", "nx63"])
def test_2d_cgc_apply_mixed_refinement_matches_oracle(over, alpha):
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = solver2d(over)
    st = oracle_setup2d("rd2d_255", **over)
    S, N, dT = 3, w.N, w.T / w.N
    n = w.nx * w.nx
    xi = draw_xi(S, w.M, 40)
    r = np.random.default_rng(7).standard_normal((S, N, n))
    u = torch.empty_like(T(r))
    solver.cgc_apply(T(xi), S, N, T(r), dT, alpha, pkg.MIXED, u)
    assert solver.krylov_stats()[1] > 0
    for s in range(S):
        op = st.operator(xi[s])
        ref = pcgc.cgc_diagonalized(op, r[s], dT, alpha)
        floor = rel(pcgc.cgc_diagonalized(op, r[s], dT, alpha, fft=True), ref)
        floor += rel(pcgc.cgc_diagonalized(st.operator(xi[s], 4.0), r[s], dT, alpha), ref)
        kry = 4 * 2.2e-16 * shifted_cond(op, dT, alpha, N) * alpha ** (-(N - 1) / N)
        d = rel(u[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * floor, kry), (s, d, floor, kry)


def test_2d_method_argument_checks():
    import paper_2510_26180_gb300 as pkg
    solver, _ = solver2d(SMALL)
    with pytest.raises(pkg.KlecgcError) as e:
        solver.set_2d_method(4)
    assert e.value.status == pkg.E_INVALID_ARG
    one_d, _ = gpu_solver("heat1d_nx63")
    with pytest.raises(pkg.KlecgcError) as e:
        one_d.set_2d_method(3)   # thread-block clusters: 2D systems only
    assert e.value.status == pkg.E_UNSUPPORTED
    big, _ = gpu_solver("rd2d_255", nx=95, N=4, J=1, M=4, gpc_degree=1, n_train=10)
    with pytest.raises(pkg.KlecgcError) as e:
        big.set_2d_method(2)
    assert e.value.status == pkg.E_UNSUPPORTED
    solver.set_2d_method(1)
