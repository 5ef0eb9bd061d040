"""Parity of every CUDA stage and of the whole solve against the CPU oracle.

Tolerances: FP64 paths 1e-12 relative L2, or 4x the method's own floor
where that is larger.  The floor has two parts, both measured per case on
the oracle alone: (i) step (c) of the diagonalized CGC multiplies roundoff
by up to alpha^{-(N-1)/N} (the paper's remark on alpha: the diagonalization's
rounding error grows as alpha shrinks), so every FP64 implementation of it
carries an error of order eps/alpha: measured as the distance between the
oracle's diagonalized result and the dense solve of the same system;
(ii) the library and the oracle compute the coefficient field independently,
so a differs in its last bits, which the shifted systems amplify by their
condition number: the distance between oracle results for a and for a
perturbed by 4 ulps;
FP32 stages get bounds derived from eps_32 = 6e-8 times the conditioning
stated at each test; the mixed solves must land within 1e-6 of the
sequential fine solution U*, the accuracy the method is measured at.
"""
import numpy as np
import pytest

from synth import draw_train, draw_xi, workload
from tests.gpu_util import gpu_solver, oracle_setup, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev():
    return torch.device("cuda:0")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def test_field_matches_input_kl():
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    xi = draw_xi(5, w.M, 11)
    a = torch.empty((5, w.nx + 1), dtype=torch.float64, device=dev())
    solver.field(T(xi), 5, a)
    for s in range(5):
        op = st.operator(xi[s])
        h = op.h
        # oracle stores A's diagonal; recover the faces from exp(g) directly
        from oracle import kl_input
        ref = np.exp(kl_input.log_coefficient_1d(xi[s], st.basis))
        assert rel(a[s].cpu().numpy(), ref) < 1e-14
        assert h == 1.0 / (w.nx + 1)


@pytest.mark.parametrize("over", [dict(), dict(nx=100, N=8, J=5), dict(nx=33, N=4, J=3)])
def test_reference_solution_matches_oracle(over):
    solver, w = gpu_solver("heat1d_nx63", **over) if over else gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63", **over) if over else oracle_setup("heat1d_nx63")
    S = 7
    xi = draw_xi(S, w.M, 12)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.reference(T(xi), S, w.N, w.J, U)
    for s in range(S):
        assert rel(U[s].cpu().numpy(), st.reference(xi[s])) < 1e-12


@pytest.mark.parametrize("over", [dict(), dict(nx=100, N=8, J=5)])
def test_fine_sweep_fp64_matches_oracle(over):
    from oracle import pcgc
    solver, w = gpu_solver("heat1d_nx63", **over) if over else gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63", **over) if over else oracle_setup("heat1d_nx63")
    S, dT = 6, w.T / w.N
    xi = draw_xi(S, w.M, 13)
    Uin = np.random.default_rng(3).standard_normal((S, w.N, w.nx))
    r = torch.empty_like(T(Uin))
    solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, 0, r)
    for s in range(S):
        op = st.operator(xi[s])
        Fend = pcgc.fine_sweep(op, st.u0, Uin[s], dT, w.J)
        b = pcgc.jump_b(op, Fend, Uin[s], dT, w.alpha)
        ref = pcgc.cgc_rhs(op, Uin[s], b, dT)
        # r = (I + dT A) F - prev: roundoff of F (eps each entry) is amplified by
        # ||I + dT A||_inf <= 1 + 4 dT max(a) / h^2 in r
        amp = 1.0 + dT * np.abs(op.dense()).sum(1).max()
        assert rel(r[s].cpu().numpy(), ref) < max(1e-12, 10 * 2.3e-16 * amp)


def test_fine_sweep_fp32_increment_form():
    # smooth start values; the FP32 F error is ~1e-7 |F| per row, amplified in
    # r by ||I + dT A|| only on the (rough) roundoff: 1e-3 bounds it here
    from oracle import pcgc
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    S, dT = 4, w.T / w.N
    xi = draw_xi(S, w.M, 14)
    Uin = np.stack([st.reference(x) for x in xi]) * 1.01
    r = torch.empty_like(T(Uin))
    solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, 1, r)
    for s in range(S):
        op = st.operator(xi[s])
        Fend = pcgc.fine_sweep(op, st.u0, Uin[s], dT, w.J)
        ref = pcgc.cgc_rhs(op, Uin[s], pcgc.jump_b(op, Fend, Uin[s], dT, w.alpha), dT)
        assert rel(r[s].cpu().numpy(), ref) < 1e-3
        # the FP32 fine end values themselves are accurate to a few eps_32
        Fg = pcgc.cgc_diagonalized(op, r[s].cpu().numpy(), dT, w.alpha)
        Fo = pcgc.cgc_diagonalized(op, ref, dT, w.alpha)
        assert rel(Fg, Fo) < 2e-6


@pytest.mark.parametrize("N,nx,alpha", [(16, 63, 1e-3), (2, 40, 0.3), (4, 33, 1e-2),
                                        (64, 100, 1e-4), (32, 129, 1e-3)])
def test_cgc_apply_fp64_matches_direct_dft(N, nx, alpha):
    from oracle import pcgc
    solver, w = gpu_solver("heat1d_nx63", nx=nx, N=N, J=2)
    st = oracle_setup("heat1d_nx63", nx=nx, N=N, J=2)
    S, dT = 5, w.T / N
    xi = draw_xi(S, w.M, 15)
    r = np.random.default_rng(4).standard_normal((S, N, nx))
    u = torch.empty_like(T(r))
    solver.cgc_apply(T(xi), S, N, T(r), dT, alpha, 0, u)
    for s in range(S):
        op = st.operator(xi[s])
        ref = pcgc.cgc_diagonalized(op, r[s], dT, alpha)
        floor = rel(pcgc.cgc_dense(op, r[s], dT, alpha), ref)
        floor += rel(pcgc.cgc_diagonalized(st.operator(xi[s], 4.0), r[s], dT, alpha), ref)
        assert rel(u[s].cpu().numpy(), ref) < max(1e-12, 4 * floor)


def test_cgc_apply_fp32():
    from oracle import pcgc
    N, nx, alpha = 16, 63, 1e-3
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    S, dT = 4, w.T / N
    xi = draw_xi(S, w.M, 16)
    r = np.random.default_rng(5).standard_normal((S, N, nx))
    u = torch.empty_like(T(r))
    solver.cgc_apply(T(xi), S, N, T(r), dT, alpha, 2, u)
    for s in range(S):
        ref = pcgc.cgc_diagonalized(st.operator(xi[s]), r[s], dT, alpha)
        assert rel(u[s].cpu().numpy(), ref) < 50 * 6e-8 / alpha


def test_guess_matches_oracle_surrogate():
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    info = solver.info()
    assert info.MQ == st.sur.MQ
    assert info.P == 15
    S = 9
    xi = draw_xi(S, w.M, 17)
    U0 = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.guess(T(xi), S, 0, U0)
    ref = st.guess(xi)
    assert rel(U0.cpu().numpy(), ref) < 1e-10
    solver.guess(T(xi), S, 1, U0)
    assert rel(U0.cpu().numpy(), ref) < 1e-5


def _solve(name, precision, S, seed, host=False, **over):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver(name, **over) if over else gpu_solver(name)
    xi = draw_xi(S, w.M, seed)
    if host:
        U = np.empty((S, w.N, w.nx))
        it = np.empty(S, dtype=np.int32)
        stt = np.empty(S, dtype=np.int32)
        code = solver.solve(xi, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, precision,
                            pkg.GUESS_GPC, U, it, stt)
        return code, U, it, stt, xi, w
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    stt = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, precision,
                        pkg.GUESS_GPC, U, it, stt)
    return code, U.cpu().numpy(), it.cpu().numpy(), stt.cpu().numpy(), xi, w


def test_solve_fp64_matches_oracle_iterations_and_iterates():
    code, U, it, stt, xi, w = _solve("heat1d_nx63", 0, 32, 1)
    st = oracle_setup("heat1d_nx63")
    assert code == 0 and np.all(stt == 0)
    worst = 0.0
    for s in range(32):
        Uo, ko, _ = st.solve_sample(xi[s])
        Uf, kf, _ = st.solve_sample(xi[s], cgc="dense")
        Up, kp, _ = st.solve_sample(xi[s], field_ulps=4.0)
        floor = rel(Uf, Uo) + rel(Up, Uo)
        assert it[s] == ko
        d = rel(U[s], Uo)
        worst = max(worst, d / max(1e-12, 4 * floor))
        assert d < max(1e-12, 4 * floor), (s, d, floor)
        assert rel(U[s], st.reference(xi[s])) < 1e-6
    print("worst GPU/oracle distance relative to the bar:", worst)


@pytest.mark.parametrize("precision", [1, 2])
def test_solve_mixed_reaches_fine_solution(precision):
    code, U, it, stt, xi, w = _solve("heat1d_nx63", precision, 32, 1)
    st = oracle_setup("heat1d_nx63")
    assert code == 0
    ko = np.array([st.solve_sample(x)[1] for x in xi])
    assert np.all(np.abs(it - ko) <= 1) and np.mean(it == ko) >= 0.9
    for s in range(32):
        assert rel(U[s], st.reference(xi[s])) < 1e-6


def test_solve_host_arrays_equal_device_arrays():
    a = _solve("heat1d_nx63", 0, 12, 5)
    b = _solve("heat1d_nx63", 0, 12, 5, host=True)
    assert a[0] == b[0] == 0
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_solve_is_deterministic():
    a = _solve("heat1d_nx63", 1, 16, 6)
    b = _solve("heat1d_nx63", 1, 16, 6)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_solve_edge_cases():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    dT = w.T / w.N
    U = torch.empty((4, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(4, dtype=torch.int32, device=dev())
    stt = torch.empty(4, dtype=torch.int32, device=dev())
    xi = draw_xi(4, w.M, 7)
    # empty batch
    assert solver.solve(T(xi), 0, dT, w.J, w.N, w.alpha, w.tol, 5, 0, 0, U) == pkg.OK
    # iteration cap reached
    code = solver.solve(T(xi), 4, dT, w.J, w.N, w.alpha, w.tol, 1, 0, 0, U, it, stt)
    assert code == pkg.E_NOT_CONVERGED
    assert np.all(it.cpu().numpy() == -1) and np.all(stt.cpu().numpy() == pkg.E_NOT_CONVERGED)
    # non-finite input
    bad = xi.copy()
    bad[2, 1] = np.nan
    code = solver.solve(T(bad), 4, dT, w.J, w.N, w.alpha, w.tol, 5, 0, 0, U, it, stt)
    assert code == pkg.E_NONFINITE
    # inconsistent N * dT, non power-of-two N, bad alpha
    with pytest.raises(pkg.KlecgcError) as e:
        solver.solve(T(xi), 4, dT * 1.01, w.J, w.N, w.alpha, w.tol, 5, 0, 0, U)
    assert e.value.status == pkg.E_INVALID_ARG
    with pytest.raises(pkg.KlecgcError) as e:
        solver.solve(T(xi), 4, w.T / 12, w.J, 12, w.alpha, w.tol, 5, 0, pkg.GUESS_ZERO, U)
    assert e.value.status == pkg.E_UNSUPPORTED
    with pytest.raises(pkg.KlecgcError) as e:
        solver.solve(T(xi), 4, dT, w.J, w.N, 1.5, w.tol, 5, 0, 0, U)
    assert e.value.status == pkg.E_INVALID_ARG


def test_zero_and_user_guess():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    S = 4
    xi = draw_xi(S, w.M, 8)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, 0,
                        pkg.GUESS_ZERO, U, it)
    assert code == 0
    for s in range(S):
        Z0 = np.zeros((w.N, w.nx))
        Uo, ko, _ = st.solve_sample(xi[s], U0=Z0)
        Uf, _, _ = st.solve_sample(xi[s], U0=Z0, cgc="dense")
        Up, _, _ = st.solve_sample(xi[s], U0=Z0, field_ulps=4.0)
        assert int(it[s]) == ko
        assert rel(U[s].cpu().numpy(), Uo) < max(1e-12, 4 * (rel(Uf, Uo) + rel(Up, Uo)))
    # the surrogate guess needs fewer iterations than the zero guess (Section 3.3)
    it2 = torch.empty(S, dtype=torch.int32, device=dev())
    ug = torch.empty_like(U)
    solver.guess(T(xi), S, 0, ug)
    solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, 0, pkg.GUESS_USER, U,
                 it2, U_guess=ug)
    assert np.all(it2.cpu().numpy() <= it.cpu().numpy())
    assert it2.cpu().numpy().sum() < it.cpu().numpy().sum()


@pytest.mark.parametrize("S,over", [(1, {}), (130, {}), (300, dict(gpc_degree=4, n_train=140)),
                                    (129, dict(nx=100, N=8, J=5))],
                         ids=["S1", "S130", "S300_P70", "S129_nx100"])
def test_guess_tensor_core_matches_fp64(S, over):
    """The mixed guess runs on the tcgen05 tensor cores (3xTF32 split); it must
    equal the FP64 guess (pinned to the oracle above) to FP32 accuracy on ragged
    tiles (S, N*Nx not multiples of the 128 x 256 tile; P padded to 32)."""
    solver, w = gpu_solver("heat1d_nx63", **over) if over else gpu_solver("heat1d_nx63")
    xi = draw_xi(S, w.M, 18)
    G64 = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    G32 = torch.empty_like(G64)
    solver.guess(T(xi), S, 0, G64)
    solver.guess(T(xi), S, 2, G32)
    assert rel(G32.cpu().numpy(), G64.cpu().numpy()) < 2e-6
    if over.get("gpc_degree"):
        assert solver.info().P == 70


def test_sharded_solve_equals_one_solve():
    """Samples are independent: solving a batch in three shards gives bitwise
    the same iterates and counts as one solve (the multi-GPU layout's
    premise, checked on one GPU)."""
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    S = 40
    xi = draw_xi(S, w.M, 23)
    dT = w.T / w.N
    for prec in (pkg.FP64, pkg.MIXED_DEFECT):
        U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
        it = torch.empty(S, dtype=torch.int32, device=dev())
        solver.solve(T(xi), S, dT, w.J, w.N, w.alpha, w.tol, w.kmax, prec, pkg.GUESS_GPC, U, it)
        parts = []
        for a, b in ((0, 7), (7, 29), (29, 40)):
            Us = torch.empty((b - a, w.N, w.nx), dtype=torch.float64, device=dev())
            its = torch.empty(b - a, dtype=torch.int32, device=dev())
            solver.solve(T(xi[a:b]), b - a, dT, w.J, w.N, w.alpha, w.tol, w.kmax, prec,
                         pkg.GUESS_GPC, Us, its)
            parts.append((Us, its))
        assert torch.equal(torch.cat([p[0] for p in parts]), U)
        assert torch.equal(torch.cat([p[1] for p in parts]), it)


def test_scratch_limit_reports_out_of_memory():
    """A scratch budget too small for a batch gives OUT_OF_MEMORY before any
    allocation; the context then still solves within (or without) a budget."""
    import paper_2510_26180_gb300 as pkg
    w = workload("heat1d_nx63")
    solver = pkg.Solver(pkg.Problem.from_workload(w), draw_train(w))
    S = 8
    xi = draw_xi(S, w.M, 24)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    dT = w.T / w.N
    solver.set_scratch_limit(4096)
    with pytest.raises(pkg.KlecgcError) as e:
        solver.solve(T(xi), S, dT, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.FP64, pkg.GUESS_GPC, U)
    assert e.value.status == pkg.E_OUT_OF_MEMORY
    with pytest.raises(pkg.KlecgcError) as e:
        solver.set_scratch_limit(-1)
    assert e.value.status == pkg.E_INVALID_ARG
    solver.set_scratch_limit(1 << 30)
    assert solver.solve(T(xi), S, dT, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.FP64,
                        pkg.GUESS_GPC, U) == pkg.OK
    solver.set_scratch_limit(0)
    solver.close()
