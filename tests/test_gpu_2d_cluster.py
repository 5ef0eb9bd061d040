"""2D systems held by a thread-block cluster (distributed shared memory)
against the sparse-direct CPU oracle.

klecgc_set_2d_method(3) forces the cluster layout of the mixed fine
propagator (FP64 iterative refinement around FP32 Jacobi-PCG, the same FP64
residual test ||b - M x||_2 <= rtol ||b||_2 in every step as the FP64 path)
and of the mixed shifted CGC solves (the same around FP32 Jacobi-COCG) also
on grids whose system fits one CTA, so that the layout meets the
oracle at sizes it solves in seconds: at nx = 15 a 16-CTA cluster gives
every CTA one grid row (each row is a block boundary and one CTA holds
none), at nx = 31 two rows, at nx = 63 four.  The reference solution U*
(Section 2, the sequential fine solution) takes the same layout.  Bars as
for the other 2D parity tests: 1e-12 relative L2 at rtol = 1e-14, or 4x the
oracle's own sensitivity to the last bits of the field where that is
larger.
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


def dev():
    return torch.device("cuda:0")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def cluster_solver(over):
    solver, w = gpu_solver("rd2d_255", **over)
    solver.set_krylov(RTOL, RTOL, 20000)
    solver.set_2d_method(3)
    return solver, w


@pytest.mark.parametrize("over", [SMALL, BIG], ids=["nx15", "nx63"])
def test_cluster_reference_matches_sparse_direct(over):
    from oracle import heat1d
    solver, w = cluster_solver(over)
    st = oracle_setup2d("rd2d_255", **over)
    S = 3
    xi = draw_xi(S, w.M, 61)
    U = torch.empty((S, w.N, w.nx * w.nx), dtype=torch.float64, device=dev())
    try:
        solver.reference(T(xi), S, w.N, w.J, U)
        assert solver.krylov_stats()[0] > 0
    finally:
        solver.set_2d_method(1)
    for s in range(S):
        ref = st.reference(xi[s])
        floor = rel(heat1d.fine_sequential(st.operator(xi[s], 4.0), st.u0, w.N, w.J, w.T), ref)
        d = rel(U[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * floor), (s, d, floor)


@pytest.mark.parametrize("over", [SMALL, MID, BIG], ids=["nx15", "nx31", "nx63"])
def test_cluster_fine_sweep_matches_oracle(over):
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = cluster_solver(over)
    st = oracle_setup2d("rd2d_255", **over)
    S, dT = 3, w.T / w.N
    xi = draw_xi(S, w.M, 62)
    Uin = np.stack([st.reference(x) for x in xi]) * 0.97 + 2e-3
    r = torch.empty_like(T(Uin))
    try:
        solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, pkg.MIXED, r)
        assert solver.krylov_stats()[0] > 0
    finally:
        solver.set_2d_method(1)
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
        d = rel(r[s].cpu().numpy(), ref)
        assert d < bar, (s, d, bar)


@pytest.mark.parametrize("over", [SMALL, MID], ids=["nx15", "nx31"])
def test_cluster_solve_matches_oracle(over):
    import paper_2510_26180_gb300 as pkg
    solver, w = cluster_solver(over)
    st = oracle_setup2d("rd2d_255", **over)
    S = 6
    xi = draw_xi(S, w.M, 63)
    n = w.nx * w.nx
    U = torch.empty((S, w.N, n), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    stt = torch.empty(S, dtype=torch.int32, device=dev())
    try:
        code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.MIXED,
                            pkg.GUESS_GPC, U, it, stt)
    finally:
        solver.set_2d_method(1)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for s in range(S):
        Uo, ko, _ = st.solve_sample(xi[s])
        Up, _, _ = st.solve_sample(xi[s], field_ulps=4.0)
        Uf, _, _ = st.solve_sample(xi[s], cgc="fft")
        floor = rel(Up, Uo) + rel(Uf, Uo)
        assert it[s] == ko
        assert rel(U[s], Uo) < max(1e-12, 4 * floor)


def shifted_cond(op, dT, alpha, N):
    from scipy.sparse.linalg import eigsh
    mu_max = eigsh(op.A, k=1, which="LA", return_eigenvectors=False)[0]
    mu_min = eigsh(op.A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    k = np.arange(N // 2 + 1)
    lam = 1.0 - alpha ** (1.0 / N) * np.exp(-2j * np.pi * k / N)
    return float(np.max(np.abs(lam + dT * mu_max) / np.abs(lam + dT * mu_min)))


@pytest.mark.parametrize("over,alpha", [(SMALL, 1e-3), (MID, 1e-2), (BIG, 1e-3)],
                         ids=["nx15", "nx31", "nx63"])
def test_cluster_cgc_apply_matches_oracle(over, alpha):
    """Eq. three steps on the cluster layout of step (b): bar as for the
    single-CTA kernels, including the attainable accuracy of an iterative
    solve (eps x the shifted system's condition number, scaled by step
    (c)'s alpha^{-(N-1)/N})."""
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = cluster_solver(over)
    st = oracle_setup2d("rd2d_255", **over)
    S, N, dT = 3, w.N, w.T / w.N
    n = w.nx * w.nx
    xi = draw_xi(S, w.M, 65)
    r = np.random.default_rng(10).standard_normal((S, N, n))
    u = torch.empty_like(T(r))
    try:
        solver.cgc_apply(T(xi), S, N, T(r), dT, alpha, pkg.MIXED, u)
        assert solver.krylov_stats()[1] > 0
    finally:
        solver.set_2d_method(1)
    for s in range(S):
        op = st.operator(xi[s])
        ref = pcgc.cgc_diagonalized(op, r[s], dT, alpha)
        floor = rel(pcgc.cgc_diagonalized(op, r[s], dT, alpha, fft=True), ref)
        floor += rel(pcgc.cgc_diagonalized(st.operator(xi[s], 4.0), r[s], dT, alpha), ref)
        kry = 4 * 2.2e-16 * shifted_cond(op, dT, alpha, N) * alpha ** (-(N - 1) / N)
        d = rel(u[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * floor, kry), (s, d, floor, kry)


def test_cluster_layout_is_bitwise_repeatable():
    import paper_2510_26180_gb300 as pkg
    solver, w = cluster_solver(MID)
    S, dT = 4, w.T / w.N
    xi = draw_xi(S, w.M, 64)
    Uin = np.random.default_rng(9).standard_normal((S, w.N, w.nx * w.nx)) * 0.1
    out = []
    try:
        for _ in range(2):
            r = torch.empty_like(T(Uin))
            solver.fine_sweep(T(xi), S, w.N, T(Uin), dT, w.J, w.alpha, pkg.MIXED, r)
            out.append(r.cpu().numpy())
    finally:
        solver.set_2d_method(1)
    assert np.array_equal(out[0], out[1])
