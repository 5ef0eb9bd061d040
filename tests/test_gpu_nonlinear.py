"""Nonlinear problems on the GPU (cubic reaction and Burgers-type convection,
simplified-Newton CGC) against the oracle: the Newton reference, whole
solves with iteration counts, the coarse start, classical parareal with
Newton propagators, the reduction to the linear problem at c = 0, and the
modes they reject.  Bars as for the linear FP64 path: 1e-12 relative L2, or
4x the oracle's own floor (dense instead of diagonalized Jbar solves, and the
field perturbed by 4 ulps) where that is larger."""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, oracle_setup_ac, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = dict(N=16, J=8)
PROBLEMS = ["ac1d_nx127", "burgers1d_nx99"]


def dev():
    return torch.device("cuda:0")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


@pytest.mark.parametrize("name", PROBLEMS)
def test_nonlinear_reference_matches_oracle(name):
    from oracle import nonlinear as nl
    solver, w = gpu_solver(name, **SMALL)
    st = oracle_setup_ac(name, **SMALL)
    S = 4
    xi = draw_xi(S, w.M, 71)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.reference(T(xi), S, w.N, w.J, U)
    for s in range(S):
        ref = st.reference(xi[s])
        refp = nl.fine_sequential(st.operator(xi[s], 4.0), st.u0, w.N, w.J, w.T)
        d = rel(U[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * rel(refp, ref)), d


@pytest.mark.parametrize("name", PROBLEMS)
@pytest.mark.parametrize("nx", [17, 128, 200, 300])
def test_nonlinear_reference_across_lane_shapes(name, nx):
    """The Newton propagator splits a column over 16 lanes up to 128 rows,
    32 lanes up to 256 (8 rows per lane, padded with identity rows) and
    keeps one thread per column above: U* of each shape against the
    oracle's sequential Newton solution."""
    from oracle import nonlinear as nl
    over = dict(nx=nx, N=8, J=4, M=3, gpc_degree=1, n_train=8)
    solver, w = gpu_solver(name, **over)
    st = oracle_setup_ac(name, **over)
    S = 3
    xi = draw_xi(S, w.M, 74)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.reference(T(xi), S, w.N, w.J, U)
    for s in range(S):
        ref = st.reference(xi[s])
        refp = nl.fine_sequential(st.operator(xi[s], 4.0), st.u0, w.N, w.J, w.T)
        d = rel(U[s].cpu().numpy(), ref)
        assert d < max(1e-12, 4 * rel(refp, ref)), (nx, s, d)


@pytest.mark.parametrize("name", PROBLEMS)
@pytest.mark.parametrize("guess", ["gpc", "coarse"])
def test_nonlinear_solve_matches_oracle(name, guess):
    import paper_2510_26180_gb300 as pkg
    from oracle import nonlinear as nl
    solver, w = gpu_solver(name, **SMALL)
    st = oracle_setup_ac(name, **SMALL)
    S = 4
    xi = draw_xi(S, w.M, 72)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    g = pkg.GUESS_GPC if guess == "gpc" else pkg.GUESS_COARSE
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.FP64, g, U, it)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for s in range(S):
        op = st.operator(xi[s])
        U0 = st.guess(xi[s])[0] if guess == "gpc" else \
            np.stack(list(_coarse(nl, op, st.u0, w.N, w.T / w.N)))
        Uo, ko, _ = st.solve_sample(xi[s], U0=U0)
        Ud, _, _ = st.solve_sample(xi[s], U0=U0, cgc="dense")
        Up, _, _ = st.solve_sample(xi[s], U0=U0, field_ulps=4.0)
        floor = rel(Ud, Uo) + rel(Up, Uo)
        assert it[s] == ko, (s, it[s], ko)
        assert rel(U[s], Uo) < max(1e-12, 4 * floor), (s, rel(U[s], Uo), floor)
        assert rel(U[s], st.reference(xi[s])) < 1e-6


@pytest.mark.parametrize("name", PROBLEMS)
def test_nonlinear_parareal_matches_oracle(name):
    """Algorithm 1 with Newton F and G from the gPC guess (KLE-CGC of the
    paper's nonlinear experiments): iteration counts equal, iterates at the
    oracle's floor, the end point at the sequential fine solution."""
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = gpu_solver(name, **SMALL)
    st = oracle_setup_ac(name, **SMALL)
    S = 4
    xi = draw_xi(S, w.M, 75)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve_parareal(T(xi), S, w.T / w.N, w.J, w.N, w.tol, w.N + 1, pkg.GUESS_GPC,
                                 U, it)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for s in range(S):
        U0 = st.guess(xi[s])[0]
        its = pcgc.parareal_classical(st.operator(xi[s]), st.u0, U0, w.T / w.N, w.J, w.N + 1)
        ko = next(k for k in range(1, len(its)) if np.max(np.abs(its[k] - its[k - 1])) <= w.tol)
        assert it[s] == ko, (s, it[s], ko)
        itp = pcgc.parareal_classical(st.operator(xi[s], 4.0), st.u0, U0, w.T / w.N, w.J, ko)
        floor = rel(itp[ko], its[ko])
        assert rel(U[s], its[ko]) < max(1e-12, 4 * floor), (s, rel(U[s], its[ko]), floor)
        assert rel(U[s], st.reference(xi[s])) < 1e-6


def _coarse(nl, op, u0, N, dT):
    v = np.asarray(u0, dtype=np.float64)
    for _ in range(N):
        v = nl.G(op, v, dT)
        yield v


@pytest.mark.parametrize("name", PROBLEMS)
def test_nonlinear_solve_with_32_lanes_per_column(name):
    """Whole solves from the coarse start at nx = 200 (F and its jump on 32
    lanes per column): iteration counts equal to the oracle's, iterates at
    its floor."""
    import paper_2510_26180_gb300 as pkg
    from oracle import nonlinear as nl
    over = dict(nx=200, N=8, J=4, M=3, gpc_degree=1, n_train=8)
    solver, w = gpu_solver(name, **over)
    st = oracle_setup_ac(name, **over)
    S = 3
    xi = draw_xi(S, w.M, 75)
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.FP64,
                        pkg.GUESS_COARSE, U, it)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for s in range(S):
        op = st.operator(xi[s])
        U0 = np.stack(list(_coarse(nl, op, st.u0, w.N, w.T / w.N)))
        Uo, ko, _ = st.solve_sample(xi[s], U0=U0)
        Ud, _, _ = st.solve_sample(xi[s], U0=U0, cgc="dense")
        Up, _, _ = st.solve_sample(xi[s], U0=U0, field_ulps=4.0)
        floor = rel(Ud, Uo) + rel(Up, Uo)
        assert it[s] == ko, (s, it[s], ko)
        assert rel(U[s], Uo) < max(1e-12, 4 * floor), (s, rel(U[s], Uo), floor)


def test_zero_reaction_matches_the_linear_solver():
    import paper_2510_26180_gb300 as pkg
    lin, w = gpu_solver("heat1d_nx63")
    nlin, _ = gpu_solver("heat1d_nx63", reaction_kind=1, cgc_newton=2)
    S = 6
    xi = T(draw_xi(S, w.M, 73))
    U1 = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    U2 = torch.empty_like(U1)
    i1 = torch.empty(S, dtype=torch.int32, device=dev())
    i2 = torch.empty_like(i1)
    assert lin.solve(xi, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, 0, pkg.GUESS_GPC, U1, i1) == 0
    assert nlin.solve(xi, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, 0, pkg.GUESS_GPC, U2, i2) == 0
    assert torch.equal(i1, i2)
    assert rel(U2.cpu().numpy(), U1.cpu().numpy()) < 1e-10


def test_nonlinear_rejects_unsupported_modes():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("ac1d_nx127", **SMALL)
    S = 2
    xi = T(draw_xi(S, w.M, 74))
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    for call in (
        lambda: solver.solve(xi, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, 5, pkg.MIXED_DEFECT,
                             pkg.GUESS_GPC, U),
        lambda: solver.fine_sweep(xi, S, w.N, U, w.T / w.N, w.J, w.alpha, 0, U),
        lambda: solver.reference_noalloc(xi, S, w.N, w.J, U),
    ):
        with pytest.raises(pkg.KlecgcError) as e:
            call()
        assert e.value.status == pkg.E_UNSUPPORTED
