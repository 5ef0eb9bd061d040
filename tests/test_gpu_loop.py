"""The device-driven parareal loop (a CUDA graph whose WHILE node repeats one
captured iteration until the stopping rule of Algorithm 2, Step 3, finds no
active sample or kmax iterations have run) against the host-driven loop:
the same kernels in the same order, so the iterates, iteration counts and
statuses must be bitwise equal, also when kmax cuts the loop short and when
every sample converges in the first iteration."""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solve(solver, w, xi, precision, guess, mode, kmax=None, parareal=False, S=None):
    S = S or len(xi)
    dev = torch.device("cuda:0")
    U = torch.full((S, w.N, w.nx ** w.dim), float("nan"), dtype=torch.float64, device=dev)
    it = torch.full((S,), -7, dtype=torch.int32, device=dev)
    st = torch.full((S,), -7, dtype=torch.int32, device=dev)
    solver.set_loop(mode)
    try:
        x = torch.from_numpy(xi).to(dev)
        if parareal:
            code = solver.solve_parareal(x, S, w.T / w.N, w.J, w.N, w.tol, kmax or w.kmax, guess,
                                         U, it, st)
        else:
            code = solver.solve(x, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, kmax or w.kmax,
                                precision, guess, U, it, st)
    finally:
        solver.set_loop(0)
    return code, U.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def _equal(a, b):
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[3], b[3])


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "MIXED_DEFECT"])
@pytest.mark.parametrize("kmax", [None, 3])
def test_graph_loop_bitwise_equals_host_loop_1d(precision, kmax):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    xi = draw_xi(24, w.M, 31)
    p = getattr(pkg, precision)
    g = _solve(solver, w, xi, p, pkg.GUESS_GPC, 0, kmax)
    h = _solve(solver, w, xi, p, pkg.GUESS_GPC, 1, kmax)
    _equal(g, h)
    if kmax is None:
        assert g[0] == pkg.OK and np.all(g[2] >= 1)
    else:
        assert np.all(g[2] == -1) and np.all(g[3] == pkg.E_NOT_CONVERGED)


def test_graph_loop_when_first_iteration_converges():
    # the user guess is the converged solution: every sample stops after one
    # iteration, and the loop body after it must change nothing
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    xi = draw_xi(8, w.M, 32)
    _, U, _, _ = _solve(solver, w, xi, pkg.FP64, pkg.GUESS_GPC, 1)
    dev = torch.device("cuda:0")
    out = []
    for mode in (0, 1):
        solver.set_loop(mode)
        Ug = torch.empty((8, w.N, w.nx), dtype=torch.float64, device=dev)
        it = torch.empty(8, dtype=torch.int32, device=dev)
        code = solver.solve(torch.from_numpy(xi).to(dev), 8, w.T / w.N, w.J, w.N, w.alpha, w.tol,
                            w.kmax, pkg.FP64, pkg.GUESS_USER, Ug, it,
                            U_guess=torch.from_numpy(U).to(dev))
        solver.set_loop(0)
        out.append((code, Ug.cpu().numpy(), it.cpu().numpy()))
    assert out[0][0] == out[1][0] == pkg.OK
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert np.all(out[0][2] == 1)


def test_graph_loop_classical_parareal_and_2d():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    xi = draw_xi(12, w.M, 33)
    _equal(_solve(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE, 0, parareal=True),
           _solve(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE, 1, parareal=True))
    s2, w2 = gpu_solver("rd2d_255", nx=15, N=8, J=4, M=4, gpc_degree=1, n_train=10)
    xi2 = draw_xi(6, w2.M, 34)
    _equal(_solve(s2, w2, xi2, pkg.FP64, pkg.GUESS_GPC, 0),
           _solve(s2, w2, xi2, pkg.FP64, pkg.GUESS_GPC, 1))


@pytest.mark.parametrize("name", ["ac1d_nx127", "burgers1d_nx99"])
def test_graph_loop_nonlinear(name):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver(name, N=16, J=8)
    xi = draw_xi(6, w.M, 35)
    _equal(_solve(solver, w, xi, pkg.FP64, pkg.GUESS_GPC, 0),
           _solve(solver, w, xi, pkg.FP64, pkg.GUESS_GPC, 1))
    _equal(_solve(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE, 0, parareal=True),
           _solve(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE, 1, parareal=True))


def test_set_loop_rejects_other_modes():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    with pytest.raises(pkg.KlecgcError):
        solver.set_loop(2)
