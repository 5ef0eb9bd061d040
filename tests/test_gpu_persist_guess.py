"""Context files (klecgc_save / klecgc_load) and the coarse-sweep guess."""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, oracle_setup, oracle_setup2d, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL2D = dict(nx=15, N=8, J=4, M=6, gpc_degree=2, n_train=56)


def dev():
    return torch.device("cuda:0")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def _run(solver, w, xi, precision, guess):
    S = xi.shape[0]
    U = torch.empty((S, w.N, w.nx ** w.dim), dtype=torch.float64, device=dev())
    it = torch.empty(S, dtype=torch.int32, device=dev())
    code = solver.solve(T(xi), S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, precision, guess,
                        U, it)
    return code, U.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("name,over", [("heat1d_nx63", {}), ("rd2d_255", SMALL2D)],
                         ids=["1d", "2d"])
def test_saved_context_reproduces_solves(tmp_path, name, over):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver(name, **over)
    if w.dim == 2:
        solver.set_krylov(1e-13, 1e-13, 5000)
    elif solver.mlp_n_params():
        rng = np.random.default_rng(0)
        solver.mlp_set(torch.from_numpy(0.01 * rng.standard_normal(solver.mlp_n_params())
                                        .astype(np.float32)).to(dev()))
    xi = draw_xi(8, w.M, 41)
    precisions = (pkg.FP64,) if w.dim == 2 else (pkg.FP64, pkg.MIXED_DEFECT)
    # the autotuner's launch-shape choices travel with the file: solve once
    # before saving so that they exist (a context that has not tuned yet and
    # its copy would each time the candidates on their own)
    for prec in precisions:
        _run(solver, w, xi, prec, pkg.GUESS_GPC)
    path = str(tmp_path / "ctx.klecgc")
    solver.save(path)
    loaded = pkg.Solver.load(path)
    assert loaded.tuning_report() == solver.tuning_report()
    a, b = solver.info(), loaded.info()
    for f in ("nx", "N", "J", "M", "P", "MQ", "n_unknowns"):
        assert getattr(a, f) == getattr(b, f)
    assert a.lambda_kept == b.lambda_kept
    for prec in precisions:
        c1, U1, i1 = _run(solver, w, xi, prec, pkg.GUESS_GPC)
        c2, U2, i2 = _run(loaded, w, xi, prec, pkg.GUESS_GPC)
        assert c1 == c2 == 0
        assert np.array_equal(i1, i2) and np.array_equal(U1, U2)
    if w.dim == 1:
        g1 = torch.empty((8, w.N, w.nx), dtype=torch.float64, device=dev())
        g2 = torch.empty_like(g1)
        solver.mlp_guess(T(xi), 8, g1)
        loaded.mlp_guess(T(xi), 8, g2)
        assert torch.equal(g1, g2)
    loaded.close()


def test_coarse_guess_1d_matches_oracle():
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = gpu_solver("heat1d_nx63")
    st = oracle_setup("heat1d_nx63")
    xi = draw_xi(6, w.M, 42)
    code, U, it = _run(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE)
    assert code == 0
    for s in range(6):
        op = st.operator(xi[s])
        U0 = pcgc.coarse_guess(op, st.u0, w.N, w.T / w.N)
        Uo, ko, _ = st.solve_sample(xi[s], U0=U0)
        Up, _, _ = st.solve_sample(xi[s], U0=U0, field_ulps=4.0)
        Uf, _, _ = st.solve_sample(xi[s], U0=U0, cgc="dense")
        assert it[s] == ko
        assert rel(U[s], Uo) < max(1e-12, 4 * (rel(Up, Uo) + rel(Uf, Uo)))


def test_coarse_guess_2d_matches_oracle():
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w = gpu_solver("rd2d_255", **SMALL2D)
    solver.set_krylov(1e-14, 1e-14, 20000)
    st = oracle_setup2d("rd2d_255", **SMALL2D)
    xi = draw_xi(4, w.M, 43)
    code, U, it = _run(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE)
    assert code == 0
    for s in range(4):
        op = st.operator(xi[s])
        U0 = pcgc.coarse_guess(op, st.u0, w.N, w.T / w.N)
        Uo, ko, _ = st.solve_sample(xi[s], U0=U0)
        Up, _, _ = st.solve_sample(xi[s], U0=U0, field_ulps=4.0)
        Uf, _, _ = st.solve_sample(xi[s], U0=U0, cgc="fft")
        assert it[s] == ko
        assert rel(U[s], Uo) < max(1e-12, 4 * (rel(Up, Uo) + rel(Uf, Uo)))
