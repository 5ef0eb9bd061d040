"""The offline stage of Algorithm 3 on the device (snapshots, Gram matrix,
Jacobi eigenpairs, modes, Householder least squares) against the oracle's
numpy/scipy surrogate built from the same training set: retained mode count,
captured energy and the guess, from n_t = 2P up to 64P training snapshots,
and with a rank-deficient Gram matrix (every training point twice)."""
import numpy as np
import pytest

from synth import draw_train, draw_xi, workload
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev():
    return torch.device("cuda:0")


def _setups(w, xi_train):
    import __graft_entry__ as g
    g.build()
    import paper_2510_26180_gb300 as pkg
    from oracle.klecgc import Setup1D
    solver = pkg.Solver(pkg.Problem.from_workload(w), xi_train)
    st = Setup1D(w, xi_train=xi_train)
    return solver, st


@pytest.mark.parametrize("n_train", [30, 240, 960], ids=["2P", "16P", "64P"])
def test_offline_stage_matches_oracle_surrogate(n_train):
    w = workload("heat1d_nx63", n_train=n_train)
    solver, st = _setups(w, draw_train(w))
    info = solver.info()
    assert info.MQ == st.sur.MQ
    assert abs(info.lambda_kept - float(np.sum(st.sur.lam))) <= 1e-12 * info.lambda_kept
    S = 8
    xi = draw_xi(S, w.M, 19)
    U0 = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.guess(torch.from_numpy(xi).to(dev()), S, 0, U0)
    ref = st.guess(xi)
    # the retained modes with the smallest eigenvalues carry eigenvector
    # rounding of order eps ||C|| / gap: the oracle's own floor is the
    # distance between its eigh- and SVD-based surrogates
    floor = rel(st.surrogate_svd().guess(xi).reshape(ref.shape), ref)
    d = rel(U0.cpu().numpy(), ref)
    assert d < max(1e-10, 4 * floor), (d, floor)
    solver.close()


def test_offline_stage_with_a_rank_deficient_gram_matrix():
    w = workload("heat1d_nx63")
    xt = draw_train(w)
    xi_train = np.concatenate([xt, xt])          # n_t = 60, rank <= 29
    w = w.with_(n_train=len(xi_train))
    solver, st = _setups(w, xi_train)
    info = solver.info()
    assert info.MQ == st.sur.MQ and info.MQ <= len(xt) - 1
    S = 6
    xi = draw_xi(S, w.M, 20)
    U0 = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
    solver.guess(torch.from_numpy(xi).to(dev()), S, 0, U0)
    ref = st.guess(xi)
    floor = rel(st.surrogate_svd().guess(xi).reshape(ref.shape), ref)
    d = rel(U0.cpu().numpy(), ref)
    assert d < max(1e-10, 4 * floor), (d, floor)
    solver.close()
