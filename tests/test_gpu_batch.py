"""Uneven batch (klecgc_solve_batch): instances with different grids, time
partitions and fine steps solved together equal the same instances solved
class by class with klecgc_solve (bit for bit: every sample's arithmetic is
independent of the batch composition; on the mixed paths the batch runs each
stage as one persistent launch over all classes with the same per-tile
bodies, and the per-class solves use the same fine kernel with the
autotuner off), which the parity tests pin to the oracle; a few instances
are also checked against the oracle directly."""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, oracle_setup, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CTXS = [("heat1d_nx63", {}), ("heat1d_nx63", dict(nx=100, N=8, J=5)),
        ("heat1d_nx63", dict(nx=33, N=4, J=3))]


def dev():
    return torch.device("cuda:0")


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    ci = rng.integers(0, len(CTXS), n)
    J = rng.choice([2, 3, 8, 16], n)
    return ci, J


def _solvers():
    return [gpu_solver(name, **over) for name, over in CTXS]


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "mixed_defect"])
@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_batch_equals_per_class_solves(precision, host):
    import paper_2510_26180_gb300 as pkg
    sv = _solvers()
    for s, _ in sv:
        s.set_tuning(0)
    n = 40
    ci, J = _batch(n, 7)
    M = sv[0][1].M
    xi = draw_xi(n, M, 51)
    sizes = [sv[c][1].N * sv[c][1].nx for c in ci]
    off = np.concatenate([[0], np.cumsum(sizes)])
    if host:
        U = np.empty(off[-1])
        it = np.empty(n, dtype=np.int32)
        stt = np.empty(n, dtype=np.int32)
        code = pkg.solve_batch([s for s, _ in sv], ci, J, xi, 1e-3, 1e-8, 60, precision,
                               pkg.GUESS_GPC, U, it, stt)
    else:
        Ud = torch.empty(int(off[-1]), dtype=torch.float64, device=dev())
        itd = torch.empty(n, dtype=torch.int32, device=dev())
        sttd = torch.empty(n, dtype=torch.int32, device=dev())
        code = pkg.solve_batch([s for s, _ in sv], ci, J, torch.from_numpy(xi).to(dev()), 1e-3,
                               1e-8, 60, precision, pkg.GUESS_GPC, Ud, itd, sttd)
        U, it, stt = Ud.cpu().numpy(), itd.cpu().numpy(), sttd.cpu().numpy()
    assert code == 0 and np.all(stt == 0)
    for c in range(len(CTXS)):
        for j in sorted(set(J[ci == c])):
            ids = np.nonzero((ci == c) & (J == j))[0]
            s, w = sv[c]
            S = len(ids)
            Uc = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev())
            itc = torch.empty(S, dtype=torch.int32, device=dev())
            s.solve(torch.from_numpy(xi[ids]).to(dev()), S, w.T / w.N, int(j), w.N, 1e-3, 1e-8,
                    60, precision, pkg.GUESS_GPC, Uc, itc)
            Uc, itc = Uc.cpu().numpy(), itc.cpu().numpy()
            for q, i in enumerate(ids):
                blk = U[off[i]:off[i + 1]].reshape(w.N, w.nx)
                assert np.array_equal(blk, Uc[q]), (c, j, i)
                assert it[i] == itc[q]
    for s, _ in sv:
        s.set_tuning(1)


def test_batch_instances_match_oracle():
    import paper_2510_26180_gb300 as pkg
    sv = _solvers()
    n = 12
    ci, J = _batch(n, 8)
    xi = draw_xi(n, sv[0][1].M, 52)
    sizes = [sv[c][1].N * sv[c][1].nx for c in ci]
    off = np.concatenate([[0], np.cumsum(sizes)])
    U = torch.empty(int(off[-1]), dtype=torch.float64, device=dev())
    it = torch.empty(n, dtype=torch.int32, device=dev())
    code = pkg.solve_batch([s for s, _ in sv], ci, J, torch.from_numpy(xi).to(dev()), 1e-3,
                           1e-8, 60, pkg.FP64, pkg.GUESS_GPC, U, it)
    assert code == 0
    U, it = U.cpu().numpy(), it.cpu().numpy()
    for i in range(n):
        name, over = CTXS[ci[i]]
        st = oracle_setup(name, **over)
        w = st.w.with_(J=int(J[i]))
        from oracle import pcgc
        op = st.operator(xi[i])
        Uo, ko, _ = pcgc.pcgc_solve(op, st.u0, st.guess(xi[i])[0], w.T / w.N, w.J, 1e-3, 1e-8, 60)
        Uf, _, _ = pcgc.pcgc_solve(op, st.u0, st.guess(xi[i])[0], w.T / w.N, w.J, 1e-3, 1e-8, 60,
                                   cgc="dense")
        Up, _, _ = pcgc.pcgc_solve(st.operator(xi[i], 4.0), st.u0, st.guess(xi[i])[0], w.T / w.N,
                                   w.J, 1e-3, 1e-8, 60)
        floor = rel(Uf, Uo) + rel(Up, Uo)
        blk = U[off[i]:off[i + 1]].reshape(w.N, w.nx)
        assert it[i] == ko
        assert rel(blk, Uo) < max(1e-12, 4 * floor)


def test_batch_argument_errors():
    import paper_2510_26180_gb300 as pkg
    sv = _solvers()
    xi = draw_xi(2, sv[0][1].M, 53)
    U = torch.empty(10, dtype=torch.float64, device=dev())
    with pytest.raises(pkg.KlecgcError) as e:
        pkg.solve_batch([s for s, _ in sv], [0, 5], [4, 4], xi, 1e-3, 1e-8, 5, 0, pkg.GUESS_GPC, U)
    assert e.value.status == pkg.E_INVALID_ARG
    with pytest.raises(pkg.KlecgcError) as e:
        pkg.solve_batch([s for s, _ in sv], [0, 1], [4, 0], xi, 1e-3, 1e-8, 5, 0, pkg.GUESS_GPC, U)
    assert e.value.status == pkg.E_INVALID_ARG
    with pytest.raises(pkg.KlecgcError) as e:
        pkg.solve_batch([s for s, _ in sv], [0, 1], [4, 4], xi, 1e-3, 1e-8, 5, 0, pkg.GUESS_USER, U)
    assert e.value.status == pkg.E_INVALID_ARG
