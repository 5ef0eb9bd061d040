"""The 1D heat workload at full size (Nx = 1023, N = 64, J = 64, M = 10, gPC
degree 3, 4096 samples in one call), in the call the benchmark times, checked
on sampled outputs that the oracle computes one by one.

* Mixed defect path from the surrogate guess (the timed configuration): every
  sample converges within kmax and the sampled results are within 1e-6
  (relative L2) of the oracle's sequential fine solution U*.
* FP64 path from the coarse-sweep start (the oracle needs no surrogate for
  it): the sampled iteration counts equal the oracle's Algorithm 2, and the
  iterates agree within max(1e-12, 4x the oracle's own floor), the floor being
  its spread under numpy's FFT instead of the direct DFT plus its spread under
  a 4-ulp perturbation of the field (about 1e-10 at this size: the iterate is
  converged to tol = 1e-8, and where it stops depends on the last bits).
"""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAME = "heat1d_nx1023"
SAMPLED = (0, 2047, 4095)


@pytest.fixture(scope="module")
def full():
    from oracle.klecgc import Setup1D
    solver, w = gpu_solver(NAME)
    st = Setup1D(w, build=False)
    xi = draw_xi(w.S, w.M, 93)
    return solver, w, st, xi


def _solve(solver, w, xi, precision, guess):
    dev = torch.device("cuda:0")
    S = w.S
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev)
    it = torch.empty(S, dtype=torch.int32, device=dev)
    stt = torch.empty(S, dtype=torch.int32, device=dev)
    code = solver.solve(torch.from_numpy(xi).to(dev), S, w.T / w.N, w.J, w.N, w.alpha, w.tol,
                        w.kmax, precision, guess, U, it, stt)
    rows = {s: U[s].cpu().numpy() for s in SAMPLED}
    return code, rows, it.cpu().numpy(), stt.cpu().numpy()


def test_timed_configuration_sampled_against_oracle(full):
    import paper_2510_26180_gb300 as pkg
    solver, w, st, xi = full
    code, rows, it, stt = _solve(solver, w, xi, pkg.MIXED_DEFECT, pkg.GUESS_GPC)
    assert code == pkg.OK
    assert np.all(stt == pkg.OK)
    assert np.all((it >= 1) & (it <= w.kmax))
    for s in SAMPLED:
        d = rel(rows[s], st.reference(xi[s]))
        assert d < 1e-6, (s, d)


def test_fp64_sampled_iterations_and_iterates_against_oracle(full):
    import paper_2510_26180_gb300 as pkg
    from oracle import pcgc
    solver, w, st, xi = full
    code, rows, it, stt = _solve(solver, w, xi, pkg.FP64, pkg.GUESS_COARSE)
    assert code == pkg.OK
    assert np.all(stt == pkg.OK)
    dT = w.T / w.N
    for s in SAMPLED:
        op = st.operator(xi[s])
        U0 = pcgc.coarse_guess(op, st.u0, w.N, dT)
        Uo, ko, _ = pcgc.pcgc_solve(op, st.u0, U0, dT, w.J, w.alpha, w.tol, w.kmax)
        Uf, _, _ = pcgc.pcgc_solve(op, st.u0, U0, dT, w.J, w.alpha, w.tol, w.kmax, cgc="fft")
        Up, _, _ = pcgc.pcgc_solve(st.operator(xi[s], 4.0), st.u0, U0, dT, w.J, w.alpha,
                                   w.tol, w.kmax)
        floor = rel(Uf, Uo) + rel(Up, Uo)
        assert it[s] == ko, (s, it[s], ko)
        d = rel(rows[s], Uo)
        assert d < max(1e-12, 4 * floor), (s, d, floor)
