"""Every launch shape of the FP32 fine propagator against the oracle's F
(Algorithm 2, step 1: J backward-Euler steps of I + dt(A + cI) on every
subinterval), each forced in turn through the autotuner's cache file:

* k_fine32 (W0R..): one warp per pair of intervals, factors in shared memory;
* k_fine32w (W1.., W2.., W4..): factors in registers, W warps per pair;
* k_fine32r (L1.., L4..): one interval per warp, factors in registers, the
  backward sweep regrouped as x = X + yin P + zin G;
* k_fine32p (P1..): as k_fine32r with each lane's rows split into two halves
  swept together in packed FP32x2 (another partition of the rows, so another
  rounding, within the same bar).

klecgc_fine_sweep returns r_n = (I + dT(A + cI)) F_n - prev_n in FP64; the
test recovers F_n = (I + dT(A + cI))^{-1} (r_n + prev_n) with the oracle's
banded solve (FP64, so the recovery adds ~1e-12 to the FP32 values) and
compares it with the oracle's F in FP64.  Start values in flux form every step
(the first launch of a solve): each step rounds a row about eight times
(flux differences, the two sweeps, the carry corrections) and the step map is
a contraction, so after J steps the error stays below J x 8 x 2^-24 relative
(3e-5 at J = 64), and in practice, the roundings being independent, near
sqrt(J) x 8 x 2^-24; the bar is 1e-5.  The increment form of the later
iterations (flux form every 16th or 32nd step) is covered by a whole mixed solve per
shape, which must reach U* to 1e-6 with iteration counts within one of the
shared-memory kernel's."""
import json

import numpy as np
import pytest

from synth import draw_xi, workload
from tests.gpu_util import gpu_solver, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = {
    63: ["W0R2", "W1R2", "L1R2", "L4R2"],
    127: ["W0R4", "L1R4", "L4R4", "P1R4"],
    255: ["W0R8", "L1R8", "L4R8", "P1R8"],
    511: ["W0R16", "W1R16", "W2R8", "L1R16", "L4R16", "P1R16"],
    1023: ["W0R32", "W2R16", "W4R8", "L1R32", "L4R32", "P1R32"],
}
SMALL = dict(M=2, gpc_degree=1, n_train=6)


def _force(solver, w, shape, tmp_path):
    key = f"{torch.cuda.get_device_name(0)}|fine32|nx={w.nx}|N={w.N}|J={w.J}"
    path = tmp_path / f"{shape}.json"
    path.write_text(json.dumps({key: shape}))
    solver.set_tuning(1, str(path))
    return key


def _oracle_F(w, xi, Uin):
    from oracle import pcgc
    from oracle.klecgc import Setup1D
    st = Setup1D(w, build=False)
    dT = w.T / w.N
    out = []
    for s in range(len(xi)):
        op = st.operator(xi[s])
        out.append(pcgc.fine_sweep(op, st.u0, Uin[s], dT, w.J))
    return np.stack(out), st


@pytest.mark.parametrize("nx,J", [(63, 16), (127, 16), (255, 16), (511, 16), (1023, 64)])
@pytest.mark.parametrize("react", [(0.0, 0.0), (0.7, 0.4)])
def test_each_fine_shape_matches_the_oracle_F(nx, J, react, tmp_path):
    import paper_2510_26180_gb300 as pkg
    c, f = react
    solver, w = gpu_solver("heat1d_nx63", nx=nx, N=8, J=J, reaction=c, forcing=f, **SMALL)
    S, dT = 3, w.T / w.N
    xi = draw_xi(S, w.M, 51)
    x = np.linspace(0.0, 1.0, nx + 2)[1:-1]
    # smooth start values of solution size, different per interval and sample
    Uin = np.stack([[np.sin(np.pi * x) * (1.0 + 0.1 * n) + 0.05 * s * np.sin(3 * np.pi * x)
                     for n in range(w.N)] for s in range(S)])
    Fo, st = _oracle_F(w, xi, Uin)
    dev = torch.device("cuda:0")
    prev = np.concatenate([w.alpha * Uin[:, -1:], Uin[:, :-1]], axis=1)
    try:
        for shape in SHAPES[nx]:
            key = _force(solver, w, shape, tmp_path)
            r = torch.empty((S, w.N, nx), dtype=torch.float64, device=dev)
            solver.fine_sweep(torch.from_numpy(xi).to(dev), S, w.N,
                              torch.from_numpy(Uin).to(dev), dT, w.J, w.alpha, pkg.MIXED, r)
            assert solver.tuning_report()[key] == shape
            r = r.cpu().numpy()
            for s in range(S):
                op = st.operator(xi[s])
                Fg = op.shifted_solve(1.0, dT, r[s] + prev[s])
                assert rel(Fg, Fo[s]) < 1e-5, (shape, s, rel(Fg, Fo[s]))
    finally:
        solver.set_tuning(1)


@pytest.mark.parametrize("nx,J", [(511, 16), (1023, 64)])
def test_each_fine_shape_solves_to_the_fine_solution(nx, J, tmp_path):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63", nx=nx, N=8, J=J, **SMALL)
    S = 6
    xi = draw_xi(S, w.M, 52)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(xi).to(dev)
    ref = torch.empty((S, w.N, nx), dtype=torch.float64, device=dev)
    solver.reference(x, S, w.N, w.J, ref)
    ref = ref.cpu().numpy()
    iters = {}
    try:
        for shape in SHAPES[nx]:
            _force(solver, w, shape, tmp_path)
            U = torch.empty((S, w.N, nx), dtype=torch.float64, device=dev)
            it = torch.empty(S, dtype=torch.int32, device=dev)
            code = solver.solve(x, S, w.T / w.N, w.J, w.N, w.alpha, w.tol, w.kmax, pkg.MIXED,
                                pkg.GUESS_GPC, U, it)
            assert code == pkg.OK, shape
            U = U.cpu().numpy()
            for s in range(S):
                assert rel(U[s], ref[s]) <= 1e-6, (shape, s)
            iters[shape] = it.cpu().numpy()
    finally:
        solver.set_tuning(1)
    base = iters[SHAPES[nx][0]]
    for shape, it in iters.items():
        assert np.all(np.abs(it - base) <= 1), (shape, it, base)
