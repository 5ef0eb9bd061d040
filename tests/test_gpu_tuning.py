"""The launch-shape autotuner of the FP32 fine propagator: it records one
valid choice per (GPU, nx, N, J), every candidate shape solves to the same
accuracy (the shapes split the rows between lanes differently, so they agree
to FP32 rounding, not bit for bit), a cache file pins the choice, and with
tuning off the fixed rule applies."""
import json

import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OVER = dict(nx=511, N=16, J=8)   # candidates: factors in shared memory (W0R16), in
                                 # registers on 1 warp x 16 rows or 2 warps x 8 rows, or
                                 # one interval per warp (1 or 4 in turn) x 16 rows, or
                                 # one interval per warp x 2 halves of 8 rows (packed)
ALL = ("W0R16", "W1R16", "W2R8", "L1R16", "L4R16", "P1R16")


def _solve(solver, w, xi, precision):
    import paper_2510_26180_gb300 as pkg
    S = len(xi)
    dev = torch.device("cuda:0")
    U = torch.empty((S, w.N, w.nx), dtype=torch.float64, device=dev)
    it = torch.empty(S, dtype=torch.int32, device=dev)
    code = solver.solve(torch.from_numpy(xi).to(dev), S, w.T / w.N, w.J, w.N, w.alpha, w.tol,
                        w.kmax, precision, pkg.GUESS_GPC, U, it)
    assert code == pkg.OK
    return U.cpu().numpy(), it.cpu().numpy()


def test_tuner_records_a_valid_choice_and_shapes_agree(tmp_path):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63", **OVER)
    xi = draw_xi(12, w.M, 41)
    dev = torch.device("cuda:0")
    ref = torch.empty((12, w.N, w.nx), dtype=torch.float64, device=dev)
    solver.reference(torch.from_numpy(xi).to(dev), 12, w.N, w.J, ref)
    ref = ref.cpu().numpy()
    solver.set_tuning(1)
    _solve(solver, w, xi, pkg.MIXED)
    rep = solver.tuning_report()
    keys = [k for k in rep if "|fine32|nx=511|N=16|J=8" in k and "|ms" not in k]
    assert len(keys) == 1 and rep[keys[0]] in ALL, rep
    results = {}
    for shape in ALL:
        path = tmp_path / f"{shape}.json"
        path.write_text(json.dumps({keys[0]: shape}))
        solver.set_tuning(1, str(path))
        for prec in (pkg.MIXED, pkg.MIXED_DEFECT):
            U, it = _solve(solver, w, xi, prec)
            results[(shape, prec)] = it
            for s in range(len(xi)):
                assert rel(U[s], ref[s]) <= 1e-6, (shape, prec, s)
        assert solver.tuning_report()[keys[0]] == shape
    for prec in (pkg.MIXED, pkg.MIXED_DEFECT):
        for shape in ALL[1:]:
            a, b = results[("W0R16", prec)], results[(shape, prec)]
            assert np.all(np.abs(a - b) <= 1)
    solver.set_tuning(1)


def test_tuning_off_uses_the_rule_and_cache_file_is_written(tmp_path):
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63", nx=511, N=8, J=4)
    xi = draw_xi(4, w.M, 42)
    path = tmp_path / "cache.json"
    solver.set_tuning(1, str(path))
    _solve(solver, w, xi, pkg.MIXED)
    assert path.exists()
    on_disk = json.loads(path.read_text())
    assert any("|fine32|nx=511|N=8|J=4" in k for k in on_disk)
    solver.set_tuning(0)
    _solve(solver, w, xi, pkg.MIXED)
    with pytest.raises(pkg.KlecgcError):
        solver.set_tuning(2)
    solver.set_tuning(1)
