"""klecgc_reference_noalloc: the allocation-free variant of klecgc_reference.

It serves callers that cannot allocate device memory (for instance code that
runs under another framework's caching allocator, or hosts that forbid
allocation after start-up); its working memory is a fixed array compiled into
the library.  Here its output is checked against klecgc_reference through the
C ABI on two calls in a row (the second reuses the array the first one left
behind), and its size limit and argument checks are exercised.  The file is
named to be collected after the parity tests.
"""
import numpy as np
import pytest

from synth import draw_xi
from tests.gpu_util import gpu_solver, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCRATCH_DOUBLES = (32 << 20) // 8


def _run(solver, w, S, seed):
    import paper_2510_26180_gb300 as pkg  # noqa: F401
    xi = torch.from_numpy(draw_xi(S, w.M, seed)).cuda()
    ref = torch.empty((S, w.N, w.nx), dtype=torch.float64, device="cuda")
    out = torch.full_like(ref, float("nan"))
    solver.reference(xi, S, w.N, w.J, ref)
    solver.reference_noalloc(xi, S, w.N, w.J, out)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_reference_on_two_calls():
    solver, w = gpu_solver("heat1d_nx63")
    for S, seed in ((9, 21), (40, 22)):
        ref, out = _run(solver, w, S, seed)
        assert np.all(np.isfinite(out))
        assert rel(out, ref) <= 1e-12


def test_noalloc_rejects_sizes_beyond_the_array():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    S = SCRATCH_DOUBLES // (6 * w.nx + 5) + 1
    xi = torch.zeros((S, w.M), dtype=torch.float64, device="cuda")
    out = torch.empty((S, w.N, w.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.KlecgcError) as e:
        solver.reference_noalloc(xi, S, w.N, w.J, out)
    assert e.value.status == pkg.E_INVALID_ARG
    assert "exceeds the static scratch" in str(e.value)
    # host arrays are refused too: staging them would need an allocation
    with pytest.raises(pkg.KlecgcError) as e:
        solver.reference_noalloc(np.zeros((2, w.M)), 2, w.N, w.J, out)
    assert e.value.status == pkg.E_INVALID_ARG
