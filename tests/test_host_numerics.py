"""The library's host numerics of klecgc_setup against the oracle, on the CPU
(no GPU): the input-KL basis (roots of the transcendental equations by
bisection in the library, by Brent's method in the oracle; separable 2D
product modes and their order) and the gPC multi-indices with their order.
Both entry points are host-only and make no CUDA call."""
import math

import numpy as np
import pytest


def _lib():
    import __graft_entry__ as g
    g.build()
    import paper_2510_26180_gb300 as pkg
    return pkg


@pytest.mark.parametrize("sigma,ell,M", [(0.5, 0.5, 10), (0.3, 0.3, 6), (0.4, 1.0, 40)])
def test_kl_basis_1d_matches_oracle(sigma, ell, M):
    from oracle import kl_input
    pkg = _lib()
    x = np.concatenate([[0.0, 1.0], np.random.default_rng(1).random(50)])
    B, lam = pkg.kl_basis(1, ell, sigma, M, x)
    ref = kl_input.field_basis_1d(sigma, ell, M, x)
    lam_ref, _, _ = kl_input.exp_cov_modes_1d(ell, M, sigma)
    assert np.allclose(lam, lam_ref, rtol=1e-13, atol=0)
    assert np.max(np.abs(B - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.all(np.diff(lam) < 0)


@pytest.mark.parametrize("sigma,ell,M", [(0.4, 0.3, 20), (0.3, 0.3, 4), (0.5, 0.7, 60)])
def test_kl_basis_2d_matches_oracle(sigma, ell, M):
    from oracle import kl_input, rd2d
    pkg = _lib()
    P = np.random.default_rng(2).random((40, 2))
    B, lam = pkg.kl_basis(2, ell, sigma, M, P)
    ref = rd2d.field_basis_2d(sigma, ell, M, (P[:, 0], P[:, 1]))
    pairs, _ = kl_input.modes_2d(sigma, ell, M)
    assert np.allclose(lam, [q[0] for q in pairs], rtol=1e-13, atol=0)
    assert np.max(np.abs(B - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.all(np.diff(lam) <= 0)


@pytest.mark.parametrize("M,p", [(4, 2), (10, 3), (20, 2), (1, 5), (3, 0), (6, 4)])
def test_gpc_indices_match_oracle_order(M, p):
    from oracle import gpc
    pkg = _lib()
    idx = pkg.gpc_indices(M, p)
    assert idx.shape == (math.comb(M + p, p), M)
    assert np.array_equal(idx, gpc.multi_indices(M, p))


def test_host_entry_points_reject_bad_arguments():
    import ctypes
    pkg = _lib()
    lib = pkg.load()
    x = np.zeros(4)
    out = np.zeros(16)
    xp, op = x.ctypes.data, out.ctypes.data
    INV, UNS = pkg.E_INVALID_ARG, pkg.E_UNSUPPORTED
    for args, want in [((3, 0.5, 0.5, 2, xp, 2, op, None), UNS),
                       ((1, 0.5, 0.5, 0, xp, 2, op, None), INV),
                       ((2, 0.5, 0.5, 1025, xp, 2, op, None), INV),
                       ((1, 0.0, 0.5, 2, xp, 2, op, None), INV),
                       ((1, math.inf, 0.5, 2, xp, 2, op, None), INV),
                       ((1, 0.5, -1.0, 2, xp, 2, op, None), INV),
                       ((1, 0.5, math.nan, 2, xp, 2, op, None), INV),
                       ((1, 0.5, 0.5, 2, None, 2, op, None), INV),
                       ((1, 0.5, 0.5, 2, xp, -1, op, None), INV)]:
        assert lib.klecgc_kl_basis(*args) == want, args
    assert lib.klecgc_kl_basis(1, 0.5, 0.5, 2, None, 0, None, None) == pkg.OK
    P = ctypes.c_int64()
    assert lib.klecgc_gpc_indices(0, 2, None, 0, ctypes.byref(P)) == INV
    assert lib.klecgc_gpc_indices(3, -1, None, 0, ctypes.byref(P)) == INV
    assert lib.klecgc_gpc_indices(3, 2, None, 0, None) == INV
    buf = np.zeros((4, 3), dtype=np.int32)
    assert lib.klecgc_gpc_indices(3, 2, buf.ctypes.data, 4, ctypes.byref(P)) == INV
    assert P.value == 10
    assert lib.klecgc_gpc_indices(40, 12, None, 0, ctypes.byref(P)) == UNS
