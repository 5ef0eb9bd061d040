"""Pins of the oracle's Algorithm 3 offline part (snapshot KL + gPC LS)."""
import numpy as np

from oracle import gpc
from oracle.surrogate import build_surrogate


def _poly_snapshots(nt, M, p, dim, modes, seed):
    """Synthetic snapshots whose coefficients are polynomials of degree <= p."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((dim, modes)))
    mean = rng.standard_normal(dim)
    idx = gpc.multi_indices(M, p)
    coef = rng.standard_normal((modes, len(idx)))

    def field(xi):
        # monomials (not the gPC basis) so the test does not reuse psi_matrix
        mono = np.stack([np.prod(xi ** k[None, :], axis=1) for k in idx], axis=1)
        return mean[None, :] + (mono @ coef.T) @ Q.T

    xi_t = rng.standard_normal((nt, M))
    return field, xi_t, field(xi_t)


def test_modes_orthonormal_and_energy_rule():
    field, xi_t, Y = _poly_snapshots(nt=40, M=3, p=2, dim=50, modes=6, seed=0)
    sur = build_surrogate(Y, xi_t, 2, 1e-10)
    G = sur.G
    assert np.allclose(G @ G.T, np.eye(G.shape[0]), atol=1e-10)
    # 6 generating directions -> rank 6 after mean removal; eps 1e-10 keeps them all
    assert sur.MQ == 6
    assert np.all(np.diff(sur.lam) <= 0)


def test_exact_recovery_of_polynomial_coefficients():
    # snapshots u(xi) = mean + sum_k c_k(xi) q_k with deg c_k <= p are in the
    # model class of Algorithm 3: the guess must reproduce u at NEW xi exactly
    field, xi_t, Y = _poly_snapshots(nt=60, M=3, p=2, dim=80, modes=5, seed=1)
    sur = build_surrogate(Y, xi_t, 2, 1e-12)
    xi_new = np.random.default_rng(9).standard_normal((7, 3))
    assert np.allclose(sur.guess(xi_new), field(xi_new), rtol=1e-9, atol=1e-9)


def test_training_snapshots_reconstructed_with_full_rank():
    # with M_Q = n_t - 1 and exact zeta (sqrt(n_t) e_k^j), step 6 without the LS
    # fit reproduces every training snapshot (completeness of the KL basis)
    rng = np.random.default_rng(2)
    nt, dim = 12, 40
    Y = rng.standard_normal((nt, dim))
    xi_t = rng.standard_normal((nt, 2))
    sur = build_surrogate(Y, xi_t, 1, 0.0)
    assert sur.MQ == nt - 1
    ubar = Y.mean(0)
    zeta = ((Y - ubar) @ sur.G.T) / np.sqrt(sur.lam)
    rec = ubar + (zeta * np.sqrt(sur.lam)) @ sur.G
    assert np.allclose(rec, Y, atol=1e-10)
    # zeta_k(xi_j) equals sqrt(n_t) times the eigenvector entry (eqs. KLE basis/parameter)
    C = ((Y - ubar) @ (Y - ubar).T) / nt
    lam, E = np.linalg.eigh(C)
    e0 = E[:, -1]
    z0 = zeta[:, 0]
    s = np.sign(z0 @ e0)
    assert np.allclose(z0, s * np.sqrt(nt) * e0, atol=1e-9)
