"""Learned initial guess (MLP) on the GPU against the FP64 oracle.

The network's GEMMs use BF16 operands with FP32 accumulation, so its
gradients are compared with the oracle's FP64 gradients at BF16 level
(relative L2 per parameter block <= 5e-2, cosine >= 0.999) on the same
(BF16-representable) weights.  Grid maps and the guess assembly are FP32 and
compared at 1e-6.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from synth import draw_xi
from tests.gpu_util import gpu_solver, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _bf16_weights(theta, sizes):
    """Weights rounded to BF16 (the GPU's GEMM operands), biases kept FP32."""
    tb = torch.from_numpy(theta.astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    k = 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        k += o * i
        tb[k:k + o] = theta[k:k + o]
        k += o
    return tb


def _bars(sizes):
    """Per-block bars on the relative L2 error of a BF16 gradient (weights,
    bias of layer l = 1..L).  BF16 keeps 8 significant bits (unit roundoff
    u = 2^-9); every GEMM rounds both operands to BF16, so the gradient of
    layer l carries about 2u from its own product and 2u from each of the
    L - l layers the backward pass crosses (their weights and the incoming
    gradient), plus the forward activations it multiplies: (L - l + 2) 2u,
    doubled for the sums' own spread: 2^-8 (L - l + 2), 1.95e-2 for the first
    of four layers down to 7.8e-3 for the last."""
    L = len(sizes) - 1
    out = []
    for l in range(1, L + 1):
        out += [2.0 ** -8 * (L - l + 2)] * 2
    return out


def test_gradient_matches_fp64_oracle():
    solver, w = gpu_solver("heat1d_nx63")
    sizes = omlp.layer_sizes(w.M, w.N)
    assert solver.mlp_n_params() == omlp.n_params(sizes)
    theta = _bf16_weights(omlp.init_params(sizes, 7), sizes)
    solver.mlp_set(theta)
    B = 50
    xi = draw_xi(B, w.M, 91)
    tg = (np.random.default_rng(3).standard_normal((B, w.N * 64)) * 0.5).astype(np.float32)
    grad = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    loss = solver.mlp_loss_grad(T(xi), T(tg), B, grad)
    lo, go = omlp.loss_and_grad(theta.astype(np.float64), sizes, xi, tg.astype(np.float64))
    assert abs(loss - lo) <= 1e-3 * lo
    errs = _block_errors(grad.cpu().numpy(), go, sizes)
    print("per-block relative L2 / cosine:", [(f"{e:.2e}", f"{c:.5f}") for e, c in errs])
    for (e, c), bar in zip(errs, _bars(sizes)):
        assert e <= bar and c >= 0.999


def test_grid_maps_match_oracle():
    solver, w = gpu_solver("heat1d_nx63")
    S = 3
    U = np.random.default_rng(5).standard_normal((S, w.N, w.nx))
    Td = torch.empty((S, w.N, 64), dtype=torch.float32, device="cuda")
    solver.downsample(T(U), S, w.N, Td)
    ref = omlp.downsample(U)
    assert np.abs(Td.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    # a network whose output is the constant b4 gives upsample(mean + std * b4)
    sizes = omlp.layer_sizes(w.M, w.N)
    theta = np.zeros(omlp.n_params(sizes), dtype=np.float32)
    rng = np.random.default_rng(6)
    y = rng.standard_normal(w.N * 64).astype(np.float32)
    theta[-w.N * 64:] = y
    mean = rng.standard_normal(w.N * 64).astype(np.float32)
    std = (0.5 + rng.random(w.N * 64)).astype(np.float32)
    solver.mlp_set(theta, mean, std)
    G = torch.empty((2, w.N, w.nx), dtype=torch.float64, device="cuda")
    solver.mlp_guess(T(draw_xi(2, w.M, 1)), 2, G)
    expect = omlp.upsample((mean.astype(np.float64) + std * y).reshape(w.N, 64), w.nx)
    for s in range(2):
        assert np.abs(G[s].cpu().numpy() - expect).max() <= 1e-6 * np.abs(expect).max()


def test_nonfinite_network_falls_back_to_gpc():
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx63")
    sizes = omlp.layer_sizes(w.M, w.N)
    theta = omlp.init_params(sizes, 2).astype(np.float32)
    theta[-1] = np.nan
    solver.mlp_set(theta)
    S = 6
    xi = T(draw_xi(S, w.M, 8))
    G = torch.empty((S, w.N, w.nx), dtype=torch.float64, device="cuda")
    assert solver.mlp_guess(xi, S, G) == pkg.E_NONFINITE
    U = torch.empty_like(G)
    it_m = torch.empty(S, dtype=torch.int32, device="cuda")
    it_g = torch.empty_like(it_m)
    dT = w.T / w.N
    assert solver.solve(xi, S, dT, w.J, w.N, w.alpha, w.tol, w.kmax, 0, pkg.GUESS_MLP, U, it_m) == 0
    U2 = torch.empty_like(G)
    assert solver.solve(xi, S, dT, w.J, w.N, w.alpha, w.tol, w.kmax, 0, pkg.GUESS_GPC, U2, it_g) == 0
    assert torch.equal(it_m, it_g) and torch.equal(U, U2)


@pytest.mark.parametrize("residual", [0, 1], ids=["direct", "residual"])
def test_training_learns_and_the_learned_guess_converges(residual):
    """Trains on 2048 references of the Nx=1023, N=64 problem and reports
    what the learned guess gains over the method's own surrogate and over a
    zero guess on 128 held-out samples (printed; the fixed point is the same).
    In residual mode the network learns the surrogate's error, and its guess
    must beat the surrogate's."""
    import paper_2510_26180_gb300 as pkg
    solver, w = gpu_solver("heat1d_nx1023")
    solver.mlp_set_residual(residual)
    try:
        _train_and_compare(pkg, solver, w, residual)
    finally:
        solver.mlp_set_residual(0)


def _train_and_compare(pkg, solver, w, residual):
    sizes = omlp.layer_sizes(w.M, w.N)
    ntr, nte = 2048, 128
    xtr, xte = T(draw_xi(ntr, w.M, 5)), T(draw_xi(nte, w.M, 6))
    Utr = torch.empty((ntr, w.N, w.nx), dtype=torch.float64, device="cuda")
    Ute = torch.empty((nte, w.N, w.nx), dtype=torch.float64, device="cuda")
    solver.reference(xtr, ntr, w.N, w.J, Utr)
    solver.reference(xte, nte, w.N, w.J, Ute)
    Ttr = torch.empty((ntr, w.N, 64), dtype=torch.float32, device="cuda")
    solver.mlp_targets(xtr, Utr, ntr, Ttr)
    if not residual:
        Tds = torch.empty_like(Ttr)
        solver.downsample(Utr, ntr, w.N, Tds)
        assert torch.equal(Ttr, Tds)
    solver.mlp_set(omlp.init_params(sizes, 11).astype(np.float32))
    losses = solver.mlp_train(xtr, Ttr, ntr, 60, 256, 1e-3, 1e-5, 1, True)
    # the surrogate's error is the harder target (what a degree-3 polynomial
    # in xi misses): its normalized loss falls less
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0] / (2 if residual else 20)
    G = torch.empty_like(Ute)
    assert solver.mlp_guess(xte, nte, G) == 0
    err = ((G - Ute).flatten(1).norm(dim=1) / Ute.flatten(1).norm(dim=1)).cpu().numpy()
    assert err.mean() < 0.1
    Gg = torch.empty_like(Ute)
    solver.guess(xte, nte, 0, Gg)
    err_gpc = ((Gg - Ute).flatten(1).norm(dim=1) / Ute.flatten(1).norm(dim=1)).cpu().numpy()
    if residual:
        assert err.mean() < err_gpc.mean(), (err.mean(), err_gpc.mean())
    U = torch.empty_like(Ute)
    it = torch.empty(nte, dtype=torch.int32, device="cuda")
    dT = w.T / w.N
    means = {}
    for name, gk in (("gpc", pkg.GUESS_GPC), ("mlp", pkg.GUESS_MLP), ("zero", pkg.GUESS_ZERO)):
        code = solver.solve(xte, nte, dT, w.J, w.N, w.alpha, w.tol, w.kmax, 2, gk, U, it)
        assert code == 0
        e = ((U - Ute).flatten(1).norm(dim=1) / Ute.flatten(1).norm(dim=1)).max().item()
        assert e <= 1e-6
        means[name] = float(it.float().mean())
    print(f"held-out ({'residual' if residual else 'direct'}): learned-guess error "
          f"{err.mean():.3e}, gPC {err_gpc.mean():.3e}, mean iterations {means}")


def _block_errors(gg, go, sizes):
    out = []
    k = 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        for n in (o * i, o):
            a, b = gg[k:k + n], go[k:k + n]
            k += n
            out.append((np.linalg.norm(a - b) / np.linalg.norm(b),
                        a @ b / (np.linalg.norm(a) * np.linalg.norm(b))))
    return out


def test_gradient_at_batch_256_on_tcgen05_matches_fp64_oracle():
    # batch 256: the products of the hidden and output layers run on the
    # tcgen05 tensor cores (M, K >= 64); the same derived bars as the small
    # batch
    solver, w = gpu_solver("heat1d_nx63")
    sizes = omlp.layer_sizes(w.M, w.N)
    theta = _bf16_weights(omlp.init_params(sizes, 8), sizes)
    solver.mlp_set(theta)
    B = 256
    xi = draw_xi(B, w.M, 92)
    tg = (np.random.default_rng(4).standard_normal((B, w.N * 64)) * 0.5).astype(np.float32)
    grad = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    loss = solver.mlp_loss_grad(T(xi), T(tg), B, grad)
    lo, go = omlp.loss_and_grad(theta.astype(np.float64), sizes, xi, tg.astype(np.float64))
    assert abs(loss - lo) <= 1e-3 * lo
    errs = _block_errors(grad.cpu().numpy(), go, sizes)
    print("per-block relative L2 / cosine:", [(f"{e:.2e}", f"{c:.5f}") for e, c in errs])
    for (e, c), bar in zip(errs, _bars(sizes)):
        assert e <= bar and c >= 0.999


def test_guess_at_512_samples_on_tcgen05_matches_oracle_forward():
    solver, w = gpu_solver("heat1d_nx63")
    sizes = omlp.layer_sizes(w.M, w.N)
    theta = _bf16_weights(omlp.init_params(sizes, 9), sizes)
    rng = np.random.default_rng(8)
    mean = rng.standard_normal(w.N * 64).astype(np.float32)
    std = (0.5 + rng.random(w.N * 64)).astype(np.float32)
    solver.mlp_set(theta, mean, std)
    S = 512
    xi = draw_xi(S, w.M, 93)
    G = torch.empty((S, w.N, w.nx), dtype=torch.float64, device="cuda")
    solver.mlp_guess(T(xi), S, G)
    G = G.cpu().numpy()
    Y = omlp.forward(theta.astype(np.float64), sizes, xi)[2]
    worst = 0.0
    for s in range(0, S, 37):
        expect = omlp.upsample((mean + std * Y[s]).reshape(w.N, 64), w.nx)
        worst = max(worst, rel(G[s], expect))
    print("worst relative L2 of the guess:", worst)
    assert worst <= 2e-2
