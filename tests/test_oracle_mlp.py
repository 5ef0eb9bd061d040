"""Pins of the oracle's MLP, Adam and grid maps (no GPU)."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    sizes = [3, 5, 4, 4, 6]
    theta = mlp.init_params(sizes, 3) + 0.05
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 3))
    T = rng.standard_normal((7, 6))
    _, g = mlp.loss_and_grad(theta, sizes, X, T)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        num[k] = (mlp.loss_and_grad(theta + e, sizes, X, T)[0]
                  - mlp.loss_and_grad(theta - e, sizes, X, T)[0]) / (2 * h)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-9)
    assert mlp.n_params(sizes) == theta.size


def test_parameter_count_of_the_workload_network():
    assert mlp.n_params(mlp.layer_sizes(10, 64)) == 1_187_072


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2: the update is -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    opt = mlp.Adam(3, lr=0.01)
    th = opt.step(np.zeros(3), g)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_grid_maps_interpolation_error_bound():
    # linear interpolation error <= h^2/8 max|f''| for f = sin(pi x)
    nx = 1023
    x = np.arange(1, nx + 1) / (nx + 1)
    f = np.sin(np.pi * x)
    d = mlp.downsample(f)
    xc = mlp.coarse_points()
    hg = 1 / (nx + 1)
    assert np.max(np.abs(d - np.sin(np.pi * xc))) <= hg ** 2 / 8 * np.pi ** 2 + 1e-15
    u = mlp.upsample(np.sin(np.pi * xc), nx)
    hc = 1 / 65
    assert np.max(np.abs(u - f)) <= hc ** 2 / 8 * np.pi ** 2 + 1e-15
    # piecewise-linear data on the coarse nodes is reproduced exactly at the nodes
    y = np.random.default_rng(2).standard_normal(64)
    up = mlp.upsample(y, 64 * 65 - 1)   # grid containing every coarse node
    idx = (np.arange(64) + 1) * 64 - 1
    assert np.allclose(up[idx], y, atol=1e-14)


def test_forward_on_hand_set_weights():
    # M = 1 -> 2 -> 2 -> 2 -> 1 with r1 = relu(x - 1/2), r2 = relu(-x):
    # W2 = [[1, 0], [1, 1]] (stored [out][in]) gives (r1, r1 + r2), W3 = I,
    # W4 = [2, 3], b4 = -10: f(x) = 5 r1 + 3 r2 - 10, negative (no ReLU on the
    # output).  A transposed W2 would give 2 r1 + 5 r2 - 10.
    sizes = [1, 2, 2, 2, 1]
    theta = np.concatenate([
        [1.0, -1.0], [-0.5, 0.0],                 # W1 [2][1], b1
        [1.0, 0.0, 1.0, 1.0], [0.0, 0.0],         # W2 [2][2], b2
        [1.0, 0.0, 0.0, 1.0], [0.0, 0.0],         # W3, b3
        [2.0, 3.0], [-10.0],                      # W4 [1][2], b4
    ])
    assert theta.size == mlp.n_params(sizes)
    X = np.array([[1.0], [-2.0], [0.2], [0.5]])
    _, _, Y = mlp.forward(theta, sizes, X)
    assert np.array_equal(Y[:, 0], np.array([-7.5, -4.0, -10.0, -10.0]))
